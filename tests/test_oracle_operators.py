"""Pins of the oracle's 1D operators and eigen decompositions (Sec. 3, Eq. 23-24;
Sec. 4, Eq. 30-31) against closed forms, identities and the continuum problem."""
import numpy as np
import pytest

from oracle import operators1d as o1
from oracle import decomposition as dec
from workloads import tanh_faces

D, N = o1.DIRICHLET, o1.NEUMANN


def _sorted_eig(m, K):
    lam, E, Einv = dec.generalized_eig(m, K)
    order = np.argsort(-lam)          # eigenvalues <= 0: closest to zero first
    return lam[order], E[:, order], Einv[order, :]


def _check_modes(E, modes):
    # every computed eigenvector is parallel to the closed-form one
    for k in range(modes.shape[1]):
        a = E[:, k] / np.linalg.norm(E[:, k])
        b = modes[:, k] / np.linalg.norm(modes[:, k])
        assert abs(abs(np.dot(a, b)) - 1.0) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 7, 16])
def test_uniform_cell_dirichlet_is_dst2(n):
    # uniform grid: eigenvalues -(4/h^2) sin^2(k pi / 2n), modes sin(k pi (i+1/2)/n), k=1..n
    h = 1.0 / n
    m, K = o1.cell_operator(tanh_faces(n, 0.0), D, D)
    lam, E, _ = _sorted_eig(m, K)
    k = np.arange(1, n + 1)
    assert np.allclose(lam, -(4 / h**2) * np.sin(k * np.pi / (2 * n)) ** 2, rtol=1e-13, atol=1e-10)
    i = np.arange(n) + 0.5
    _check_modes(E, np.sin(np.pi * np.outer(i, k) / n))


@pytest.mark.parametrize("n", [2, 9, 16])
def test_uniform_cell_neumann_is_dct2(n):
    h = 1.0 / n
    m, K = o1.cell_operator(tanh_faces(n, 0.0), N, N)
    lam, E, _ = _sorted_eig(m, K)
    k = np.arange(0, n)
    assert lam[0] == 0.0
    assert np.allclose(lam, -(4 / h**2) * np.sin(k * np.pi / (2 * n)) ** 2, rtol=1e-13, atol=1e-10)
    i = np.arange(n) + 0.5
    _check_modes(E, np.cos(np.pi * np.outer(i, k) / n))


@pytest.mark.parametrize("n", [2, 8, 17])
def test_uniform_face_dirichlet_is_dst1(n):
    h = 1.0 / n
    m, K = o1.face_operator(tanh_faces(n, 0.0))
    lam, E, _ = _sorted_eig(m, K)
    k = np.arange(1, n)
    assert np.allclose(lam, -(4 / h**2) * np.sin(k * np.pi / (2 * n)) ** 2, rtol=1e-13, atol=1e-10)
    j = np.arange(1, n)
    _check_modes(E, np.sin(np.pi * np.outer(j, k) / n))


def test_uniform_mixed_walls_quarter_wave():
    # Dirichlet at 0, Neumann at 1 on a uniform grid: modes sin((k-1/2) pi (i+1/2)/n),
    # eigenvalues -(4/h^2) sin^2((2k-1) pi / 4n)
    n = 11
    h = 1.0 / n
    m, K = o1.cell_operator(tanh_faces(n, 0.0), D, N)
    lam, E, _ = _sorted_eig(m, K)
    k = np.arange(1, n + 1)
    assert np.allclose(lam, -(4 / h**2) * np.sin((2 * k - 1) * np.pi / (4 * n)) ** 2, rtol=1e-13)
    i = np.arange(n) + 0.5
    _check_modes(E, np.sin(np.pi * np.outer(i, k - 0.5) / n))


@pytest.mark.parametrize("kind,bc", [("cell", (D, D)), ("cell", (N, N)), ("cell", (D, N)),
                                     ("cell", (N, D)), ("face", (D, D))])
@pytest.mark.parametrize("beta", [1.5, 2.0])
@pytest.mark.parametrize("n", [37, 64, 256])
def test_eigen_invariants_stretched(kind, bc, beta, n):
    # Eq. 24: D = E Lambda E^{-1}; M-orthonormal eigenvectors E^T M E = I
    m, K = o1.operator_for(tanh_faces(n, beta), kind, *bc)
    lam, E, Einv = dec.generalized_eig(m, K)
    Dm = o1.second_derivative(m, K)
    scale = np.abs(lam).max()
    assert np.abs(Dm @ E - E * lam[None, :]).max() <= 1e-12 * scale * np.abs(E).max()
    assert np.abs(E.T @ (m[:, None] * E) - np.eye(len(m))).max() < 1e-12
    assert np.abs(Einv @ E - np.eye(len(m))).max() < 1e-12
    assert np.all(lam <= 0.0)


def test_first_derivative_identities():
    # staggered div*grad is the zero-flux cell operator, grad*div the face operator
    f = tanh_faces(23, 1.7)
    Dv, Gr = o1.div_1d(f), o1.grad_1d(f)
    mc, Kc = o1.cell_operator(f, N, N)
    mf, Kf = o1.face_operator(f)
    assert np.allclose(Dv @ Gr, o1.second_derivative(mc, Kc), rtol=0, atol=1e-9)
    assert np.allclose(Gr @ Dv, o1.second_derivative(mf, Kf), rtol=0, atol=1e-9)
    # discrete divergence theorem: sum_i h_i (D u)_i = u_n - u_0 = 0
    h = np.diff(f)
    u = np.random.default_rng(0).standard_normal(22)
    assert abs(np.dot(h, Dv @ u)) < 1e-13 * np.abs(u).sum()


def _conv_errors(kind, bc, ns, beta):
    errs = []
    for n in ns:
        f = tanh_faces(n, beta)
        m, K = o1.operator_for(f, kind, *bc)
        h = np.diff(f)
        c = 0.5 * (f[:-1] + f[1:])
        x = c if kind == "cell" else f[1:-1]
        if bc == (D, D):
            u = np.sin(np.pi * x)
        elif bc == (N, N):
            u = np.cos(np.pi * x)
        else:
            u = np.sin(0.5 * np.pi * x)
        g = -np.pi**2 * u if bc != (D, N) else -(0.5 * np.pi) ** 2 * u
        Dm = o1.second_derivative(m, K)
        if bc == (N, N):
            # singular: solve on the zero-mean subspace, compare with the mean removed
            A = np.vstack([np.hstack([Dm, np.ones((n, 1))]), np.hstack([h[None, :], [[0.0]]])])
            gg = g - np.dot(h, g) / h.sum()
            sol = np.linalg.solve(A, np.concatenate([gg, [0.0]]))[:n]
            ref = u - np.dot(h, u) / h.sum()
        else:
            sol = np.linalg.solve(Dm, g)
            ref = u
        errs.append(np.abs(sol - ref).max())
    return np.array(errs)


@pytest.mark.parametrize("kind,bc", [("cell", (D, D)), ("cell", (N, N)), ("cell", (D, N)), ("face", (D, D))])
def test_second_order_convergence_to_continuum(kind, bc):
    # the discrete operators converge at second order to d2/dx2 with the stated walls
    errs = _conv_errors(kind, bc, [32, 64, 128], 1.5)
    ratios = errs[:-1] / errs[1:]
    assert np.all(ratios > 3.5), (errs, ratios)
    assert errs[-1] < 1e-3


def test_wrong_wall_distance_is_caught():
    # a plausible mistake (full-cell instead of half-cell wall distance) breaks the
    # convergence pin: the pin is sensitive to the wall treatment
    import oracle.operators1d as mod
    orig = mod.cell_operator

    def wrong(faces, bc_lo=D, bc_hi=D):
        m, K = orig(faces, bc_lo, bc_hi)
        h = np.diff(np.asarray(faces))
        if bc_lo == D:
            K[0, 0] += 2.0 / h[0] - 1.0 / h[0]
        if bc_hi == D:
            K[-1, -1] += 2.0 / h[-1] - 1.0 / h[-1]
        return m, K

    mod.cell_operator = wrong
    try:
        errs = _conv_errors("cell", (D, D), [32, 64, 128], 1.5)
    finally:
        mod.cell_operator = orig
    assert not np.all(errs[:-1] / errs[1:] > 3.5) or errs[-1] > 1e-3
