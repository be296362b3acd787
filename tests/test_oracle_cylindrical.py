"""Pins of the oracle's cylindrical-coordinate operators and their eigen
decomposition inverses (Sec. 6, Eq. 41-46)."""
import numpy as np
import pytest

from oracle import cylindrical as cy
from workloads import tanh_faces

D, N = cy.DIRICHLET, cy.NEUMANN


def annulus(n, a=0.5, b=1.5, beta=1.5):
    return a + (b - a) * tanh_faces(n, beta)


def test_periodic_operator_fourier_eigenvalues():
    # uniform periodic second difference: Lambda_k = -(4/h^2) sin^2(pi k / M)
    M = 12
    m, K = cy.periodic_operator(M)
    h = 2 * np.pi / M
    lam = np.sort(np.linalg.eigvalsh(K / h))
    ref = np.sort(-(4.0 / h ** 2) * np.sin(np.pi * np.arange(M) / M) ** 2)
    assert np.abs(lam - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("axis", [False, True])
def test_radial_operator_structure(axis):
    rf = tanh_faces(20, 1.2) if axis else annulus(20)
    A, K, g = cy.radial_operator(rf, N, N)
    assert np.abs(K - K.T).max() == 0.0
    # zero-flux walls (or the axis and a zero-flux wall): constants are the null space
    assert np.abs(K.sum(axis=1)).max() <= 1e-12 * np.abs(K).max()
    # A sums to the annular area of the whole radial interval
    assert abs(A.sum() - 0.5 * (rf[-1] ** 2 - rf[0] ** 2)) <= 1e-14
    # the discrete 1/r^2 tends to 1/c^2 at second order in h / c
    h = np.diff(rf)
    c = 0.5 * (rf[1:] + rf[:-1])
    assert np.all(np.abs(g * c * c - 1.0) <= 0.5 * (h / c) ** 2 + 1e-14)


def test_radial_operator_is_the_divergence_form():
    # for u = r^2: (1/r)(r u')' = 4 exactly in the interior (linear flux profile)
    rf = annulus(16)
    A, K, g = cy.radial_operator(rf, N, N)
    c = 0.5 * (rf[1:] + rf[:-1])
    Du = (K @ (c * c)) / A
    # the two-point gradient of r^2 is exact at face midpoints of the centres;
    # interior rows reproduce 4 up to the face/centre offset of a stretched grid
    assert np.abs(Du[1:-1] - 4.0).max() <= 0.1


CASES = [
    (annulus(9), (D, D), (D, D), 1.0, 1.0),
    (annulus(7), (N, D), (D, N), 1e-3, 1.0),
    (annulus(8), (D, N), (N, N), 1.0, 0.0),
    (tanh_faces(8, 1.2), (N, D), (D, D), 0.3, 1.0),    # full cylinder: the axis
    (tanh_faces(6, 1.2), (N, N), (D, N), 1.0, 1.0),
]


@pytest.mark.parametrize("rf,bc_r,bc_z,lam,sigma", CASES)
def test_tpt_and_tpf_equal_the_direct_solve(rf, bc_r, bc_z, lam, sigma):
    # Eq. 44 (Thomas per mode pair) and Eq. 46 (radial eigen per theta mode)
    # against the sparse direct solve of the assembled operator
    M = 10
    zf = tanh_faces(7, 1.5)
    shape = (len(zf) - 1, M, len(rf) - 1)
    f = np.random.default_rng(3).uniform(-1, 1, shape)
    ref = cy.direct_solve(f, rf, M, zf, lam, sigma, bc_r, bc_z)
    for solver in (cy.tpt_solve, cy.tpf_solve):
        got = solver(f, rf, M, zf, lam, sigma, bc_r, bc_z)
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), solver.__name__


def test_singular_laplacian_rejected():
    with pytest.raises(ValueError):
        cy.tpt_solve(np.zeros((4, 6, 5)), annulus(5), 6, tanh_faces(4, 1.0), 1.0, 0.0, (N, N), (N, N))


def _manufactured_error(n, sigma, lam, axis):
    # u = R(r) cos(2 theta) sin(pi z) with R vanishing on the radial wall(s);
    # f = sigma u - lam (u_rr + u_r / r - 4 u / r^2 + u_zz)
    M = 4 * n
    zf = tanh_faces(n, 1.3)
    if axis:
        rf = tanh_faces(n, 1.0)[:]            # [0, 1], axis at r = 0
        # R = r^2 (1 - r^2): regular at the axis for the mode cos(2 theta)
        R = lambda r: r ** 2 * (1 - r ** 2)  # noqa: E731
        R1 = lambda r: 2 * r - 4 * r ** 3  # noqa: E731
        R2 = lambda r: 2 - 12 * r ** 2  # noqa: E731
        bc_r = (N, D)
    else:
        a, b = 0.5, 1.5
        rf = annulus(n, a, b, 1.3)
        k = np.pi / (b - a)
        R = lambda r: np.sin(k * (r - a))  # noqa: E731
        R1 = lambda r: k * np.cos(k * (r - a))  # noqa: E731
        R2 = lambda r: -k * k * np.sin(k * (r - a))  # noqa: E731
        bc_r = (D, D)
    c = 0.5 * (rf[1:] + rf[:-1])
    th = (np.arange(M) + 0.5) * 2 * np.pi / M
    zc = 0.5 * (zf[1:] + zf[:-1])
    Z, T, Rr = np.meshgrid(zc, th, c, indexing="ij")
    u = R(Rr) * np.cos(2 * T) * np.sin(np.pi * Z)
    lap = (R2(Rr) + R1(Rr) / Rr - 4 * R(Rr) / Rr ** 2 - np.pi ** 2 * R(Rr)) * np.cos(2 * T) * np.sin(np.pi * Z)
    f = sigma * u - lam * lap
    got = cy.tpt_solve(f, rf, M, zf, lam, sigma, bc_r, (D, D))
    return np.abs(got - u).max() / np.abs(u).max()


@pytest.mark.parametrize("axis", [False, True])
def test_second_order_convergence_to_an_analytic_solution(axis):
    errs = [_manufactured_error(n, 1.0, 0.5, axis) for n in (8, 16, 32)]
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert errs[-1] < 5e-3 and all(r > 3.0 for r in ratios), (errs, ratios)


def _mutant_no_face_radius(rfaces, bc_in=D, bc_out=D):
    # planted mistake: Cartesian radial fluxes (the face radius dropped)
    A, K, g = _ORIG_RADIAL(rfaces, bc_in, bc_out)
    rho = np.asarray(rfaces, dtype=np.float64)
    h = np.diff(rho)
    c = 0.5 * (rho[1:] + rho[:-1])
    n = h.size
    K2 = np.zeros_like(K)
    for i in range(n - 1):
        w = 1.0 / (c[i + 1] - c[i])
        K2[i, i + 1] = K2[i + 1, i] = w
        K2[i, i] -= w
        K2[i + 1, i + 1] -= w
    if rho[0] > 0 and bc_in == D:
        K2[0, 0] -= 2.0 / h[0]
    if bc_out == D:
        K2[n - 1, n - 1] -= 2.0 / h[n - 1]
    return A, K2, g


def _mutant_theta_sign(rfaces, bc_in=D, bc_out=D):
    # planted mistake: the theta term with the wrong sign
    A, K, g = _ORIG_RADIAL(rfaces, bc_in, bc_out)
    return A, K, -g


_ORIG_RADIAL = cy.radial_operator


@pytest.mark.parametrize("mutant", [_mutant_no_face_radius, _mutant_theta_sign])
def test_planted_mistakes_fail_the_convergence_pin(monkeypatch, mutant):
    monkeypatch.setattr(cy, "radial_operator", mutant)
    errs = [_manufactured_error(n, 1.0, 0.5, False) for n in (8, 16, 32)]
    converges = errs[-1] < 5e-3 and all(errs[i] / errs[i + 1] > 3.0 for i in range(2))
    assert not converges, errs
