"""Pins of the oracle's staggered Stokes inverse (Sec. 2, Eq. 8-9, the three-step
algorithm and the preconditioned Krylov solve of the pressure matrix)."""
import numpy as np
import pytest

from oracle import assembled as asm
from oracle import stokes as st
from workloads import box_faces, mac_shapes, rhs_gaussian, tanh_faces


def _faces():
    return [tanh_faces(4, 1.5), tanh_faces(5, 1.5), tanh_faces(6, 2.0)]


def _forcing(faces, seed=0):
    vs, _ = st.shapes(faces)
    return [rhs_gaussian(vs[c], seed + c) for c in range(3)]


def test_shapes_match_workloads():
    faces = _faces()
    vs, ps = st.shapes(faces)
    ms = mac_shapes((4, 5, 6))
    assert vs == [ms["u"], ms["v"], ms["w"]] and ps == ms["p"]


@pytest.mark.parametrize("dt", [1e-2, 1.0, 1e3])
def test_direct_solve_residual_and_divergence(dt):
    faces = _faces()
    f = _forcing(faces)
    vel, p = st.stokes_direct(faces, dt, 1000.0, f)
    mom, div = st.saddle_residual(faces, dt, 1000.0, f, vel, p)
    assert mom < 1e-12 and div < 1e-12
    vol = asm.volumes(st.pressure_ops(faces))
    assert abs(np.dot(vol, p.ravel())) < 1e-12 * np.abs(p).max()


def test_manufactured_pressure_only():
    # f = dt * G p0 with zero-mean p0 has the exact solution u = 0, p = p0
    faces = _faces()
    dt = 0.5
    _, ps = st.shapes(faces)
    vol = asm.volumes(st.pressure_ops(faces))
    p0 = rhs_gaussian(ps, 11).ravel()
    p0 -= np.dot(vol, p0) / vol.sum()
    D, G = st.div_grad_3d(faces)
    vs, _ = st.shapes(faces)
    f = [(dt * (G[c] @ p0)).reshape(vs[c]) for c in range(3)]
    vel, p = st.stokes_direct(faces, dt, 100.0, f)
    assert max(np.abs(v).max() for v in vel) < 1e-11 * np.abs(p0).max()
    assert np.abs(p.ravel() - p0).max() < 1e-11 * np.abs(p0).max()


def test_manufactured_divergence_free_velocity():
    # u = v - G (DG)^+ D v is discretely divergence free; with p0 it gives
    # f = H u + dt G p0 and the solve must return (u, p0)
    faces = _faces()
    dt, Re = 2.0, 50.0
    lam = dt / Re
    D, G = st.div_grad_3d(faces)
    vs, ps = st.shapes(faces)
    vol = asm.volumes(st.pressure_ops(faces))
    v = [rhs_gaussian(vs[c], 20 + c).ravel() for c in range(3)]
    Lp = sum((D[c] @ G[c]).toarray() for c in range(3))
    dv = sum(D[c] @ v[c] for c in range(3))
    phi = np.linalg.lstsq(Lp, dv, rcond=None)[0]
    u = [v[c] - G[c] @ phi for c in range(3)]
    assert np.abs(sum(D[c] @ u[c] for c in range(3))).max() < 1e-10
    p0 = rhs_gaussian(ps, 30).ravel()
    p0 -= np.dot(vol, p0) / vol.sum()
    f = [(asm.helmholtz(st.component_ops(faces, c), lam) @ u[c] + dt * (G[c] @ p0)).reshape(vs[c])
         for c in range(3)]
    vel, p = st.stokes_direct(faces, dt, Re, f)
    for c in range(3):
        assert np.abs(vel[c].ravel() - u[c]).max() < 1e-10 * np.abs(u[c]).max()
    assert np.abs(p.ravel() - p0).max() < 1e-10 * np.abs(p0).max()


@pytest.mark.parametrize("dt", [1e-2, 1e3])
def test_three_step_equals_direct(dt):
    faces = _faces()
    f = _forcing(faces, 5)
    vel_d, p_d = st.stokes_direct(faces, dt, 1000.0, f)
    vel_t, p_t = st.stokes_three_step_dense(faces, dt, 1000.0, f)
    for c in range(3):
        assert np.abs(vel_t[c] - vel_d[c]).max() < 1e-10 * np.abs(vel_d[c]).max()
    assert np.abs(p_t - p_d).max() < 1e-9 * np.abs(p_d).max()


@pytest.mark.parametrize("dt", [1e-2, 1.0, 1e3])
def test_semi_direct_bicgstab_equals_direct(dt):
    faces = _faces()
    f = _forcing(faces, 9)
    vel_d, p_d = st.stokes_direct(faces, dt, 1000.0, f)
    vel, p, it, rel = st.stokes_semi_direct(faces, dt, 1000.0, f, tol=1e-12)
    assert rel <= 1e-12 and it < 60
    for c in range(3):
        assert np.abs(vel[c] - vel_d[c]).max() < 1e-9 * np.abs(vel_d[c]).max()
    assert np.abs(p - p_d).max() < 1e-8 * np.abs(p_d).max()


def test_chorin_limit():
    # dt -> 0: H -> I and C -> D G, the pressure Laplacian (Sec. 2, after Eq. 9)
    faces = _faces()
    D, G = st.div_grad_3d(faces)
    Lp = sum((D[c] @ G[c]).toarray() for c in range(3))
    errs = []
    for dt in (1e-4, 1e-5, 1e-6):
        C = st.pressure_matrix(faces, dt, 1.0)
        errs.append(np.abs(C - Lp).max() / np.abs(Lp).max())
    errs = np.array(errs)
    assert errs[-1] < 1e-2 and np.all(errs[:-1] / errs[1:] > 5.0), errs


def test_pressure_matrix_is_volume_self_adjoint_not_symmetric():
    # C is not symmetric as a plain matrix on a stretched grid (Sec. 2), but V*C is
    # symmetric because D = -V^{-1} G^T M_u
    faces = _faces()
    C = st.pressure_matrix(faces, 0.3, 10.0)
    vol = asm.volumes(st.pressure_ops(faces))
    VC = vol[:, None] * C
    assert np.abs(VC - VC.T).max() < 1e-11 * np.abs(VC).max()
    assert np.abs(C - C.T).max() > 1e-6 * np.abs(C).max()
    # singular: constants are in the null space
    assert np.abs(C @ np.ones(C.shape[0])).max() < 1e-10 * np.abs(C).max()


def test_preconditioned_iterations_small_at_small_dt():
    # with the pressure-Laplacian preconditioner C is close to identity at small dt
    faces = [tanh_faces(8, 1.5)] * 3
    f = _forcing(faces, 2)
    _, _, it_small, _ = st.stokes_semi_direct(faces, 1e-2, 1000.0, f, tol=1e-10)
    assert it_small <= 3


@pytest.mark.parametrize("dt", [1e-2, 1.0, 1e3])
def test_cahouet_chabard_preconditioner_equals_direct(dt):
    # the viscous-corrected preconditioner changes the iteration, not the answer
    faces = _faces()
    f = _forcing(faces, 13)
    vel_d, p_d = st.stokes_direct(faces, dt, 1000.0, f)
    vel, p, it, rel = st.stokes_semi_direct(faces, dt, 1000.0, f, tol=1e-12, precond="cahouet-chabard")
    assert rel <= 1e-12
    for c in range(3):
        assert np.abs(vel[c] - vel_d[c]).max() < 1e-9 * np.abs(vel_d[c]).max()
    assert np.abs(p - p_d).max() < 1e-8 * np.abs(p_d).max()


def test_cahouet_chabard_exact_on_uniform_periodic_analogue():
    # with commuting operators C = L (I - lam L)^{-1}; check that L^{-1} - lam I inverts it
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    mu = -np.linspace(0.5, 40.0, 12)
    L = Q @ np.diag(mu) @ Q.T
    lam = 0.7
    C = L @ np.linalg.inv(np.eye(12) - lam * L)
    P = np.linalg.inv(L) - lam * np.eye(12)
    assert np.abs(P @ C - np.eye(12)).max() < 1e-12


def test_bicgstab_l_with_l1_is_bicgstab():
    # BiCGstab(1) and van der Vorst's BiCGstab generate the same iterates: two
    # independent formulations of the method agree step by step
    rng = np.random.default_rng(0)
    n = 30
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    Md = np.diag(A).copy()
    b = rng.standard_normal(n)
    for k in (1, 2, 3, 5, 8):
        x1, _, r1 = st.bicgstab(lambda v: A @ v, lambda v: v / Md, b, 0.0, k)
        xl, _, rl = st.bicgstab_l(lambda v: A @ v, lambda v: v / Md, b, 1, 0.0, k)
        assert np.abs(x1 - xl).max() <= 1e-12 * np.abs(x1).max()
        assert abs(r1 - rl) <= 1e-10 * r1 + 1e-14


@pytest.mark.parametrize("ell", [2, 3])
def test_bicgstab_l_solves_nonsymmetric(ell):
    rng = np.random.default_rng(ell)
    n = 40
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.25
    b = rng.standard_normal(n)
    x, it, rel = st.bicgstab_l(lambda v: A @ v, lambda v: v, b, ell, 1e-13, 200)
    assert rel <= 1e-12
    assert np.abs(x - np.linalg.solve(A, b)).max() <= 1e-10 * np.abs(np.linalg.solve(A, b)).max()


@pytest.mark.parametrize("dt", [1e-2, 1.0, 1e3])
@pytest.mark.parametrize("precond", ["laplace", "cahouet-chabard"])
def test_semi_direct_bicgstab2_matches_direct(dt, precond):
    # the paper's Krylov solver (Sec. 2) inside the three-step algorithm
    faces = [tanh_faces(6, 1.5), tanh_faces(7, 1.5), tanh_faces(8, 2.0)]
    vs, ps = st.shapes(faces)
    f = [rhs_gaussian(vs[c], c) for c in range(3)]
    vd, pd = st.stokes_direct(faces, dt, 1000.0, f)
    v, p, it, rel = st.stokes_semi_direct(faces, dt, 1000.0, f, tol=1e-12, precond=precond, krylov="bicgstab2")
    assert rel <= 1e-12
    for c in range(3):
        assert np.abs(v[c] - vd[c]).max() <= 1e-10 * np.abs(vd[c]).max()
    assert np.abs(p - pd).max() <= 1e-9 * np.abs(pd).max()


def _weighted_spd(n, seed):
    # A = W^{-1} S with S symmetric positive definite: self-adjoint and positive
    # definite in the inner product weighted by W
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.2, 3.0, n)
    X = rng.standard_normal((n, n))
    S = X @ X.T + n * np.eye(n)
    return w, S / w[:, None]


def test_pcg_solves_weighted_spd_system():
    # against the dense solve, with and without a (weighted-SPD) preconditioner
    w, A = _weighted_spd(40, 3)
    b = np.random.default_rng(4).standard_normal(40)
    ref = np.linalg.solve(A, b)
    d = np.diag(A)
    for B in (lambda v: v, lambda v: v / d):
        x, it, rel = st.pcg(lambda v: A @ v, B, b, w, 1e-13, 200)
        assert rel <= 1e-13 and it <= 40
        assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()


def test_pcg_exact_preconditioner_converges_in_one_step():
    w, A = _weighted_spd(25, 5)
    Ainv = np.linalg.inv(A)
    b = np.random.default_rng(6).standard_normal(25)
    x, it, rel = st.pcg(lambda v: A @ v, lambda v: Ainv @ v, b, w, 1e-12, 10)
    assert it == 1 and rel <= 1e-12


def test_pcg_energy_error_decreases_and_terminates():
    # CG minimises the A-norm of the error over the Krylov space in the weighted
    # inner product: that norm never increases, and with n distinct eigenvalues the
    # iteration ends within n steps (up to rounding)
    n = 12
    w, A = _weighted_spd(n, 7)
    b = np.random.default_rng(8).standard_normal(n)
    ref = np.linalg.solve(A, b)
    errs = []
    for k in range(1, n + 1):
        x, _, _ = st.pcg(lambda v: A @ v, lambda v: v, b, w, 0.0, k)
        e = x - ref
        errs.append(float(np.sum(w * e * (A @ e))))
    errs = np.array(errs)
    assert np.all(errs[1:] <= errs[:-1] * (1 + 1e-9))
    assert errs[-1] <= 1e-20 * float(np.sum(w * ref * (A @ ref)))
    # the Euclidean inner product is the wrong one for this A: its iterates lose
    # the monotone energy error or fail to terminate in n steps
    bad = []
    for k in range(1, n + 1):
        x, _, _ = st.pcg(lambda v: A @ v, lambda v: v, b, np.ones(n), 0.0, k)
        e = x - ref
        bad.append(float(np.sum(w * e * (A @ e))))
    bad = np.array(bad)
    assert bad[-1] > 1e3 * errs[-1] or np.any(bad[1:] > bad[:-1] * (1 + 1e-9))


@pytest.mark.parametrize("dt", [1e-2, 1.0, 1e3])
@pytest.mark.parametrize("precond", ["laplace", "cahouet-chabard"])
def test_semi_direct_cg_matches_direct(dt, precond):
    # -C is self-adjoint positive definite on zero-mean pressures in the
    # volume-weighted inner product, so CG applies to the pressure system
    faces = [tanh_faces(6, 1.5), tanh_faces(7, 1.5), tanh_faces(8, 2.0)]
    vs, ps = st.shapes(faces)
    f = [rhs_gaussian(vs[c], 20 + c) for c in range(3)]
    vd, pd = st.stokes_direct(faces, dt, 1000.0, f)
    v, p, it, rel = st.stokes_semi_direct(faces, dt, 1000.0, f, tol=1e-12, precond=precond, krylov="cg")
    assert rel <= 1e-12
    for c in range(3):
        assert np.abs(v[c] - vd[c]).max() <= 1e-10 * np.abs(vd[c]).max()
    assert np.abs(p - pd).max() <= 1e-9 * np.abs(pd).max()


def test_cg_with_exact_pressure_inverse_takes_one_step():
    # preconditioned by the exact inverse of -C on zero-mean pressures (dense
    # pseudo-inverse), CG ends after one step: pins the sign conventions
    faces = _faces()
    dt, Re = 0.5, 10.0
    C = st.pressure_matrix(faces, dt, Re)
    vol = asm.volumes(st.pressure_ops(faces))
    P = np.eye(len(vol)) - np.outer(np.ones(len(vol)), vol) / vol.sum()  # zero-mean projector
    Cp = np.linalg.pinv(-C @ P) @ P
    b = np.random.default_rng(13).standard_normal(len(vol))
    b -= np.dot(vol, b) / vol.sum()
    x, it, rel = st.pcg(lambda v: -C @ v, lambda v: P @ (Cp @ v), -b, vol, 1e-10, 5)
    assert it == 1 and rel <= 1e-10
