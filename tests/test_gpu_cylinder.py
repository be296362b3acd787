"""GPU cylindrical-coordinate inverses (Sec. 6, Eq. 41-46) through the C ABI
(fdi_plan_create_cyl), against the oracle's sparse direct solve (the plain
definition) and its TPT / TPF decompositions, on an annulus and on a full
cylinder (the axis as a face of zero area), every wall kind, FP64 TPT, FP64
TPF and the mixed-precision TPT."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import cylindrical as cy
from workloads import rhs_uniform, tanh_faces

pytestmark = pytest.mark.gpu

D, N = cy.DIRICHLET, cy.NEUMANN


@pytest.fixture(scope="module")
def fdi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2461_gb300 import build
    build.build()
    import paper_1107_2461_gb300 as pkg
    return pkg


def annulus(n, a=0.5, b=1.5, beta=1.5):
    return a + (b - a) * tanh_faces(n, beta)


def cylinder(n, beta=1.2):
    rf = tanh_faces(n, beta)
    rf[0] = 0.0
    return rf


def rel_residual(rf, M, zf, bc_r, bc_z, u, f, lam, sigma):
    L = cy.assembled(rf, M, zf, bc_r, bc_z)
    A = sigma * sp.identity(L.shape[0]) - lam * L
    r = np.ravel(f) - A @ np.ravel(u)
    return np.linalg.norm(r) / np.linalg.norm(np.ravel(f))


def gpu_solve(fdi, plan, f, lam, sigma):
    import torch
    rhs = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    out = torch.empty_like(rhs)
    fdi.field_solve(plan, fdi.FIELD_CELL, sigma, lam, rhs, out)
    torch.cuda.synchronize()
    _, steps, rel, status = fdi.last_result(plan)
    return out.cpu().numpy(), steps, rel, status


MODES = [("fp64", False), ("fp64", True), ("mixed", False)]


def prec_of(fdi, name):
    return fdi.PREC_FP64 if name == "fp64" else fdi.PREC_MIXED_F16


def tol_of(name):
    return 1e-11 if name == "fp64" else 1e-10


# (radial faces, bc_r (inner, outer), bc_z): annulus with every radial wall
# combination, and the full cylinder (inner condition ignored at the axis)
CASES = [
    ("annulus", (D, D), (D, D)),
    ("annulus", (N, D), (D, N)),
    ("annulus", (D, N), (N, N)),
    ("cylinder", (D, D), (D, D)),
    ("cylinder", (D, N), (D, D)),
    ("cylinder", (N, D), (N, N)),
]


@pytest.mark.parametrize("prec_name,tpf", MODES)
@pytest.mark.parametrize("geom,bc_r,bc_z", CASES)
def test_cylinder_matches_direct_solve(fdi, prec_name, tpf, geom, bc_r, bc_z):
    # ragged extents: 13 radial, 10 theta, 9 axial cells
    nr, M, nz = 13, 10, 9
    rf = annulus(nr) if geom == "annulus" else cylinder(nr)
    zf = 2.0 * tanh_faces(nz, 1.3)
    f = rhs_uniform((nz, M, nr), 5)
    for lam, sigma in ((1.0, 1.0), (1e-3, 1.0), (1.0, 0.0)):
        closed = (geom == "cylinder" or bc_r[0] == N) and bc_r[1] == N
        if sigma == 0.0 and closed and bc_z == (N, N):
            continue  # the singular zero-flux Laplacian, excluded by the oracle too
        ref = cy.direct_solve(f, rf, M, zf, lam, sigma, bc_r, bc_z)
        plan = fdi.plan_create_cyl(rf, M, zf, bc_r, bc_z, prec=prec_of(fdi, prec_name), tpf=tpf)
        try:
            got, steps, rel, st = gpu_solve(fdi, plan, f, lam, sigma)
        finally:
            plan.destroy()
        tol = tol_of(prec_name)
        assert st == 0 and rel <= tol, (lam, sigma, steps, rel, st)
        assert rel_residual(rf, M, zf, bc_r, bc_z, got, f, lam, sigma) <= tol
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max(), (lam, sigma)


@pytest.mark.parametrize("prec_name,tpf", MODES)
def test_cylinder_larger_grid_against_oracle_decomposition(fdi, prec_name, tpf):
    # several transform tiles and Thomas blocks, ragged: 70 radial, 48 theta,
    # 37 axial cells on a full cylinder with a zero-flux outer wall
    nr, M, nz = 70, 48, 37
    rf = cylinder(nr)
    zf = 3.0 * tanh_faces(nz, 1.5)
    bc_r, bc_z = (D, N), (D, D)
    f = rhs_uniform((nz, M, nr), 11)
    lam = 0.25
    plan = fdi.plan_create_cyl(rf, M, zf, bc_r, bc_z, prec=prec_of(fdi, prec_name), tpf=tpf)
    try:
        got, steps, rel, st = gpu_solve(fdi, plan, f, lam, 1.0)
    finally:
        plan.destroy()
    tol = tol_of(prec_name)
    assert st == 0 and rel <= tol, (steps, rel, st)
    assert rel_residual(rf, M, zf, bc_r, bc_z, got, f, lam, 1.0) <= tol
    ref = (cy.tpf_solve if tpf else cy.tpt_solve)(f, rf, M, zf, lam, 1.0, bc_r, bc_z)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def test_theta_eigenbasis_is_the_periodic_operators(fdi):
    # the closed-form theta basis of the plan diagonalises the oracle's periodic
    # operator and is orthonormal in its cell widths
    M = 15
    rf, zf = annulus(6), tanh_faces(5, 1.0)
    plan = fdi.plan_create_cyl(rf, M, zf)
    try:
        lam, E, Einv = plan.eigen(fdi.FIELD_CELL, 1)
        lr, Er, _ = plan.eigen(fdi.FIELD_CELL, 0)
    finally:
        plan.destroy()
    m, K = cy.periodic_operator(M)
    Dm = K / m[:, None]
    assert np.abs(Dm @ E - E * lam[None, :]).max() <= 1e-12 * np.abs(lam).max()
    assert np.abs(E.T @ (m[:, None] * E) - np.eye(M)).max() <= 1e-13
    assert np.abs(Einv @ E - np.eye(M)).max() <= 1e-13
    # the radial basis diagonalises D_rr = diag(A)^-1 K_r
    A, Kr, _ = cy.radial_operator(rf, D, D)
    assert np.abs((Kr / A[:, None]) @ Er - Er * lr[None, :]).max() <= 1e-11 * np.abs(lr).max()


def test_cylinder_rejections(fdi):
    rf, zf = cylinder(8), tanh_faces(6, 1.0)
    with pytest.raises(fdi.FdiError) as e:
        fdi.plan_create_cyl(rf, 8, zf, prec=fdi.PREC_MIXED_F16, tpf=True)
    assert e.value.status == fdi.ERR_UNSUPPORTED
    with pytest.raises(fdi.FdiError) as e:
        fdi.plan_create_cyl(rf, 2, zf)
    assert e.value.status == fdi.ERR_INVALID_ARG
    with pytest.raises(fdi.FdiError) as e:
        fdi.plan_create_cyl(rf - 0.5, 8, zf)
    assert e.value.status == fdi.ERR_INVALID_ARG
    # the singular zero-flux Laplacian
    import torch
    plan = fdi.plan_create_cyl(rf, 8, zf, (N, N), (N, N))
    try:
        x = torch.zeros((6, 8, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(fdi.FdiError) as e:
            fdi.laplace_solve(plan, x, torch.empty_like(x))
        assert e.value.status == fdi.ERR_UNSUPPORTED
    finally:
        plan.destroy()
