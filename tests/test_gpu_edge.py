"""Edge cases of the C ABI on the GPU: the smallest grids the plan accepts, the
longest single direction, a zero right-hand side and non-finite input, for the
FP64 and the mixed-precision paths (Sec. 3, Eq. 25-29; the Stokes inverse of
Sec. 2)."""
import numpy as np
import pytest

from oracle import assembled as asm
from oracle import stokes as st
from workloads import rhs_gaussian, rhs_uniform, tanh_faces

pytestmark = pytest.mark.gpu

D, N = 0, 1


@pytest.fixture(scope="module")
def fdi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2461_gb300 import build
    build.build()
    import paper_1107_2461_gb300 as pkg
    return pkg


def solve(fdi, plan, lam, sigma, f):
    import torch
    rhs = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    out = torch.empty_like(rhs)
    fdi.field_solve(plan, fdi.FIELD_CELL, sigma, lam, rhs, out)
    torch.cuda.synchronize()
    it, steps, rel, status = fdi.last_result(plan)
    return out.cpu().numpy(), steps, rel, status


def precs(fdi):
    return [(fdi.PREC_FP64, 1e-11, 1e-10), (fdi.PREC_MIXED_F16, 1e-10, 1e-8)]


@pytest.mark.parametrize("n", [(2, 2, 2), (2, 3, 2), (256, 2, 2), (2, 256, 3), (3, 2, 256)])
@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
def test_extreme_shapes(fdi, n, which, bc):
    # the smallest cell grid (2 cells a direction) and one direction at the
    # largest size with the others at the smallest
    prec, tol, vtol = precs(fdi)[which]
    faces = [tanh_faces(n[d], 1.5) for d in range(3)]
    b = (D, D, D) if bc == "dirichlet" else (N, N, N)
    lam, sigma = (0.7, 1.0) if bc == "dirichlet" else (1.0, 0.0)
    ops = asm.cell_ops(faces, b, b)
    f = rhs_uniform(n[::-1], 17)
    plan = fdi.plan_create(faces, n, b, b, prec=prec)
    try:
        got, steps, rel, status = solve(fdi, plan, lam, sigma, f)
    finally:
        plan.destroy()
    assert status == 0 and rel <= tol, (steps, rel)
    assert asm.relative_residual(ops, got, f, lam, sigma) <= tol
    ref = asm.solve(ops, f, lam, sigma)
    assert np.abs(got - ref).max() <= vtol * np.abs(ref).max()
    if asm.is_singular(ops, sigma):
        vol = asm.volumes(ops)
        assert abs(np.dot(vol, got.ravel())) <= 1e-10 * np.abs(got).max() * vol.sum()


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("singular", [False, True])
def test_zero_rhs_gives_zero(fdi, which, singular):
    # A x = 0 has x = 0 (for the singular problem: the zero-mean solution); the
    # first check already meets the tolerance, so no refinement step runs
    prec, _, _ = precs(fdi)[which]
    n = (40, 33, 20)
    faces = [tanh_faces(n[d], 1.5) for d in range(3)]
    b = (N, N, N) if singular else (D, D, D)
    plan = fdi.plan_create(faces, n, b, b, prec=prec)
    try:
        got, steps, rel, status = solve(fdi, plan, 1.0, 0.0 if singular else 1.0, np.zeros(n[::-1]))
    finally:
        plan.destroy()
    assert status == 0 and steps == 0 and rel == 0.0
    assert not np.any(got)


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_rhs_is_invalid_argument(fdi, which, bad):
    # a non-finite right-hand side is reported as an argument error after the
    # solve, and the plan stays usable for the next solve
    prec, tol, _ = precs(fdi)[which]
    n = (24, 20, 16)
    faces = [tanh_faces(n[d], 1.5) for d in range(3)]
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 4)
    g = f.copy()
    g[5, 7, 11] = bad
    plan = fdi.plan_create(faces, n, prec=prec)
    try:
        with pytest.raises(fdi.FdiError) as e:
            solve(fdi, plan, 1.0, 1.0, g)
        assert e.value.status == fdi.ERR_INVALID_ARG
        assert "non-finite" in str(e.value)
        got, steps, rel, status = solve(fdi, plan, 1.0, 1.0, f)
    finally:
        plan.destroy()
    assert status == 0 and rel <= tol
    assert asm.relative_residual(ops, got, f, 1.0) <= tol


def stokes(fdi, faces, f, prec, dt=0.1):
    import torch
    n = tuple(len(fc) - 1 for fc in faces)
    plan = fdi.plan_create(faces, n, grid=fdi.GRID_MAC, prec=prec)
    try:
        ft = [torch.from_numpy(np.ascontiguousarray(fc)).cuda() for fc in f]
        ut = [torch.empty_like(t) for t in ft]
        _, ps = st.shapes(faces)
        pt = torch.empty(ps, dtype=torch.float64, device="cuda")
        fdi.stokes_solve(plan, dt, 1000.0, ft, ut, pt)
        torch.cuda.synchronize()
        it, _, rel, status = fdi.last_result(plan)
    finally:
        plan.destroy()
    return [t.cpu().numpy() for t in ut], pt.cpu().numpy(), it, rel, status


@pytest.mark.parametrize("which", [0, 1])
def test_smallest_mac_stokes(fdi, which):
    # 3 cells a direction: two interior faces per velocity direction
    prec, tol, _ = precs(fdi)[which]
    faces = [tanh_faces(3, 1.5), tanh_faces(3, 1.2), tanh_faces(3, 2.0)]
    vs, _ = st.shapes(faces)
    f = [rhs_gaussian(vs[c], 30 + c) for c in range(3)]
    vel_d, p_d = st.stokes_direct(faces, 0.1, 1000.0, f)
    vel, p, it, rel, status = stokes(fdi, faces, f, prec)
    assert status == 0 and rel <= tol, (it, rel)
    for c in range(3):
        assert np.abs(vel[c] - vel_d[c]).max() <= 1e-8 * np.abs(vel_d[c]).max()
    assert np.abs(p - p_d).max() <= 1e-7 * np.abs(p_d).max()


@pytest.mark.parametrize("which", [0, 1])
def test_stokes_non_finite_forcing_is_invalid_argument(fdi, which):
    prec, _, _ = precs(fdi)[which]
    faces = [tanh_faces(8, 1.5), tanh_faces(7, 1.5), tanh_faces(6, 1.5)]
    vs, _ = st.shapes(faces)
    f = [rhs_gaussian(vs[c], 40 + c) for c in range(3)]
    f[1][2, 3, 1] = np.nan
    with pytest.raises(fdi.FdiError) as e:
        stokes(fdi, faces, f, prec)
    assert e.value.status == fdi.ERR_INVALID_ARG


def test_wait_limit_runs_out_then_plan_recovers(fdi):
    # The tensor-core transform's roles hand shared-memory stages to one
    # another through bounded waits.  A limit of one cycle makes the first
    # wait for a TMA load run out: the kernel drains its issued copies and MMAs,
    # frees its tensor memory, returns, and the solve reports FDI_ERR_TIMEOUT
    # (no fault; the context stays usable).  With the default limit restored,
    # the same plan solves to its tolerance.
    n = (64, 64, 24)
    faces = [tanh_faces(n[d], 1.5) for d in range(3)]
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 5)
    plan = fdi.plan_create(faces, n, prec=fdi.PREC_MIXED_F16)
    try:
        fdi.set_wait_limit(plan, 1)
        for _ in range(2):  # the flag stays set until the limit is set again
            with pytest.raises(fdi.FdiError) as e:
                solve(fdi, plan, 1.0, 1.0, f)
            assert e.value.status == fdi.ERR_TIMEOUT
        fdi.set_wait_limit(plan, 0)
        got, steps, rel, status = solve(fdi, plan, 1.0, 1.0, f)
        assert status == 0 and rel <= 1e-10, (steps, rel)
        assert asm.relative_residual(ops, got, f, 1.0) <= 1e-10
    finally:
        plan.destroy()
    plan = fdi.plan_create(faces, n)
    try:
        with pytest.raises(fdi.FdiError) as e:
            fdi.set_wait_limit(plan, -1)
        assert e.value.status == fdi.ERR_INVALID_ARG
    finally:
        plan.destroy()
