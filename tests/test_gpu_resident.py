"""Resident small-grid solve (fdi_plan_set_resident): every pass of the
mixed-precision TPT solve and its refinement rounds in one cooperative launch
(fields with x, y extents <= 128), against the FP64 oracle and against the
pass-by-pass solve, through the C ABI."""
import numpy as np
import pytest

from oracle import assembled as asm
from oracle import decomposition as dec
from workloads import box_faces, rhs_uniform, tanh_faces

pytestmark = pytest.mark.gpu

D, N = 0, 1
MIXED_TOL = 1e-10


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


# (n, walls lo, walls hi, lambda, sigma): plane classes 64 and 128, odd and
# tiny extents, one plane, long z lines, the zero-flux Laplace problem
CASES = [
    ((16, 12, 9), (D, D, D), (D, D, D), 1.0, 1.0),
    ((61, 64, 33), (D, N, D), (N, D, N), 0.3, 1.0),
    ((64, 64, 64), (D, D, D), (D, D, D), 1e-3, 1.0),
    ((100, 128, 40), (D, D, N), (D, D, D), 1e-5, 1.0),
    ((2, 3, 2), (D, D, D), (D, D, D), 1.0, 1.0),
    ((33, 7, 2), (D, D, D), (D, D, D), 1.0, 1.0),
    ((8, 8, 250), (D, D, D), (D, D, D), 1.0, 1.0),
    ((48, 40, 36), (N, N, N), (N, N, N), 1.0, 0.0),
    ((128, 20, 17), (N, D, N), (N, N, N), 1.0, 0.0),
]


@pytest.mark.parametrize("n,lo,hi,lam,sigma", CASES)
def test_resident_one_launch_against_oracle(fdi, n, lo, hi, lam, sigma):
    faces = [tanh_faces(n[0], 1.5), tanh_faces(n[1], 2.0), tanh_faces(n[2], 1.2)]
    ops = asm.cell_ops(faces, lo, hi)
    f = rhs_uniform(n[::-1], sum(n))
    plan = fdi.plan_create(faces, n, lo, hi, prec=fdi.PREC_MIXED_F16)
    fdi.set_resident(plan, True)
    try:
        got, steps, rel, st = solve(fdi, plan, lam, sigma, f)
        assert st == 0 and rel <= MIXED_TOL, (steps, rel)
        assert fdi.last_launch_count(plan) == 1
    finally:
        plan.destroy()
    assert asm.relative_residual(ops, got, f, lam, sigma) <= MIXED_TOL
    ref = dec.tpt_solve(f, ops, lam, sigma)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    if asm.is_singular(ops, sigma):
        vol = asm.volumes(ops)
        assert abs(np.dot(vol, got.ravel())) <= 1e-10 * np.abs(got).max() * vol.sum()


def test_resident_and_pass_by_pass_agree(fdi):
    # the two routes take different arithmetic (FP32 plane products against
    # split-fp16 tensor-core passes) to the same tolerance
    n = (96, 80, 48)
    faces = box_faces(n, 1.5)
    f = rhs_uniform(n[::-1], 11)
    plan = fdi.plan_create(faces, n, prec=fdi.PREC_MIXED_F16)
    fdi.set_resident(plan, True)
    try:
        a, _, rel_a, st_a = solve(fdi, plan, 0.05, 1.0, f)
        assert fdi.last_launch_count(plan) == 1
        fdi.set_resident(plan, False)
        b, _, rel_b, st_b = solve(fdi, plan, 0.05, 1.0, f)
        assert fdi.last_launch_count(plan) > 5
    finally:
        plan.destroy()
    assert st_a == 0 and st_b == 0 and rel_a <= MIXED_TOL and rel_b <= MIXED_TOL
    assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()


def test_resident_repeat_is_bitwise(fdi):
    # the same solve twice (eager, then through the plan's graph cache on a
    # side stream): bitwise equal
    import torch
    n = (40, 56, 30)
    faces = box_faces(n, 1.5)
    f = rhs_uniform(n[::-1], 4)
    plan = fdi.plan_create(faces, n, prec=fdi.PREC_MIXED_F16)
    fdi.set_resident(plan, True)
    try:
        first, _, _, st = solve(fdi, plan, 0.2, 1.0, f)
        assert st == 0
        rhs = torch.from_numpy(f).cuda()
        out = torch.empty_like(rhs)
        s = torch.cuda.Stream()
        for _ in range(3):
            out.zero_()
            with torch.cuda.stream(s):
                fdi.field_solve(plan, fdi.FIELD_CELL, 1.0, 0.2, rhs, out, s)
            s.synchronize()
            assert fdi.last_result(plan)[3] == 0
            assert np.array_equal(out.cpu().numpy(), first)
    finally:
        plan.destroy()


def test_resident_wait_limit_runs_out_then_plan_recovers(fdi):
    # A one-cycle limit makes the grid barrier's first wait run out: the CTA
    # raises the abort flag, every CTA returns at its next barrier, the last
    # one out re-arms the barrier, and the solve reports FDI_ERR_TIMEOUT (no
    # fault).  With the default limit the same plan solves to its tolerance.
    n = (64, 64, 24)
    faces = [tanh_faces(n[d], 1.5) for d in range(3)]
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 5)
    plan = fdi.plan_create(faces, n, prec=fdi.PREC_MIXED_F16)
    fdi.set_resident(plan, True)
    try:
        fdi.set_wait_limit(plan, 1)
        for _ in range(2):
            with pytest.raises(fdi.FdiError) as e:
                solve(fdi, plan, 1.0, 1.0, f)
            assert e.value.status == fdi.ERR_TIMEOUT
        fdi.set_wait_limit(plan, 0)
        got, steps, rel, status = solve(fdi, plan, 1.0, 1.0, f)
        assert status == 0 and rel <= MIXED_TOL, (steps, rel)
        assert asm.relative_residual(ops, got, f, 1.0) <= MIXED_TOL
    finally:
        plan.destroy()
