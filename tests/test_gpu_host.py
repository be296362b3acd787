"""Host-buffer solves (fdi_field_solve_host): the pipelined host <-> device copies
around a sequence of direct solves (Sec. 3) give the same bits as the device
solves of the same right-hand sides, for both precisions."""
import numpy as np
import pytest

from oracle import assembled as asm
from workloads import rhs_uniform, tanh_faces

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


def device_solve(fdi, plan, sigma, lam, f):
    import torch
    rhs = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    out = torch.empty_like(rhs)
    s = torch.cuda.Stream()
    fdi.field_solve(plan, fdi.FIELD_CELL, sigma, lam, rhs, out, s)
    s.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("which", ["fp64", "mixed"])
@pytest.mark.parametrize("count", [1, 2, 5])
def test_host_pipeline_matches_device_solves(fdi, which, count):
    import torch
    prec = fdi.PREC_FP64 if which == "fp64" else fdi.PREC_MIXED_F16
    tol = 1e-11 if which == "fp64" else 1e-10
    n = (48, 40, 36)
    faces = [tanh_faces(n[d], 1.5) for d in range(3)]
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    fs = [rhs_uniform(n[::-1], 50 + i) for i in range(count)]
    plan = fdi.plan_create(faces, n, prec=prec)
    try:
        # pinned tensors for even indices, plain numpy arrays for odd ones
        rhs = [torch.from_numpy(f).pin_memory() if i % 2 == 0 else f.copy() for i, f in enumerate(fs)]
        out = [torch.empty(n[::-1], dtype=torch.float64).pin_memory() if i % 2 == 0 else np.empty(n[::-1])
               for i in range(count)]
        s = torch.cuda.Stream()
        rel = fdi.field_solve_host(plan, fdi.FIELD_CELL, 1.0, 0.8, rhs, out, s)
        # twice more with the same arrays: the alternating staging buffers now
        # replay captured graphs
        for _ in range(2):
            rel2 = fdi.field_solve_host(plan, fdi.FIELD_CELL, 1.0, 0.8, rhs, out, s)
            assert rel2 == rel
        refs = [device_solve(fdi, plan, 1.0, 0.8, f) for f in fs]
    finally:
        plan.destroy()
    assert len(rel) == count and max(rel) <= tol
    for i in range(count):
        got = out[i].numpy() if hasattr(out[i], "numpy") else out[i]
        assert np.array_equal(got, refs[i]), i
        assert asm.relative_residual(ops, got, fs[i], 0.8) <= tol


def test_host_pipeline_in_place_and_laplace(fdi):
    # out[i] = rhs[i] (in place), the singular zero-flux Laplacian (sigma = 0)
    n = (32, 24, 20)
    faces = [tanh_faces(n[d], 1.2) for d in range(3)]
    b = (N, N, N)
    ops = asm.cell_ops(faces, b, b)
    fs = [rhs_uniform(n[::-1], 70 + i) for i in range(3)]
    plan = fdi.plan_create(faces, n, b, b, prec=fdi.PREC_MIXED_F16)
    try:
        bufs = [f.copy() for f in fs]
        rel = fdi.field_solve_host(plan, fdi.FIELD_CELL, 0.0, 1.0, bufs, bufs)
    finally:
        plan.destroy()
    assert max(rel) <= 1e-10
    vol = asm.volumes(ops)
    for f, u in zip(fs, bufs):
        assert asm.relative_residual(ops, u, f, 1.0, 0.0) <= 1e-10
        assert abs(np.dot(vol, u.ravel())) <= 1e-10 * np.abs(u).max() * vol.sum()


def test_host_pipeline_reports_the_bad_rhs(fdi):
    import torch
    n = (24, 20, 16)
    faces = [tanh_faces(n[d], 1.5) for d in range(3)]
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    fs = [rhs_uniform(n[::-1], 80 + i) for i in range(4)]
    fs[2][3, 4, 5] = np.nan
    out = [np.empty(n[::-1]) for _ in range(4)]
    plan = fdi.plan_create(faces, n, prec=fdi.PREC_MIXED_F16)
    try:
        with pytest.raises(fdi.FdiError) as e:
            fdi.field_solve_host(plan, fdi.FIELD_CELL, 1.0, 1.0, fs, out, torch.cuda.Stream())
        assert e.value.status == fdi.ERR_INVALID_ARG
        assert "right-hand side 2" in str(e.value)
        assert fdi.field_solve_host(plan, fdi.FIELD_CELL, 1.0, 1.0, [], []) == []
    finally:
        plan.destroy()
    for i in (0, 1, 3):
        assert asm.relative_residual(ops, out[i], fs[i], 1.0) <= 1e-10
