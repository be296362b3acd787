"""GPU parity of the mixed-precision path: split-fp16 tensor-core transforms
(tcgen05), FP32 Thomas sweep, double-float refinement (Sec. 3 TPT), against the
FP64 CPU oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import assembled as asm
from oracle import decomposition as dec
from oracle import operators1d as o1
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


def pitch4(n):
    return (n + 3) // 4 * 4


@pytest.mark.parametrize("n,rows", [(n, r) for n in (16, 64, 100, 129, 256) for r in (128, 1000)] +
                         [(256, 63488), (128, 65529), (100, 40000)])
@pytest.mark.parametrize("inverse", [1, 0])
def test_tensor_core_transform_matches_fp64(fdi, n, rows, inverse):
    # (the last three: more tiles than SMs with a partial last wave, which runs
    # as half-width items; a ragged last tile among them)
    # one split-fp16 pass out[r][k] = sum_j T[k][j] in[r][j] vs the FP64 product
    import torch
    faces = [tanh_faces(n, 1.5), tanh_faces(8, 1.0), tanh_faces(8, 1.0)]
    plan = fdi.plan_create(faces, (n, 8, 8), prec=fdi.PREC_MIXED_F16)
    lam, E, Einv = plan.eigen(fdi.FIELD_CELL, 0)
    T = Einv if inverse else E
    p = pitch4(n)
    x = np.zeros((rows, p), dtype=np.float32)
    x[:, :n] = np.random.default_rng(n + rows).uniform(-1, 1, (rows, n)).astype(np.float32)
    xin = torch.from_numpy(x).cuda()
    out = torch.zeros_like(xin)
    fdi.apply_transform(plan, fdi.FIELD_CELL, 0, inverse, xin, out, rows)
    torch.cuda.synchronize()
    got = out.cpu().numpy()[:, :n].astype(np.float64)
    ref = x[:, :n].astype(np.float64) @ T.T
    # error of the split product relative to sum_j |T_kj x_j| (~2^-21 per term
    # plus FP32 accumulation)
    scale = np.abs(x[:, :n]).astype(np.float64) @ np.abs(T).T
    err = np.abs(got - ref) / scale
    plan.destroy()
    assert err.max() < 2e-6, err.max()


def mixed_solve(fdi, faces, bc_lo, bc_hi, lam, sigma, f, alias=False, resident=False):
    # resident=True: the resident launch (one cooperative launch per solve)
    # instead of the pass-by-pass solve
    import torch
    n = tuple(len(fc) - 1 for fc in faces)
    plan = fdi.plan_create(faces, n, bc_lo, bc_hi, prec=fdi.PREC_MIXED_F16)
    fdi.set_resident(plan, resident)
    rhs = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    out = rhs if alias else torch.empty_like(rhs)
    fdi.field_solve(plan, fdi.FIELD_CELL, sigma, lam, rhs, out)
    torch.cuda.synchronize()
    it, steps, rel, st = fdi.last_result(plan)
    got = out.cpu().numpy()
    plan.destroy()
    return got, steps, rel, st


@pytest.mark.parametrize("resident", [True, False])
def test_small_mixed_solve(fdi, resident):
    n = (32, 32, 32)
    faces = box_faces(n, 1.5)
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 0)
    got, steps, rel, st = mixed_solve(fdi, faces, (D, D, D), (D, D, D), 1.0, 1.0, f, resident=resident)
    assert st == 0 and rel <= MIXED_TOL, (steps, rel)
    assert asm.relative_residual(ops, got, f, 1.0) <= MIXED_TOL
    ref = asm.solve(ops, f, 1.0)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


BCS = [((D, D, D), (D, D, D)), ((N, N, N), (N, N, N)), ((D, N, D), (N, D, N)), ((N, N, D), (N, N, N))]


@pytest.mark.parametrize("resident", [True, False])
@pytest.mark.parametrize("lo,hi", BCS)
@pytest.mark.parametrize("lam,sigma", [(1e-5, 1.0), (1e-3, 1.0), (1.0, 1.0), (1.0, 0.0)])
def test_ragged_grids_mixed(fdi, lo, hi, lam, sigma, resident):
    # sizes that are not multiples of the 128-row tile / 64-wide K chunk / 32-wide N pad
    # (resident: plane class 128, odd x extent, scalar residual pairs)
    n = (67, 13, 29)
    faces = [tanh_faces(67, 1.5), tanh_faces(13, 2.0), tanh_faces(29, 1.2)]
    ops = asm.cell_ops(faces, lo, hi)
    f = rhs_uniform(n[::-1], 3)
    got, steps, rel, st = mixed_solve(fdi, faces, lo, hi, lam, sigma, f, resident=resident)
    assert st == 0 and rel <= MIXED_TOL, (steps, rel)
    assert asm.relative_residual(ops, got, f, lam, sigma) <= MIXED_TOL
    ref = asm.solve(ops, f, lam, sigma)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    if asm.is_singular(ops, sigma):
        vol = asm.volumes(ops)
        assert abs(np.dot(vol, got.ravel())) <= 1e-10 * np.abs(got).max() * vol.sum()


def test_out_may_alias_rhs_mixed(fdi):
    n = (40, 24, 20)
    faces = box_faces(n, 1.5)
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 5)
    got, _, rel, st = mixed_solve(fdi, faces, (D, D, D), (D, D, D), 0.3, 1.0, f, alias=True)
    assert st == 0 and rel <= MIXED_TOL
    assert asm.relative_residual(ops, got, f, 0.3) <= MIXED_TOL


@pytest.mark.parametrize("resident", [True, False])
def test_config2_shape_mixed(fdi, resident):
    # 128^3, tanh 2.0: three Dirichlet Helmholtz (dt in {1e-2, 1, 1e3}, Re 1000) + one
    # zero-flux Laplace, refined to 1e-10 and checked against the oracle
    n = (128, 128, 128)
    faces = box_faces(n, 2.0)
    for seed, dt in enumerate([1e-2, 1.0, 1e3]):
        lam = dt / 1000.0
        ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
        f = rhs_uniform(n[::-1], seed)
        got, steps, rel, st = mixed_solve(fdi, faces, (D, D, D), (D, D, D), lam, 1.0, f, resident=resident)
        assert st == 0 and rel <= MIXED_TOL, (dt, steps, rel)
        assert asm.relative_residual(ops, got, f, lam) <= MIXED_TOL
        ref = dec.tpt_solve(f, ops, lam)
        assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    ops = asm.cell_ops(faces, (N, N, N), (N, N, N))
    f = rhs_uniform(n[::-1], 3)
    got, steps, rel, st = mixed_solve(fdi, faces, (N, N, N), (N, N, N), 1.0, 0.0, f, resident=resident)
    assert st == 0 and rel <= MIXED_TOL, (steps, rel)
    assert asm.relative_residual(ops, got, f, 1.0, 0.0) <= MIXED_TOL


def test_bench_workload_256_mixed(fdi):
    # the benchmarked solve: 256^3, tanh 1.5, Dirichlet, lambda = 1, TPT; residual
    # checked with the oracle's assembled operator, values against the oracle TPT
    n = (256, 256, 256)
    faces = box_faces(n, 1.5)
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 0)
    got, steps, rel, st = mixed_solve(fdi, faces, (D, D, D), (D, D, D), 1.0, 1.0, f)
    assert st == 0 and rel <= MIXED_TOL, (steps, rel)
    assert asm.relative_residual(ops, got, f, 1.0) <= MIXED_TOL
    ref = dec.tpt_solve(f, ops, 1.0)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


def test_mixed_refined_to_fp64_tolerance(fdi):
    # the mixed path with one more refinement step reaches the FP64 path's
    # tolerance (1e-11): 128^3, tanh 2.0, the three Helmholtz lambdas and the
    # zero-flux Laplacian, residuals recomputed with the oracle's operator
    import torch
    n = (128, 128, 128)
    faces = box_faces(n, 2.0)
    cases = [((D, D, D), lam, 1.0, s) for s, lam in enumerate([1e-5, 1e-3, 1.0])] + [((N, N, N), 1.0, 0.0, 3)]
    for bc, lam, sigma, seed in cases:
        ops = asm.cell_ops(faces, bc, bc)
        f = rhs_uniform(n[::-1], seed)
        plan = fdi.plan_create(faces, n, bc, bc, prec=fdi.PREC_MIXED_F16)
        try:
            plan.set_tolerances(1e-11, 3)
            rhs = torch.from_numpy(f).cuda()
            out = torch.empty_like(rhs)
            fdi.field_solve(plan, fdi.FIELD_CELL, sigma, lam, rhs, out)
            torch.cuda.synchronize()
            it, steps, rel, st = fdi.last_result(plan)
        finally:
            plan.destroy()
        got = out.cpu().numpy()
        assert st == 0 and rel <= 1e-11, (lam, sigma, steps, rel)
        assert asm.relative_residual(ops, got, f, lam, sigma) <= 1e-11


def _mixed_tpf(fdi, faces, bc, lam, sigma, f, tol=None):
    import torch
    n = tuple(len(fc) - 1 for fc in faces)
    plan = fdi.plan_create(faces, n, bc, bc, prec=fdi.PREC_MIXED_F16, thomas_axis=-1)
    try:
        # a pipeline that stops making progress reports a wait limit quickly
        fdi.set_wait_limit(plan, 100_000_000)
        if tol is not None:
            plan.set_tolerances(tol, 3)
        rhs = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        out = torch.empty_like(rhs)
        fdi.field_solve(plan, fdi.FIELD_CELL, sigma, lam, rhs, out)
        torch.cuda.synchronize()
        _, steps, rel, st = fdi.last_result(plan)
    finally:
        plan.destroy()
    return out.cpu().numpy(), steps, rel, st


@pytest.mark.parametrize("n,bc,lam,sigma", [
    ((16, 12, 9), (D, D, D), 1.0, 1.0),       # one z chunk, ragged plane (192 rows)
    ((40, 36, 33), (N, D, N), 1e-3, 1.0),     # two z chunks, ragged chunk
    ((24, 20, 70), (D, N, D), 1.0, 0.0),      # three z chunks, Laplacian
    ((32, 28, 17), (N, N, N), 1.0, 0.0),      # the singular zero-flux Laplacian
])
def test_mixed_tpf_small(fdi, n, bc, lam, sigma):
    # mixed-precision TPF (Eq. 29): the z transforms on the tensor cores and the
    # spectral divide, refined to 1e-10, against the oracle's TPF and its
    # assembled operator
    faces = box_faces(n, 1.5)
    ops = asm.cell_ops(faces, bc, bc)
    f = rhs_uniform(n[::-1], 31)
    got, steps, rel, st = _mixed_tpf(fdi, faces, bc, lam, sigma, f)
    assert st == 0 and rel <= MIXED_TOL, (steps, rel, st)
    assert asm.relative_residual(ops, got, f, lam, sigma) <= MIXED_TOL
    ref = dec.tpf_solve(f, ops, lam, sigma)
    if sigma == 0.0 and bc == (N, N, N):
        V = asm.volumes(ops)
        got = got - np.sum(V * got.ravel()) / V.sum()
        ref = ref - np.sum(V * ref.ravel()) / V.sum()
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("n", [(128, 64, 40), (128, 128, 128), (256, 256, 256)])
def test_mixed_tpf_at_scale(fdi, n):
    # larger grids, after the small ones: many plane tiles, two to eight z
    # chunks; the 256^3 benchmark grid included
    faces = box_faces(n, 1.5)
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 7)
    got, steps, rel, st = _mixed_tpf(fdi, faces, (D, D, D), 1.0, 1.0, f)
    assert st == 0 and rel <= MIXED_TOL, (steps, rel, st)
    assert asm.relative_residual(ops, got, f, 1.0) <= MIXED_TOL
    ref = dec.tpf_solve(f, ops, 1.0)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
