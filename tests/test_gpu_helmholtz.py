"""GPU parity of the Helmholtz / Laplace inverses against the FP64 CPU oracle,
called through the C ABI (Sec. 3, Eq. 25-29; TPT at the end of Sec. 3)."""
import numpy as np
import pytest

from oracle import assembled as asm
from oracle import decomposition as dec
from oracle import operators1d as o1
from workloads import box_faces, rhs_uniform, tanh_faces

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


def gpu_solve(fdi, faces, bc_lo, bc_hi, lam, sigma, f, prec, thomas_axis=2, alias=False, tol=None):
    import torch
    n = tuple(len(fc) - 1 for fc in faces)
    plan = fdi.plan_create(faces, n, bc_lo, bc_hi, prec=prec, thomas_axis=thomas_axis)
    if tol is not None:
        plan.set_tolerances(tol, 3)
    rhs = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    out = rhs if alias else torch.empty_like(rhs)
    fdi.field_solve(plan, fdi.FIELD_CELL, sigma, lam, rhs, out)
    torch.cuda.synchronize()
    it, steps, rel, st = fdi.last_result(plan)
    got = out.cpu().numpy()
    plan.destroy()
    return got, steps, rel, st


def rel_err(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("kind", ["cellDD", "cellNN", "cellDN", "face"])
@pytest.mark.parametrize("n", [5, 33, 64, 256])
def test_eigen_decomposition_matches_oracle(fdi, kind, n):
    # Eq. 24 on the GPU: Lambda and D = E Lambda E^{-1} agree with the oracle
    import torch  # noqa: F401
    faces = [tanh_faces(n, 2.0), tanh_faces(8, 1.0), tanh_faces(8, 1.0)]
    if kind == "face":
        plan = fdi.plan_create(faces, (n, 8, 8), grid=fdi.GRID_MAC)
        lam, E, Einv = plan.eigen(fdi.FIELD_U, 0)
        m, K = o1.face_operator(faces[0])
    else:
        bc = {"cellDD": (D, D), "cellNN": (N, N), "cellDN": (D, N)}[kind]
        plan = fdi.plan_create(faces, (n, 8, 8), (bc[0], D, D), (bc[1], D, D))
        lam, E, Einv = plan.eigen(fdi.FIELD_CELL, 0)
        m, K = o1.cell_operator(faces[0], *bc)
    plan.destroy()
    lam_o, _, _ = dec.generalized_eig(m, K)
    scale = np.abs(lam_o).max()
    assert np.abs(np.sort(lam) - np.sort(lam_o)).max() <= 1e-13 * scale * max(1, n / 16)
    Dm = o1.second_derivative(m, K)
    assert np.abs(E @ np.diag(lam) @ Einv - Dm).max() <= 1e-12 * scale
    assert np.abs(Einv @ E - np.eye(len(m))).max() <= 1e-12
    assert np.abs(E.T @ (m[:, None] * E) - np.eye(len(m))).max() <= 1e-12
    if kind == "cellNN":
        assert lam[0] == 0.0 and np.ptp(E[:, 0]) < 1e-14


def test_config1_tpf_fp64(fdi):
    # 16^3, tanh factor 1.5, Dirichlet, lambda = 1e3/1000, eigen decomposition in all
    # three directions, checked against the assembled operator solved directly
    n = (16, 16, 16)
    faces = box_faces(n, 1.5)
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 0)
    lam = 1e3 / 1000.0
    ref = asm.solve(ops, f, lam)
    got, steps, rel, st = gpu_solve(fdi, faces, (D, D, D), (D, D, D), lam, 1.0, f, fdi.PREC_FP64, thomas_axis=-1)
    assert st == 0 and rel <= 1e-11
    assert rel_err(got, ref) <= 1e-11
    assert asm.relative_residual(ops, got, f, lam) <= 1e-11


BCS = [((D, D, D), (D, D, D)), ((N, N, N), (N, N, N)), ((D, N, D), (N, D, N)), ((N, N, D), (N, N, N))]


@pytest.mark.parametrize("lo,hi", BCS)
@pytest.mark.parametrize("lam,sigma", [(1e-5, 1.0), (1e-3, 1.0), (1.0, 1.0), (1.0, 0.0)])
@pytest.mark.parametrize("axis", [2, -1])
def test_ragged_grids_fp64(fdi, lo, hi, lam, sigma, axis):
    # sizes that are not multiples of the 64-wide tiles, with a ragged tail
    n = (67, 13, 29)
    faces = [tanh_faces(67, 1.5), tanh_faces(13, 2.0), tanh_faces(29, 1.2)]
    ops = asm.cell_ops(faces, lo, hi)
    f = rhs_uniform(n[::-1], 3)
    ref = asm.solve(ops, f, lam, sigma)
    got, steps, rel, st = gpu_solve(fdi, faces, lo, hi, lam, sigma, f, fdi.PREC_FP64, thomas_axis=axis)
    assert st == 0 and rel <= 1e-11, (steps, rel)
    assert rel_err(got, ref) <= 1e-10
    assert asm.relative_residual(ops, got, f, lam, sigma) <= 1e-11
    if asm.is_singular(ops, sigma):
        vol = asm.volumes(ops)
        assert abs(np.dot(vol, got.ravel())) <= 1e-12 * np.abs(got).max() * vol.sum()


def test_out_may_alias_rhs(fdi):
    n = (20, 17, 11)
    faces = box_faces(n, 1.5)
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 5)
    ref = asm.solve(ops, f, 0.3)
    got, _, rel, st = gpu_solve(fdi, faces, (D, D, D), (D, D, D), 0.3, 1.0, f, fdi.PREC_FP64, alias=True)
    assert st == 0 and rel <= 1e-11 and rel_err(got, ref) <= 1e-11


def test_largest_direction_256(fdi):
    n = (256, 9, 256)
    faces = [tanh_faces(256, 1.5), tanh_faces(9, 1.5), tanh_faces(256, 2.0)]
    ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform(n[::-1], 9)
    ref = dec.tpt_solve(f, ops, 1.0)
    got, _, rel, st = gpu_solve(fdi, faces, (D, D, D), (D, D, D), 1.0, 1.0, f, fdi.PREC_FP64)
    assert st == 0 and rel <= 1e-11
    assert rel_err(got, ref) <= 1e-10


def test_config2_shape_fp64(fdi):
    # 128^3, tanh factor 2.0: three Dirichlet Helmholtz solves (dt in {1e-2, 1, 1e3},
    # Re = 1000) and one zero-flux Laplace solve; full comparison with the oracle
    n = (128, 128, 128)
    faces = box_faces(n, 2.0)
    for seed, dt in enumerate([1e-2, 1.0, 1e3]):
        lam = dt / 1000.0
        ops = asm.cell_ops(faces, (D, D, D), (D, D, D))
        f = rhs_uniform(n[::-1], seed)
        got, _, rel, st = gpu_solve(fdi, faces, (D, D, D), (D, D, D), lam, 1.0, f, fdi.PREC_FP64)
        assert st == 0 and rel <= 1e-11
        ref = dec.tpt_solve(f, ops, lam)
        assert rel_err(got, ref) <= 1e-10
    ops = asm.cell_ops(faces, (N, N, N), (N, N, N))
    f = rhs_uniform(n[::-1], 3)
    got, _, rel, st = gpu_solve(fdi, faces, (N, N, N), (N, N, N), 1.0, 0.0, f, fdi.PREC_FP64)
    assert st == 0 and rel <= 1e-11
    ref = dec.tpt_solve(f, ops, 1.0, 0.0)
    assert rel_err(got, ref) <= 1e-9
    assert asm.relative_residual(ops, got, f, 1.0, 0.0) <= 1e-11


@pytest.mark.parametrize("bc,sigma", [((D, D, D), 1.0), ((N, D, N), 1.0), ((D, N, D), 0.0)])
def test_tpf_128cube_against_oracle(fdi, bc, sigma):
    # FP64 TPF (eigen transforms in x, y and z, Eq. 29) at 128^3: the z
    # transform runs over many slab tiles; compared element by element with
    # the oracle's TPF and checked against its assembled operator
    n = (128, 128, 128)
    faces = box_faces(n, 2.0)
    ops = asm.cell_ops(faces, bc, bc)
    f = rhs_uniform(n[::-1], 21)
    lam = 1.0
    got, steps, rel, st = gpu_solve(fdi, faces, bc, bc, lam, sigma, f, fdi.PREC_FP64, thomas_axis=-1)
    assert st == 0 and rel <= 1e-11, (steps, rel)
    assert asm.relative_residual(ops, got, f, lam, sigma) <= 1e-11
    ref = dec.tpf_solve(f, ops, lam, sigma)
    assert rel_err(got, ref) <= 1e-10
