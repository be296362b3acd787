"""Thomas sweeps along x or y (Sec. 3: the sweep runs along one direction, the
paper choosing the one with the most points): plans on anisotropic grids whose
longest direction is not z, against the oracle's assembled operator."""
import numpy as np
import pytest

from oracle import assembled as asm
from oracle import decomposition as dec
from oracle import operators1d as o1
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


def solve(fdi, faces, n, lo, hi, axis, prec, lam, sigma, f, alias=False):
    import torch
    plan = fdi.plan_create(faces, n, lo, hi, prec=prec, thomas_axis=axis)
    try:
        rhs = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        out = rhs if alias else torch.empty_like(rhs)
        s = torch.cuda.Stream()
        for _ in range(3):  # eager, captured, replayed
            if alias:
                rhs.copy_(torch.from_numpy(np.ascontiguousarray(f)))
            fdi.field_solve(plan, fdi.FIELD_CELL, sigma, lam, rhs, out, s)
            s.synchronize()
            it, steps, rel, st = fdi.last_result(plan)
            assert st == 0, (steps, rel)
        return out.cpu().numpy(), rel
    finally:
        plan.destroy()


CASES = [
    ((40, 12, 16), 0, (D, D, D), (D, D, D), 0.7, 1.0),
    ((40, 12, 16), 0, (N, N, N), (N, N, N), 1.0, 0.0),
    ((13, 37, 10), 1, (D, N, D), (N, D, D), 0.3, 1.0),
    ((13, 37, 10), 1, (N, N, N), (N, N, N), 1.0, 0.0),
    ((33, 21, 9), -2, (D, D, N), (D, D, D), 1e-3, 1.0),
]


@pytest.mark.parametrize("n,axis,lo,hi,lam,sigma", CASES)
@pytest.mark.parametrize("which", ["fp64", "mixed"])
def test_thomas_axis_x_y(fdi, n, axis, lo, hi, lam, sigma, which):
    prec = fdi.PREC_FP64 if which == "fp64" else fdi.PREC_MIXED_F16
    tol = 1e-11 if which == "fp64" else 1e-10
    faces = [tanh_faces(n[0], 1.5), tanh_faces(n[1], 2.0), tanh_faces(n[2], 1.2)]
    ops = asm.cell_ops(faces, lo, hi)
    f = rhs_uniform(n[::-1], 7)
    got, rel = solve(fdi, faces, n, lo, hi, axis, prec, lam, sigma, f)
    assert rel <= tol
    assert asm.relative_residual(ops, got, f, lam, sigma) <= tol
    ref = asm.solve(ops, f, lam, sigma)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    if asm.is_singular(ops, sigma):
        vol = asm.volumes(ops)
        assert abs(np.dot(vol, got.ravel())) <= 1e-10 * np.abs(got).max() * vol.sum()


def test_thomas_axis_matches_z_solve_and_aliasing(fdi):
    # the same problem solved with the sweeps along x and along z agrees to the
    # solver accuracy; out may alias rhs on a permuted plan
    n = (24, 16, 20)
    faces = [tanh_faces(n[d], 1.5) for d in range(3)]
    f = rhs_uniform(n[::-1], 3)
    bc = (D, D, D)
    ux, _ = solve(fdi, faces, n, bc, bc, 0, fdi.PREC_FP64, 0.5, 1.0, f, alias=True)
    uz, _ = solve(fdi, faces, n, bc, bc, 2, fdi.PREC_FP64, 0.5, 1.0, f)
    assert np.abs(ux - uz).max() <= 1e-12 * np.abs(uz).max()


def test_eigen_directions_follow_the_caller(fdi):
    # fdi_plan_eigen takes the caller's direction on a permuted plan
    n = (30, 12, 8)
    faces = [tanh_faces(n[0], 1.5), tanh_faces(n[1], 2.0), tanh_faces(n[2], 1.2)]
    plan = fdi.plan_create(faces, n, (D, N, D), (D, D, N), thomas_axis=-2)
    try:
        for d, (lo, hi) in enumerate([(D, D), (N, D), (D, N)]):
            lam, E, Einv = plan.eigen(fdi.FIELD_CELL, d)
            m, K = o1.cell_operator(faces[d], lo, hi)
            lam_o, _, _ = dec.generalized_eig(m, K)
            assert len(lam) == n[d]
            assert np.abs(np.sort(lam) - np.sort(lam_o)).max() <= 1e-12 * np.abs(lam_o).max()
    finally:
        plan.destroy()


def test_staggered_plan_keeps_z(fdi):
    faces = [tanh_faces(8, 1.5), tanh_faces(6, 1.5), tanh_faces(5, 1.5)]
    with pytest.raises(fdi.FdiError):
        fdi.plan_create(faces, (8, 6, 5), grid=fdi.GRID_MAC, thomas_axis=0)
