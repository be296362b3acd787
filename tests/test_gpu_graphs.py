"""CUDA-graph replay of repeated field solves: the captured launch sequence
gives the same results as the eager one, follows new data behind the same
arrays, and is dropped when the arguments change."""
import numpy as np
import pytest

from oracle import decomposition as dec
from oracle import operators1d as o1
from workloads import box_faces, rhs_uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2461_gb300 import build
    build.build()
    import paper_1107_2461_gb300 as pkg
    return pkg


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_matches_eager(fdi, prec):
    import torch
    n = (40, 36, 33)
    faces = box_faces(n, 1.5)
    p = fdi.PREC_FP64 if prec == "fp64" else fdi.PREC_MIXED_F16
    plan = fdi.plan_create(faces, n, prec=p)
    ref_plan = fdi.plan_create(faces, n, prec=p)
    fdi.set_graphs(ref_plan, False)
    stream = torch.cuda.Stream()
    rhs = torch.empty(n[::-1], dtype=torch.float64, device="cuda")
    out = torch.empty_like(rhs)
    ref = torch.empty_like(rhs)
    launches = []
    for call, (lam, seed) in enumerate([(0.5, 0), (0.5, 1), (0.5, 2), (0.5, 3), (2.0, 4), (2.0, 5), (2.0, 6)]):
        with torch.cuda.stream(stream):
            rhs.copy_(torch.from_numpy(rhs_uniform(n[::-1], seed)))
            fdi.helmholtz_solve(plan, lam, rhs, out, stream)
            fdi.helmholtz_solve(ref_plan, lam, rhs, ref, stream)
        stream.synchronize()
        launches.append(fdi.last_launch_count(plan))
        it, steps, res, status = fdi.last_result(plan)
        assert status == 0, (call, status)
        # identical launch sequence, identical arithmetic: bitwise equal
        assert torch.equal(out, ref), call
    # replayed calls report the captured launch count
    assert len(set(launches)) == 1 and launches[0] > 0
    # the last solve against the oracle
    ops = [o1.cell_operator(faces[d], o1.DIRICHLET, o1.DIRICHLET) for d in range(3)]
    want = dec.solve(rhs_uniform(n[::-1], 6), ops, 2.0, 1.0, "tpt")
    got = out.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
    plan.destroy()
    ref_plan.destroy()


def test_graph_dropped_on_new_arrays(fdi):
    import torch
    n = (24, 20, 18)
    faces = box_faces(n, 1.2)
    plan = fdi.plan_create(faces, n, prec=fdi.PREC_MIXED_F16)
    stream = torch.cuda.Stream()
    a = torch.from_numpy(rhs_uniform(n[::-1], 7)).cuda()
    b = torch.from_numpy(rhs_uniform(n[::-1], 8)).cuda()
    oa, ob = torch.empty_like(a), torch.empty_like(b)
    with torch.cuda.stream(stream):
        for _ in range(3):
            fdi.helmholtz_solve(plan, 1.0, a, oa, stream)
        fdi.helmholtz_solve(plan, 1.0, b, ob, stream)  # new arrays: eager, graph dropped
        fdi.helmholtz_solve(plan, 1.0, a, oa, stream)
    stream.synchronize()
    ops = [o1.cell_operator(faces[d], o1.DIRICHLET, o1.DIRICHLET) for d in range(3)]
    for x, o, seed in ((a, oa, 7), (b, ob, 8)):
        want = dec.solve(rhs_uniform(n[::-1], seed), ops, 1.0, 1.0, "tpt")
        assert np.abs(o.cpu().numpy() - want).max() <= 1e-9 * np.abs(want).max()
    plan.destroy()


def test_thomas_factor_cache_alternating_lambdas(fdi):
    # FP64 TPT sweeps reuse their line factors while (sigma, lambda, field)
    # repeats; alternating lambdas on one plan and stream, so that a graph
    # captured for lambda_1 is replayed after the cache holds lambda_2's
    # factors: every result must still be the oracle's (the device-side key
    # check makes the replay factorise again)
    import numpy as np
    import torch
    from oracle import assembled as asm
    from workloads import box_faces, rhs_uniform
    n = (40, 36, 33)
    faces = box_faces(n, 1.5)
    ops = asm.cell_ops(faces, (0, 0, 0), (0, 0, 0))
    f = rhs_uniform(n[::-1], 3)
    plan = fdi.plan_create(faces, n)
    stream = torch.cuda.Stream()
    rhs = torch.from_numpy(f).cuda()
    outs = {lam: torch.empty_like(rhs) for lam in (1.0, 1e-3)}
    try:
        for lam in (1.0, 1.0, 1e-3, 1.0, 1e-3, 1.0, 1.0):
            fdi.helmholtz_solve(plan, lam, rhs, outs[lam], stream)
            stream.synchronize()
            _, _, rel, st = fdi.last_result(plan)
            assert st == 0 and rel <= 1e-11, (lam, rel)
            assert asm.relative_residual(ops, outs[lam].cpu().numpy(), f, lam) <= 1e-11
    finally:
        plan.destroy()


def test_mixed_thomas_fp64_recurrence(fdi):
    # configuration 4: the mixed path's z sweep as an FP64 recurrence with
    # cached line factors (on the FP32 fields); refined to the same tolerance
    import torch
    from oracle import assembled as asm
    from workloads import box_faces, rhs_uniform
    for n, bc, lam, sigma in (((64, 48, 40), (0, 0, 0), 1.0, 1.0), ((32, 40, 24), (1, 0, 1), 1e-3, 1.0),
                              ((24, 20, 18), (1, 1, 1), 1.0, 0.0)):
        faces = box_faces(n, 1.5)
        ops = asm.cell_ops(faces, bc, bc)
        f = rhs_uniform(n[::-1], 4)
        plan = fdi.plan_create(faces, n, bc, bc, prec=fdi.PREC_MIXED_F16)
        try:
            fdi.set_thomas_config(plan, 4)
            rhs = torch.from_numpy(f).cuda()
            out = torch.empty_like(rhs)
            for _ in range(2):  # the second solve takes the cached factors
                fdi.field_solve(plan, fdi.FIELD_CELL, sigma, lam, rhs, out)
                torch.cuda.synchronize()
                _, steps, rel, st = fdi.last_result(plan)
                assert st == 0 and rel <= 1e-10, (n, steps, rel)
                assert asm.relative_residual(ops, out.cpu().numpy(), f, lam, sigma) <= 1e-10
        finally:
            plan.destroy()
