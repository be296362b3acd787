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
