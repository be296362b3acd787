"""Batched Helmholtz solves over uneven stretched grids (64 Arnoldi-style
right-hand sides with their own lambda, grids from {32..160} with aspect up to
1:4): concurrent plans on a stream pool, one captured CUDA graph per repeated
batch, autotuned configurations.  Every result must equal the same solve run
alone (bitwise: the same launch sequence on the same plan) and meet the
tolerance against the FP64 oracle."""
import numpy as np
import pytest

from oracle import decomposition as dec
from oracle import operators1d as o1
from workloads import mixed_shape_batch, rhs_uniform, tanh_faces

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


def make_batch(fdi, count, prec, seed=0, resident=False):
    import torch
    probs = mixed_shape_batch(count, seed)
    plans, lams, rhs, outs, host = [], [], [], [], []
    for q, (n, beta, lam) in enumerate(probs):
        faces = [tanh_faces(n[d], beta) for d in range(3)]
        plans.append(fdi.plan_create(faces, n, prec=prec))
        fdi.set_resident(plans[-1], resident)
        f = rhs_uniform(n[::-1], q + 1)
        host.append((faces, f))
        rhs.append(torch.from_numpy(f).cuda())
        outs.append(torch.empty_like(rhs[-1]))
        lams.append(lam)
    return probs, plans, lams, rhs, outs, host


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_resident"])
def test_batch_equals_alone_and_oracle(fdi, prec):
    # mixed_resident: the grids with x, y extents <= 128 share resident
    # launches in the batch and each has its own alone
    import torch
    p = fdi.PREC_FP64 if prec == "fp64" else fdi.PREC_MIXED_F16
    count = 16 if prec == "fp64" else 64
    probs, plans, lams, rhs, outs, host = make_batch(fdi, count, p, resident=prec == "mixed_resident")
    stream = torch.cuda.Stream()
    # alone: each plan solved by itself on the legacy stream (eager)
    alone = []
    for q in range(count):
        o = torch.empty_like(rhs[q])
        fdi.helmholtz_solve(plans[q], lams[q], rhs[q], o)
        torch.cuda.synchronize()
        assert fdi.last_result(plans[q])[3] == 0
        alone.append(o.cpu().numpy())
    # in the batch: eager, then captured, then replayed
    for rep in range(3):
        for o in outs:
            o.zero_()
        with torch.cuda.stream(stream):
            fdi.helmholtz_solve_batched(plans, lams, rhs, outs, stream)
        stream.synchronize()
        for q in range(count):
            it, steps, res, status = fdi.last_result(plans[q])
            assert status == 0, (rep, q, status, res)
            assert np.array_equal(outs[q].cpu().numpy(), alone[q]), (rep, q)
    # a few against the oracle (smallest problems)
    order = sorted(range(count), key=lambda q: np.prod(probs[q][0]))[:3]
    for q in order:
        faces, f = host[q]
        ops = [o1.cell_operator(faces[d], o1.DIRICHLET, o1.DIRICHLET) for d in range(3)]
        want = dec.solve(f, ops, lams[q], 1.0, "tpt")
        assert np.abs(alone[q] - want).max() <= 1e-9 * np.abs(want).max(), q
    for pl in plans:
        pl.destroy()


def test_repeated_plan_in_batch_is_serialised(fdi):
    # the same plan twice in one batch: its solves share a stream, in order
    import torch
    n = (48, 32, 64)
    faces = [tanh_faces(n[d], 1.4) for d in range(3)]
    plan = fdi.plan_create(faces, n, prec=fdi.PREC_MIXED_F16)
    a = torch.from_numpy(rhs_uniform(n[::-1], 3)).cuda()
    b = torch.from_numpy(rhs_uniform(n[::-1], 4)).cuda()
    oa, ob = torch.empty_like(a), torch.empty_like(b)
    stream = torch.cuda.Stream()
    for _ in range(3):
        with torch.cuda.stream(stream):
            fdi.helmholtz_solve_batched([plan, plan], [0.3, 0.01], [a, b], [oa, ob], stream)
        stream.synchronize()
    ops = [o1.cell_operator(faces[d], o1.DIRICHLET, o1.DIRICHLET) for d in range(3)]
    for o, f, lam in ((oa, rhs_uniform(n[::-1], 3), 0.3), (ob, rhs_uniform(n[::-1], 4), 0.01)):
        want = dec.solve(f, ops, lam, 1.0, "tpt")
        assert np.abs(o.cpu().numpy() - want).max() <= 1e-9 * np.abs(want).max()
    plan.destroy()


def test_autotune_keeps_results_and_seeds_new_plans(fdi):
    import torch
    n = (64, 48, 96)
    faces = [tanh_faces(n[d], 1.5) for d in range(3)]
    plan = fdi.plan_create(faces, n, prec=fdi.PREC_MIXED_F16)
    f = torch.from_numpy(rhs_uniform(n[::-1], 9)).cuda()
    before = torch.empty_like(f)
    fdi.helmholtz_solve(plan, 0.5, f, before)
    scratch = torch.empty_like(f)
    t = fdi.autotune(plan, 0.5, f, scratch, reps=2)
    assert t in (2, 3, 64, 128)
    after = torch.empty_like(f)
    fdi.helmholtz_solve(plan, 0.5, f, after)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    # every configuration computes the same bits
    for tt in (2, 3, 64, 128):
        fdi.set_thomas_config(plan, tt)
        o = torch.empty_like(f)
        fdi.helmholtz_solve(plan, 0.5, f, o)
        torch.cuda.synchronize()
        assert torch.equal(o, before), tt
    plan.destroy()
