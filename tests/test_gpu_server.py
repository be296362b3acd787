"""Serving runtime (fdi_server_*): Stokes-inverse requests with uneven grids,
differing dt / Re and both precisions, admitted by device-memory footprint and
run concurrently.  Each result must be the same alone and in the mix, and meet
its tolerance (checked against the oracle's assembled operators)."""
import numpy as np
import pytest

from oracle import stokes as st
from workloads import rhs_gaussian, tanh_faces

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


def mac_shapes(n):
    nx, ny, nz = n
    return [(nz, ny, nx - 1), (nz, ny - 1, nx), (nz - 1, ny, nx)], (nz, ny, nx)


def make_requests(count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(count):
        n = tuple(int(v) for v in rng.choice([12, 16, 20, 24, 32], size=3))
        dt = float(10.0 ** rng.uniform(-2.0, 3.0))
        Re = float(rng.choice([100.0, 1000.0, 5000.0]))
        prec = 3 if q % 3 else 0
        vs, ps = mac_shapes(n)
        f = [np.ascontiguousarray(rhs_gaussian(vs[c], 100 * q + c)) for c in range(3)]
        reqs.append((n, dt, Re, prec, f))
    return reqs


def run(fdi, reqs, slots, budget, alone):
    srv = fdi.Server(budget, slots)
    outs, tickets = [], []
    for (n, dt, Re, prec, f) in reqs:
        vs, ps = mac_shapes(n)
        u = [np.zeros(s) for s in vs]
        p = np.zeros(ps)
        t = srv.submit(n, 1.5, dt, Re, f, u, p, prec=prec)
        tickets.append(t)
        outs.append((u, p))
        if alone:
            srv.poll(t, wait=True)
    srv.drain()
    res = [srv.poll(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    return outs, res, stats


def test_same_alone_and_in_mix(fdi):
    reqs = make_requests(12, 0)
    a_out, a_res, _ = run(fdi, reqs, 1, 8 << 30, alone=True)
    m_out, m_res, stats = run(fdi, reqs, 4, 8 << 30, alone=False)
    for q, (n, dt, Re, prec, f) in enumerate(reqs):
        tol = 1e-11 if prec == 0 else 1e-10
        for r in (a_res[q], m_res[q]):
            assert r["state"] == 2 and r["status"] == 0 and r["rel_residual"] <= tol, (q, r)
        for c in range(3):
            assert np.array_equal(a_out[q][0][c], m_out[q][0][c]), (q, c)
        assert np.array_equal(a_out[q][1], m_out[q][1]), q
    assert stats["completed"] == len(reqs)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    # the saddle system itself, with the oracle's assembled operators
    for q in range(3):
        n, dt, Re, prec, f = reqs[q]
        faces = [tanh_faces(n[d], 1.5) for d in range(3)]
        mom, div = st.saddle_residual(faces, dt, Re, f, m_out[q][0], m_out[q][1])
        assert mom <= 1e-8 and div <= 1e-7, (q, mom, div)


def test_admission_by_footprint_and_eviction(fdi):
    reqs = make_requests(8, 1)
    need = max(fdi.stokes_plan_bytes_estimate(n, prec) + 8 * (2 * sum(np.prod(s) for s in mac_shapes(n)[0])
                                                              + np.prod(n)) for (n, _, _, prec, _) in reqs)
    budget = int(1.2 * need)  # one request at a time fits
    out, res, stats = run(fdi, reqs, 4, budget, alone=False)
    assert all(r["status"] == 0 and r["state"] == 2 for r in res)
    assert stats["peak_bytes"] <= budget
    keys = {(n, prec) for (n, _, _, prec, _) in reqs}
    if len(keys) > 1:
        assert stats["plans_evicted"] >= 1
    ref, _, _ = run(fdi, reqs, 1, 8 << 30, alone=True)
    for q in range(len(reqs)):
        assert np.array_equal(out[q][1], ref[q][1]), q


def test_rejects_request_above_budget(fdi):
    n = (32, 32, 32)
    vs, ps = mac_shapes(n)
    f = [np.zeros(s) for s in vs]
    u = [np.zeros(s) for s in vs]
    p = np.zeros(ps)
    srv = fdi.Server(1 << 20, 2)
    with pytest.raises(fdi.FdiError):
        srv.submit(n, 1.5, 1.0, 1000.0, f, u, p)
    srv.close()
