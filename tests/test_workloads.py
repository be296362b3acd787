"""The seeded synthetic inputs stand in for the paper's workloads (Sec. 5): the
stretched faces, the right-hand sides, the uneven-grid batch and the serving
arrival process follow their stated recipes and are reproducible."""
import numpy as np

import workloads as w


def test_tanh_faces_cluster_at_both_walls():
    for n, beta in ((16, 1.5), (256, 2.0)):
        x = w.tanh_faces(n, beta)
        h = np.diff(x)
        assert x[0] == 0.0 and abs(x[-1] - 1.0) < 1e-15 and np.all(h > 0)
        # symmetric about the centre, smallest cells at the walls
        assert np.allclose(x + x[::-1], 1.0, atol=1e-15)
        assert abs(h[0] - h.min()) <= 1e-15 and abs(h[n // 2 - 1] - h.max()) <= 1e-14
    # beta = 0: uniform
    assert np.allclose(np.diff(w.tanh_faces(8, 0.0)), 1.0 / 8)


def test_rhs_generators_are_seeded():
    a = w.rhs_uniform((4, 5, 6), 3)
    assert np.array_equal(a, w.rhs_uniform((4, 5, 6), 3))
    assert not np.array_equal(a, w.rhs_uniform((4, 5, 6), 4))
    assert a.dtype == np.float64 and a.min() >= -1.0 and a.max() <= 1.0
    g = w.rhs_gaussian((200, 200), 1)
    assert abs(g.mean()) < 0.02 and abs(g.std() - 1.0) < 0.02


def test_uneven_batch_recipe():
    # grids from {32, ..., 160} per direction with aspect <= 4, beta ~ U[1, 2],
    # lambda log-uniform in [1e-4, 1]
    probs = w.mixed_shape_batch(64, 0)
    assert probs == w.mixed_shape_batch(64, 0) and len(probs) == 64
    sizes = {32, 48, 64, 96, 128, 160}
    for n, beta, lam in probs:
        assert set(n) <= sizes and max(n) / min(n) <= 4.0
        assert 1.0 <= beta <= 2.0 and 1e-4 <= lam <= 1.0
    lams = np.log10([p[2] for p in probs])
    assert lams.min() < -3.0 and lams.max() > -1.0  # spread over the decades


def test_poisson_arrivals_rate():
    t = w.poisson_arrivals(2000, 200.0, 0)
    assert np.all(np.diff(t) > 0)
    assert abs(2000 / t[-1] - 200.0) < 15.0
    assert np.array_equal(t, w.poisson_arrivals(2000, 200.0, 0))
