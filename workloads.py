"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the solution method: it only makes grids
(face coordinates) and right-hand sides from seeds, so that the CUDA path and
the CPU oracle see bit-identical inputs.

Grid recipe (the paper only says the finite-volume grid is "stretched near the
boundaries", Sec. 5.1): faces on [0, 1]

    x_i = 1/2 * (1 + tanh(beta * (2 i / n - 1)) / tanh(beta)),  i = 0..n,

with beta the stretching factor; beta = 0 gives the uniform grid.

Right-hand sides: numpy.random.default_rng(seed), uniform[-1, 1] or standard
normal, in FP64, C-order [n_z][n_y][n_x] (x fastest).
"""
from __future__ import annotations

import numpy as np


def tanh_faces(n: int, beta: float) -> np.ndarray:
    """n + 1 ascending face coordinates on [0, 1], clustered at both walls."""
    if n < 1:
        raise ValueError("n must be >= 1")
    s = np.arange(n + 1, dtype=np.float64) / n
    if beta == 0.0:
        x = s.copy()
    else:
        x = 0.5 * (1.0 + np.tanh(beta * (2.0 * s - 1.0)) / np.tanh(beta))
    x[0], x[-1] = 0.0, 1.0
    return x


def box_faces(n, beta):
    """Face lists for a box with n = (n_x, n_y, n_z) cells and stretching beta
    (scalar or per-direction)."""
    betas = beta if np.ndim(beta) else (beta, beta, beta)
    return [tanh_faces(int(n[d]), float(betas[d])) for d in range(3)]


def rhs_uniform(shape, seed: int) -> np.ndarray:
    """i.i.d. uniform[-1, 1] FP64 field of the given C-order shape."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=tuple(shape))


def rhs_gaussian(shape, seed: int) -> np.ndarray:
    """i.i.d. N(0, 1) FP64 field of the given C-order shape."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=tuple(shape))


def mac_shapes(n):
    """C-order shapes (z, y, x) of the staggered u, v, w and p fields for n cells."""
    nx, ny, nz = n
    return {
        "u": (nz, ny, nx - 1),
        "v": (nz, ny - 1, nx),
        "w": (nz - 1, ny, nx),
        "p": (nz, ny, nx),
    }


def mixed_shape_batch(count: int, seed: int, sizes=(32, 48, 64, 96, 128, 160),
                      max_aspect: float = 4.0):
    """Draw `count` problems (n, beta, lambda) for a batch of uneven grids.

    n_d is drawn from `sizes` per direction, redrawn until max/min <= max_aspect;
    beta ~ U[1, 2]; lambda log-uniform in [1e-4, 1].
    """
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = tuple(int(v) for v in rng.choice(sizes, size=3))
        if max(n) / min(n) > max_aspect:
            continue
        beta = float(rng.uniform(1.0, 2.0))
        lam = float(10.0 ** rng.uniform(-4.0, 0.0))
        out.append((n, beta, lam))
    return out


def poisson_arrivals(count: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given mean rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
