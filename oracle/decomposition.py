"""Lynch eigenvalue-decomposition solvers TPF and TPT, done naively (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3 of the paper:
  * each 1D operator is diagonalised once, D = E Lambda E^{-1} (Eq. 24);
  * TPF: u = (E_x (x) E_y (x) E_z) Lambda^{-1} (E_x^{-1} (x) E_y^{-1} (x) E_z^{-1}) f
    with Lambda_ijk the sum of the 1D eigenvalues (Eq. 25, 26, 29), shifted for
    the Helmholtz operator (Eq. 27);
  * Neumann problem: a zero Lambda_ijk is replaced by 1 (Eq. 28);
  * TPT: the eigen decomposition in one direction is replaced by the Thomas
    algorithm on the 3-point stencil (Haidvogel-Zang, end of Sec. 3).

In the operator scaling A = sigma*I - lam*Laplacian (see oracle/assembled.py)
the divisor of mode (i, j, k) is sigma - lam*(Lx_i + Ly_j + Lz_k).

The generalised form: D = M^{-1} K with M diagonal and K symmetric, so
S = M^{-1/2} K M^{-1/2} = Q Lambda Q^T is a symmetric eigenproblem and
E = M^{-1/2} Q, E^{-1} = Q^T M^{1/2}.

Reading of Eq. 28 used here: for the zero-flux operator the null eigenpair is
known exactly (Lambda = 0, constant eigenvector), so it is set exactly instead
of trusting a computed eigenvalue of size 1e-13, and the other eigenvectors are
projected onto its M-orthogonal complement (eigenvectors of the symmetric
pencil (K, M) are M-orthogonal to it); the right-hand side of the
singular problem is projected to zero volume-weighted mean first, after which
Eq. 28's "divide by 1" leaves the null-mode coefficient at (rounding-level)
zero.  In TPT the singular Thomas line (null mode in both transformed
directions) is solved with its first unknown pinned to zero, then shifted to
zero weighted mean.
"""
from __future__ import annotations

import numpy as np

from . import assembled as asm


def generalized_eig(m, K):
    """(lam, E, Einv) with K E = M E diag(lam) and Einv = E^{-1} (Eq. 24)."""
    m = np.asarray(m, dtype=np.float64)
    s = np.sqrt(m)
    S = K / s[:, None] / s[None, :]
    S = 0.5 * (S + S.T)
    lam, Q = np.linalg.eigh(S)
    if np.allclose(K.sum(axis=1), 0.0, atol=1e-12 * np.abs(K).max()):
        # zero-flux operator: exact null pair (constant vector, Lambda = 0)
        i0 = int(np.argmin(np.abs(lam)))
        lam[i0] = 0.0
        q0 = s / np.linalg.norm(s)
        if np.dot(q0, Q[:, i0]) < 0:
            q0 = -q0
        Q[:, i0] = q0
        # the other eigenvectors are orthogonal to the exact null vector: remove
        # the component rounding left along it
        others = [k for k in range(Q.shape[1]) if k != i0]
        Q[:, others] -= np.outer(q0, q0 @ Q[:, others])
        Q[:, others] /= np.linalg.norm(Q[:, others], axis=0)[None, :]
    E = Q / s[:, None]
    Einv = Q.T * s[None, :]
    return lam, E, Einv


def _apply_along(T, f, axis):
    """Contract matrix T with array f along `axis` (out[..i..] = sum_j T[i,j] f[..j..])."""
    return np.moveaxis(np.tensordot(T, f, axes=([1], [axis])), 0, axis)


# direction d (0 = x, 1 = y, 2 = z) lives on C-order array axis 2 - d
def _axis(d):
    return 2 - d


def tpf_solve(f, ops, lam, sigma=1.0):
    """TPF: eigen decomposition in all three directions (Eq. 29 with Eq. 27/28)."""
    f = np.array(f, dtype=np.float64)
    singular = asm.is_singular(ops, sigma)
    if singular:
        f = asm.project_zero_mean(f, asm.volumes(ops)).reshape(f.shape)
    eig = [generalized_eig(m, K) for (m, K) in ops]
    g = f
    for d in range(3):
        g = _apply_along(eig[d][2], g, _axis(d))          # E_d^{-1}
    Lx, Ly, Lz = eig[0][0], eig[1][0], eig[2][0]
    Lsum = Lz[:, None, None] + Ly[None, :, None] + Lx[None, None, :]
    div = sigma - lam * Lsum
    if singular:
        div = np.where(Lsum == 0.0, 1.0, div)              # Eq. 28
    g = g / div
    for d in range(3):
        g = _apply_along(eig[d][1], g, _axis(d))          # E_d
    return g


def thomas(lower, diag, upper, rhs):
    """Thomas algorithm for tridiagonal systems, vectorised over trailing axes.

    lower[k] multiplies u[k-1], upper[k] multiplies u[k]+1 (lower[0], upper[-1]
    unused); diag and rhs have the line index as axis 0.
    """
    n = diag.shape[0]
    cp = np.empty_like(diag)
    dp = np.empty_like(rhs)
    cp[0] = upper[0] / diag[0]
    dp[0] = rhs[0] / diag[0]
    for k in range(1, n):
        den = diag[k] - lower[k] * cp[k - 1]
        cp[k] = upper[k] / den if k < n - 1 else 0.0
        dp[k] = (rhs[k] - lower[k] * dp[k - 1]) / den
    u = np.empty_like(rhs)
    u[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        u[k] = dp[k] - cp[k] * u[k + 1]
    return u


def tpt_solve(f, ops, lam, sigma=1.0, thomas_dir=2):
    """TPT: eigen decomposition in two directions, Thomas along `thomas_dir`
    (end of Sec. 3).  Each line (a, b) of transformed modes solves

        [(sigma - lam*(L_a + L_b)) M_t - lam K_t] u = M_t f_hat
    """
    f = np.array(f, dtype=np.float64)
    singular = asm.is_singular(ops, sigma)
    if singular:
        f = asm.project_zero_mean(f, asm.volumes(ops)).reshape(f.shape)
    t = thomas_dir
    others = [d for d in range(3) if d != t]
    eig = {d: generalized_eig(*ops[d]) for d in others}
    g = f
    for d in others:
        g = _apply_along(eig[d][2], g, _axis(d))
    # bring the Thomas axis to the front: shape (n_t, *rest)
    g = np.moveaxis(g, _axis(t), 0)
    rest_shape = g.shape[1:]
    # sum of the two transformed eigenvalues on the remaining axes (in C order)
    ax = sorted(others, reverse=True)          # remaining array axes are in C order
    La = eig[ax[0]][0]
    Lb = eig[ax[1]][0]
    Lab = La[:, None] + Lb[None, :]
    m_t, K_t = ops[t]
    n_t = m_t.size
    s = sigma - lam * Lab                      # per-line shift, shape rest_shape
    diag = s[None, :, :] * m_t[:, None, None] - lam * np.diag(K_t)[:, None, None]
    off = -lam * np.diag(K_t, 1)
    lower = np.zeros(n_t)
    upper = np.zeros(n_t)
    lower[1:] = off
    upper[:-1] = off
    rhs = m_t[:, None, None] * g
    lower_b = np.broadcast_to(lower[:, None, None], diag.shape)
    upper_b = np.broadcast_to(upper[:, None, None], diag.shape)
    if singular:
        null = (Lab == 0.0)
        ii = np.argwhere(null)
        u = np.empty_like(rhs)
        regular = ~null
        # regular lines
        u[:, regular] = thomas(lower_b[:, regular], diag[:, regular],
                               upper_b[:, regular], rhs[:, regular])
        for (a, b) in ii:
            r = g[:, a, b] - np.dot(m_t, g[:, a, b]) / m_t.sum()
            line = np.zeros(n_t)
            line[1:] = thomas(lower[1:], diag[1:, a, b], upper[1:], (m_t * r)[1:])
            line -= np.dot(m_t, line) / m_t.sum()
            u[:, a, b] = line
    else:
        u = thomas(lower_b, diag, upper_b, rhs)
    g = np.moveaxis(u.reshape((n_t,) + rest_shape), 0, _axis(t))
    for d in others:
        g = _apply_along(eig[d][1], g, _axis(d))
    return g


def solve(f, ops, lam, sigma=1.0, method="tpt", thomas_dir=2):
    if method == "tpf":
        return tpf_solve(f, ops, lam, sigma)
    if method == "tpt":
        return tpt_solve(f, ops, lam, sigma, thomas_dir)
    raise ValueError(method)
