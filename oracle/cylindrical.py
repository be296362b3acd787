"""Helmholtz / Poisson operators in cylindrical coordinates and their
eigen-decomposition inverses (oracle, FP64; Sec. 6, Eq. 41-46).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The Laplacian in cylindrical coordinates (Eq. 41),
    D_rr u + (1/r^2) D_thth u + D_zz u,   D_rr = (1/r) d/dr (r d/dr),
does not split into a Kronecker sum because of the 1/r^2 factor; the paper
diagonalises the theta and z directions (Eq. 42-43) and is left, for each pair
of modes (m, n), with one radial problem (Eq. 44) solved by the Thomas
algorithm (TPT), or diagonalises the M radial operators D_rr + lambda_th,m/r^2
as well (Eq. 45) and divides (Eq. 46, TPF).

Finite-volume reading used here (the paper prints no stencil):
  cells (r_i, theta_j, z_k), C order [k][j][i] (r fastest);
  radial faces rho_0 < ... < rho_K (rho_0 = 0 is the axis: its face has zero
  area, so no flux crosses it), centres c_i, annular areas
  A_i = (rho_{i+1}^2 - rho_i^2) / 2;
  radial flux through face rho_{i+1}: rho_{i+1} (u_{i+1} - u_i) / (c_{i+1} - c_i);
  a Dirichlet wall (value 0) at rho_0 > 0 or rho_K: flux over half a cell;
  M_r = diag(A_i), K_r the symmetric flux matrix, D_rr = M_r^{-1} K_r;
  theta: M uniform cells on the full circle (periodic), D_thth the periodic
  second difference / h_th^2;  the 1/r^2 of Eq. 41 becomes, per radial cell,
  g_i = h_r,i / (c_i A_i) (the arc flux h_r h_z / (c_i h_th) divided by the
  cell volume A_i h_th h_z), which tends to 1 / c_i^2;
  z: the cell operator of operators1d.
So the discrete operator is
  L = D_rr (x) I (x) I + diag(g) (x) D_thth (x) I + I (x) I (x) D_zz
(written in the r, theta, z order of Eq. 44) and A = sigma I - lambda L.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import decomposition as dec
from . import operators1d as o1

DIRICHLET = o1.DIRICHLET
NEUMANN = o1.NEUMANN


def radial_operator(rfaces, bc_in=DIRICHLET, bc_out=DIRICHLET):
    """(A, K, g) of the radial operator D_rr = diag(A)^-1 K and the theta
    coefficient g (the discrete 1/r^2).  rfaces[0] = 0 makes the inner boundary
    the axis (bc_in is then ignored: no flux through a face of zero area)."""
    rho = np.asarray(rfaces, dtype=np.float64)
    if rho.ndim != 1 or rho.size < 2 or np.any(np.diff(rho) <= 0) or rho[0] < 0:
        raise ValueError("radial faces must be ascending and non-negative")
    h = np.diff(rho)
    c = 0.5 * (rho[:-1] + rho[1:])
    A = 0.5 * (rho[1:] ** 2 - rho[:-1] ** 2)
    n = h.size
    K = np.zeros((n, n))
    for i in range(n - 1):
        w = rho[i + 1] / (c[i + 1] - c[i])
        K[i, i + 1] += w
        K[i + 1, i] += w
        K[i, i] -= w
        K[i + 1, i + 1] -= w
    if rho[0] > 0 and bc_in == DIRICHLET:
        K[0, 0] -= rho[0] / (0.5 * h[0])
    if bc_out == DIRICHLET:
        K[n - 1, n - 1] -= rho[n] / (0.5 * h[n - 1])
    g = h / (c * A)
    return A, K, g


def periodic_operator(M):
    """Periodic second difference on M uniform cells of the full circle
    (h = 2 pi / M): (m, K) with D_thth = diag(m)^-1 K, m = h."""
    h = 2.0 * np.pi / M
    K = np.zeros((M, M))
    for j in range(M):
        K[j, j] -= 2.0 / h
        K[j, (j + 1) % M] += 1.0 / h
        K[j, (j - 1) % M] += 1.0 / h
    return np.full(M, h), K


def _dense_D(m, K):
    return K / np.asarray(m)[:, None]


def assembled(rfaces, M, zfaces, bc_r=(DIRICHLET, DIRICHLET), bc_z=(DIRICHLET, DIRICHLET)):
    """Sparse L of the module docstring, rows in C order [k][j][i] (Eq. 41)."""
    A, Kr, g = radial_operator(rfaces, *bc_r)
    mt, Kt = periodic_operator(M)
    mz, Kz = o1.cell_operator(zfaces, *bc_z)
    Dr = sp.csr_matrix(_dense_D(A, Kr))
    Dt = sp.csr_matrix(_dense_D(mt, Kt))
    Dz = sp.csr_matrix(_dense_D(mz, Kz))
    Ir, It, Iz = sp.identity(A.size), sp.identity(M), sp.identity(mz.size)
    # C order [k][j][i]: kron(z, theta, r)
    L = sp.kron(Iz, sp.kron(It, Dr)) + sp.kron(Iz, sp.kron(Dt, sp.diags(g))) + sp.kron(Dz, sp.kron(It, Ir))
    return L.tocsr()


def volumes(rfaces, M, zfaces):
    """Cell volumes A_i h_th h_z,k in C order [k][j][i]."""
    A, _, _ = radial_operator(rfaces)
    hz, _ = o1.widths_centres(zfaces)
    return (hz[:, None, None] * np.full(M, 2.0 * np.pi / M)[None, :, None] * A[None, None, :]).ravel()


def direct_solve(f, rfaces, M, zfaces, lam, sigma=1.0, bc_r=(DIRICHLET, DIRICHLET), bc_z=(DIRICHLET, DIRICHLET)):
    """(sigma I - lam L) u = f by a sparse direct solve: the plain definition."""
    L = assembled(rfaces, M, zfaces, bc_r, bc_z)
    A = sigma * sp.identity(L.shape[0]) - lam * L
    return spla.spsolve(A.tocsc(), np.ravel(f)).reshape(np.shape(f))


def _theta_z_transforms(M, zfaces, bc_z):
    mt, Kt = periodic_operator(M)
    lt, Et, Eti = dec.generalized_eig(mt, Kt)
    mz, Kz = o1.cell_operator(zfaces, *bc_z)
    lz, Ez, Ezi = dec.generalized_eig(mz, Kz)
    return (lt, Et, Eti), (lz, Ez, Ezi)


def _check_regular(rfaces, bc_r, bc_z, sigma):
    closed_r = (rfaces[0] == 0 or bc_r[0] == NEUMANN) and bc_r[1] == NEUMANN
    if sigma == 0.0 and closed_r and tuple(bc_z) == (NEUMANN, NEUMANN):
        raise ValueError("the zero-flux Laplacian is singular; not handled by this oracle")


def tpt_solve(f, rfaces, M, zfaces, lam, sigma=1.0, bc_r=(DIRICHLET, DIRICHLET), bc_z=(DIRICHLET, DIRICHLET)):
    """Eq. 42-44: transform along theta and z (E^{-1}), one tridiagonal radial
    problem [sigma - lam (D_rr + lambda_th,m g + lambda_z,n)] a = f_hat per
    (m, n) solved by the Thomas algorithm (multiplied by diag(A) to make it
    symmetric), transform back."""
    _check_regular(rfaces, bc_r, bc_z, sigma)
    A, Kr, g = radial_operator(rfaces, *bc_r)
    (lt, Et, Eti), (lz, Ez, Ezi) = _theta_z_transforms(M, zfaces, bc_z)
    F = np.asarray(f, dtype=np.float64)                        # [k][j][i]
    Fh = np.einsum("nk,mj,kji->nmi", Ezi, Eti, F)              # [n][m][i]
    nr = A.size
    diag0 = np.diag(Kr)
    off = np.array([Kr[i, i + 1] for i in range(nr - 1)])
    # per (n, m): (sigma A - lam K_r - lam lambda_th,m A g - lam lambda_z,n A) a = A f_hat
    D = (sigma * A[None, None, :] - lam * diag0[None, None, :] - lam * lt[None, :, None] * (A * g)[None, None, :]
         - lam * lz[:, None, None] * A[None, None, :])
    lower = np.zeros(nr)
    upper = np.zeros(nr)
    lower[1:] = -lam * off
    upper[:-1] = -lam * off
    rhs = A[None, None, :] * Fh
    # Thomas along the radial index (axis 0 of the arrays handed to it)
    a = dec.thomas(np.broadcast_to(lower[:, None, None], (nr,) + D.shape[:2]),
                   np.moveaxis(D, 2, 0), np.broadcast_to(upper[:, None, None], (nr,) + D.shape[:2]),
                   np.moveaxis(rhs, 2, 0))
    a = np.moveaxis(a, 0, 2)                                   # [n][m][i]
    return np.einsum("kn,jm,nmi->kji", Ez, Et, a)


def tpf_solve(f, rfaces, M, zfaces, lam, sigma=1.0, bc_r=(DIRICHLET, DIRICHLET), bc_z=(DIRICHLET, DIRICHLET)):
    """Eq. 45-46: besides theta and z, the radial operator of every theta mode,
    D_rr + lambda_th,m diag(g), is diagonalised (M generalised eigenproblems with
    the same diag(A)); the coefficient (i, m, n) is divided by
    sigma - lam (lambda_i,m + lambda_z,n)."""
    _check_regular(rfaces, bc_r, bc_z, sigma)
    A, Kr, g = radial_operator(rfaces, *bc_r)
    (lt, Et, Eti), (lz, Ez, Ezi) = _theta_z_transforms(M, zfaces, bc_z)
    F = np.asarray(f, dtype=np.float64)
    Fh = np.einsum("nk,mj,kji->nmi", Ezi, Eti, F)              # [n][m][i]
    out = np.empty_like(Fh)
    for m in range(M):
        lr, Er, Eri = dec.generalized_eig(A, Kr + lt[m] * np.diag(A * g))
        coef = Fh[:, m, :] @ Eri.T                             # [n][i']
        coef = coef / (sigma - lam * (lr[None, :] + lz[:, None]))
        out[:, m, :] = coef @ Er.T
    return np.einsum("kn,jm,nmi->kji", Ez, Et, out)
