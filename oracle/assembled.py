"""Assembled 3D operators and their direct solves (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The plain definition of what the fast solvers compute.  The discrete Laplacian
is the Kronecker sum of the 1D operators (Sec. 3, Eq. 23 in 2D and its 3D form
before Eq. 29), and the Helmholtz operator adds a multiple of the identity
(Eq. 27).  In the scaling used here the operator is

    A = sigma * I - lam * (D_x (+) D_y (+) D_z)

with sigma = 1, lam = dt/Re for the implicit viscous step (the paper's
H = Delta - I/dt of Eq. 1 multiplied by -dt, viscosity 1/Re), and sigma = 0,
lam = 1 for the Laplace problem -Delta u = f.

Fields are C-order arrays [n_z][n_y][n_x] flattened with x fastest, so the
flat index is (k*n_y + j)*n_x + i and D_x acts on the fastest index.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import operators1d as o1


def kron_sum(Dx, Dy, Dz):
    """Dx (+) Dy (+) Dz for C-order [z][y][x] flattening (Eq. 23 / Eq. 29)."""
    nx, ny, nz = Dx.shape[0], Dy.shape[0], Dz.shape[0]
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    Sx, Sy, Sz = sp.csr_matrix(Dx), sp.csr_matrix(Dy), sp.csr_matrix(Dz)
    return (sp.kron(Iz, sp.kron(Iy, Sx)) + sp.kron(Iz, sp.kron(Sy, Ix))
            + sp.kron(Sz, sp.kron(Iy, Ix))).tocsr()


def laplacian(ops):
    """Assembled Laplacian from three (m, K) 1D operators (x, y, z)."""
    Ds = [o1.second_derivative(m, K) for (m, K) in ops]
    return kron_sum(*Ds)


def helmholtz(ops, lam, sigma=1.0):
    """A = sigma*I - lam*Laplacian (Eq. 27 in the scaling of the module docstring)."""
    L = laplacian(ops)
    return (sigma * sp.identity(L.shape[0]) - lam * L).tocsr()


def cell_ops(faces, bc_lo, bc_hi):
    """Cell-kind (m, K) for the three directions of a box."""
    return [o1.cell_operator(faces[d], bc_lo[d], bc_hi[d]) for d in range(3)]


def volumes(ops):
    """Control-volume sizes (the diagonal of M_x (x) M_y (x) M_z), C-order flat."""
    mx, my, mz = (np.asarray(m) for (m, _) in ops)
    return np.einsum("k,j,i->kji", mz, my, mx).ravel()


def is_singular(ops, sigma):
    """-Delta with zero-flux walls on every side has the constants as null space."""
    if sigma != 0.0:
        return False
    return all(np.allclose(K.sum(axis=1), 0.0, atol=1e-12 * np.abs(K).max()) for (_, K) in ops)


def project_zero_mean(f, vol):
    """f - (V^T f / V^T 1) * 1 : the volume-weighted mean removed."""
    f = np.asarray(f, dtype=np.float64).ravel()
    return f - np.dot(vol, f) / vol.sum()


def solve(ops, f, lam, sigma=1.0):
    """Direct sparse solve of A u = f (the plain definition of the inverse).

    For the pure-Neumann Laplacian (sigma = 0, zero-flux walls everywhere) the
    operator is singular (Eq. 28 and Sec. 2 on the pressure being defined up to
    a constant); f is first projected to zero volume-weighted mean and the
    bordered system [A 1; V^T 0] picks the solution with V^T u = 0.
    """
    shape = tuple(m.size for (m, _) in ops)[::-1]
    f = np.asarray(f, dtype=np.float64).ravel()
    A = helmholtz(ops, lam, sigma)
    if is_singular(ops, sigma):
        vol = volumes(ops)
        fp = project_zero_mean(f, vol)
        N = A.shape[0]
        B = sp.bmat([[A, sp.csr_matrix(np.ones((N, 1)))],
                     [sp.csr_matrix(vol[None, :]), None]]).tocsc()
        u = spla.splu(B).solve(np.concatenate([fp, [0.0]]))[:N]
    else:
        u = spla.splu(A.tocsc()).solve(f)
    return u.reshape(shape)


def apply(ops, u, lam, sigma=1.0):
    """A u with the assembled matrix."""
    shape = np.shape(u)
    return (helmholtz(ops, lam, sigma) @ np.asarray(u).ravel()).reshape(shape)


def relative_residual(ops, u, f, lam, sigma=1.0):
    """||f - A u||_2 / ||f||_2 with the assembled matrix (f projected first in the
    singular Neumann case)."""
    f = np.asarray(f, dtype=np.float64).ravel()
    if is_singular(ops, sigma):
        f = project_zero_mean(f, volumes(ops))
    r = f - helmholtz(ops, lam, sigma) @ np.asarray(u).ravel()
    return float(np.linalg.norm(r) / np.linalg.norm(f))


def stencil_matrix_by_loops(faces, bc_lo, bc_hi, lam, sigma=1.0):
    """Dense A assembled cell by cell from face fluxes with plain Python loops.

    A second, independent route to the same operator as `helmholtz(cell_ops(...))`
    for tiny grids: for every cell and each of its six faces the flux is
    (u_nb - u_c) / distance (interior), (0 - u_c) / (h/2) at a Dirichlet wall and
    0 at a Neumann wall; the Laplacian is the net flux divided by the cell width
    in that direction.  Used only as a brute-force pin.
    """
    fx, fy, fz = (np.asarray(f, dtype=np.float64) for f in faces)
    n = (fx.size - 1, fy.size - 1, fz.size - 1)
    fcs = (fx, fy, fz)
    N = n[0] * n[1] * n[2]
    A = np.zeros((N, N))

    def flat(i, j, k):
        return (k * n[1] + j) * n[0] + i

    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                row = flat(i, j, k)
                A[row, row] += sigma
                idx = [i, j, k]
                for d in range(3):
                    f = fcs[d]
                    p = idx[d]
                    h = f[p + 1] - f[p]
                    cp = 0.5 * (f[p] + f[p + 1])
                    for side in (-1, +1):
                        q = p + side
                        if 0 <= q < n[d]:
                            cq = 0.5 * (f[q] + f[q + 1])
                            coef = 1.0 / abs(cq - cp) / h
                            nb = list(idx)
                            nb[d] = q
                            A[row, flat(*nb)] -= lam * coef
                            A[row, row] += lam * coef
                        else:
                            bc = bc_lo[d] if side < 0 else bc_hi[d]
                            if bc == o1.DIRICHLET:
                                A[row, row] += lam * (2.0 / h) / h
    return A
