"""1D finite-volume operators on a stretched orthogonal grid (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper writes the discrete Laplacian as a Kronecker sum of 1D second
derivative operators D_xx, D_yy, D_zz (Sec. 3, Eq. 23 and Eq. 29) on an
orthogonal, stretched, staggered finite-volume grid (Sec. 5.1), and the
staggered first derivatives as 1D operators D_u^x, D_p^x (Sec. 4, Eq. 30-31).
It does not print the 1D stencils; the finite-volume reading used here is:

  faces x_0 < ... < x_n, widths h_i = x_{i+1} - x_i, centres c_i (0-based).

  cell kind (n unknowns at cell centres):
      (D u)_i = [ (u_{i+1}-u_i)/(c_{i+1}-c_i) - (u_i-u_{i-1})/(c_i-c_{i-1}) ] / h_i
      Dirichlet wall (value 0): wall flux (u_0 - 0)/(h_0/2)   (half-cell distance)
      Neumann wall: zero flux.
  face kind (n-1 unknowns at the interior faces x_1..x_{n-1}, walls u=0):
      (D u)_j = [ (u_{j+1}-u_j)/h_j - (u_j-u_{j-1})/h_{j-1} ] / (c_j - c_{j-1})

Each operator is returned as D = M^{-1} K with M diagonal (control-volume
widths) and K symmetric tridiagonal, so that the generalised eigenproblem
K q = Lambda M q is symmetric-definite (the form used for Eq. 24).

Staggered first derivatives (Sec. 2: divergence uses the velocity boundary
values, the pressure gradient uses no pressure boundary value):
      div  (cells <- faces): (D u)_i = (u_{i+1} - u_i) / h_i,   u_0 = u_n = 0
      grad (faces <- cells): (G p)_j = (p_j - p_{j-1}) / (c_j - c_{j-1})
so that div*grad is the cell-Neumann operator and grad*div the face operator.
"""
from __future__ import annotations

import numpy as np

DIRICHLET = 0
NEUMANN = 1


def widths_centres(faces):
    x = np.asarray(faces, dtype=np.float64)
    if x.ndim != 1 or x.size < 2 or np.any(np.diff(x) <= 0):
        raise ValueError("faces must be a strictly ascending 1D array of length >= 2")
    h = np.diff(x)
    c = 0.5 * (x[:-1] + x[1:])
    return h, c


def cell_operator(faces, bc_lo=DIRICHLET, bc_hi=DIRICHLET):
    """(m, K) of the cell-centred second derivative: D = diag(m)^-1 K.

    Sec. 3 (Eq. 23) with the finite-volume fluxes listed in the module docstring.
    """
    h, c = widths_centres(faces)
    n = h.size
    K = np.zeros((n, n))
    for i in range(n - 1):
        g = 1.0 / (c[i + 1] - c[i])
        K[i, i + 1] += g
        K[i + 1, i] += g
        K[i, i] -= g
        K[i + 1, i + 1] -= g
    if bc_lo == DIRICHLET:
        K[0, 0] -= 2.0 / h[0]
    if bc_hi == DIRICHLET:
        K[n - 1, n - 1] -= 2.0 / h[n - 1]
    return h.copy(), K


def face_operator(faces):
    """(m, K) of the second derivative for unknowns on the n-1 interior faces
    (staggered normal velocity component), walls u = 0.  Sec. 2, D1 of Eq. 1."""
    h, c = widths_centres(faces)
    n = h.size
    if n < 2:
        raise ValueError("face operator needs n >= 2 cells")
    m = c[1:] - c[:-1]          # dual widths of faces 1..n-1
    K = np.zeros((n - 1, n - 1))
    # cell i joins faces i and i+1 with coefficient 1/h_i; faces 0 and n are walls
    for i in range(n):
        g = 1.0 / h[i]
        a, b = i - 1, i          # unknown indices of faces i and i+1
        if 0 <= a < n - 1:
            K[a, a] -= g
        if 0 <= b < n - 1:
            K[b, b] -= g
        if 0 <= a < n - 1 and 0 <= b < n - 1:
            K[a, b] += g
            K[b, a] += g
    return m, K


def second_derivative(m, K):
    """D = M^{-1} K as a dense matrix."""
    return K / np.asarray(m)[:, None]


def div_1d(faces):
    """Divergence along one direction, cells <- interior faces (Eq. 30's D_u^x)."""
    h, _ = widths_centres(faces)
    n = h.size
    D = np.zeros((n, n - 1))
    for i in range(n):
        if i < n - 1:
            D[i, i] += 1.0 / h[i]      # + u_{i+1}  (face i+1 -> column i)
        if i > 0:
            D[i, i - 1] -= 1.0 / h[i]  # - u_i      (face i   -> column i-1)
    return D


def grad_1d(faces):
    """Pressure gradient along one direction, interior faces <- cells (Eq. 31's D_p^x)."""
    _, c = widths_centres(faces)
    n = c.size
    G = np.zeros((n - 1, n))
    for j in range(1, n):
        g = 1.0 / (c[j] - c[j - 1])
        G[j - 1, j] += g
        G[j - 1, j - 1] -= g
    return G


def operator_for(faces, kind, bc_lo=DIRICHLET, bc_hi=DIRICHLET):
    """(m, K) for kind 'cell' (with wall types) or 'face' (no-slip walls)."""
    if kind == "cell":
        return cell_operator(faces, bc_lo, bc_hi)
    if kind == "face":
        return face_operator(faces)
    raise ValueError(kind)
