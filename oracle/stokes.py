"""Staggered (MAC) Stokes operator and its inverses (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2, Eq. 8: the semi-implicit Stokes system [H_c  -grad_c p ; div u = 0].
Scaling used here (the paper's Eq. 8 multiplied by -dt, viscosity 1/Re):

    (I - lam*Delta_c) u_c + dt * (G p)_c = f_c,  c in {u, v, w},   D u = 0,
    lam = dt / Re,

on a staggered grid with no-slip walls: u on the interior x-faces, v on the
interior y-faces, w on the interior z-faces, p at cell centres.  The velocity
Laplacian of component c uses the face operator along c and the cell-Dirichlet
operator across it; D and G are the staggered div and grad of
oracle/operators1d.py.  Pressure is defined up to a constant (Sec. 2); it is
returned with zero volume-weighted mean.

The three-step semi-direct inverse (Sec. 2, 3D steps after Eq. 9), with q = dt*p:
  1. u_hat_c = H_c^{-1} f_c
  2. solve C q = D u_hat,  C = sum_c D_c H_c^{-1} G_c   (Eq. 9, the pressure matrix)
  3. u_c = u_hat_c - H_c^{-1} (G q)_c
Step 2 is solved by a Krylov method preconditioned by the inverse pressure
Laplacian L_p = D G (Sec. 2, after Eq. 9): plain BiCGstab (van der Vorst), the
paper's BiCGstab(2) (Sleijpen & Fokkema's BiCGstab(ell), ell = 2), or
conjugate gradients in the volume-weighted inner product.  C is not symmetric
as a matrix (Sec. 2) but it is self-adjoint in that inner product: D is minus
the volume-weighted adjoint of G, and M_u H_c^{-1} is symmetric, so
V C = -G^T (M_u H^{-1}) G with V the cell volumes; -C is positive definite on
the zero-mean pressures, and so are -L_p^{-1} and -L_p^{-1} + lam*I.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assembled as asm
from . import decomposition as dec
from . import operators1d as o1

COMPONENTS = ("u", "v", "w")


def component_ops(faces, c):
    """Three (m, K) 1D operators (x, y, z) of velocity component c (0, 1, 2)."""
    ops = []
    for d in range(3):
        if d == c:
            ops.append(o1.face_operator(faces[d]))
        else:
            ops.append(o1.cell_operator(faces[d], o1.DIRICHLET, o1.DIRICHLET))
    return ops


def pressure_ops(faces):
    return [o1.cell_operator(faces[d], o1.NEUMANN, o1.NEUMANN) for d in range(3)]


def _kron3(Az, Ay, Ax):
    return sp.kron(sp.csr_matrix(Az), sp.kron(sp.csr_matrix(Ay), sp.csr_matrix(Ax))).tocsr()


def div_grad_3d(faces):
    """Sparse D_c (cells <- component c) and G_c (component c <- cells), Eq. 30-31."""
    n = [len(f) - 1 for f in faces]
    I = [sp.identity(n[d]) for d in range(3)]
    Dd = [o1.div_1d(faces[d]) for d in range(3)]
    Gd = [o1.grad_1d(faces[d]) for d in range(3)]
    D = [_kron3(I[2], I[1], Dd[0]), _kron3(I[2], Dd[1], I[0]), _kron3(Dd[2], I[1], I[0])]
    G = [_kron3(I[2], I[1], Gd[0]), _kron3(I[2], Gd[1], I[0]), _kron3(Gd[2], I[1], I[0])]
    return D, G


def shapes(faces):
    nx, ny, nz = (len(f) - 1 for f in faces)
    return [(nz, ny, nx - 1), (nz, ny - 1, nx), (nz - 1, ny, nx)], (nz, ny, nx)


def saddle_matrix(faces, dt, Re):
    """Assembled Stokes matrix of Eq. 8 in the scaling of the module docstring."""
    lam = dt / Re
    H = [asm.helmholtz(component_ops(faces, c), lam) for c in range(3)]
    D, G = div_grad_3d(faces)
    return sp.bmat([[H[0], None, None, dt * G[0]],
                    [None, H[1], None, dt * G[1]],
                    [None, None, H[2], dt * G[2]],
                    [D[0], D[1], D[2], None]]).tocsr()


def _split(x, faces):
    vs, ps = shapes(faces)
    out, o = [], 0
    for s in vs + [ps]:
        sz = int(np.prod(s))
        out.append(x[o:o + sz].reshape(s))
        o += sz
    return out


def stokes_direct(faces, dt, Re, f):
    """Direct sparse solve of the bordered saddle system (the plain definition).

    The extra unknown mu multiplies a column of ones on the continuity rows and
    the extra row imposes zero volume-weighted mean pressure.
    """
    S = saddle_matrix(faces, dt, Re)
    vs, ps = shapes(faces)
    nv = sum(int(np.prod(s)) for s in vs)
    npr = int(np.prod(ps))
    vol = asm.volumes(pressure_ops(faces))
    col = np.zeros((S.shape[0], 1))
    col[nv:, 0] = 1.0
    row = np.zeros((1, S.shape[0]))
    row[0, nv:] = vol
    B = sp.bmat([[S, sp.csr_matrix(col)], [sp.csr_matrix(row), None]]).tocsc()
    rhs = np.concatenate([np.ravel(fc) for fc in f] + [np.zeros(npr), [0.0]])
    x = spla.splu(B).solve(rhs)[:-1]
    u, v, w, p = _split(x, faces)
    return (u, v, w), p


def saddle_residual(faces, dt, Re, f, vel, p):
    """(momentum relative residual, ||D u||_2 / ||u||_2) with assembled operators."""
    lam = dt / Re
    D, G = div_grad_3d(faces)
    num = 0.0
    den = 0.0
    for c in range(3):
        Hc = asm.helmholtz(component_ops(faces, c), lam)
        r = np.ravel(f[c]) - Hc @ np.ravel(vel[c]) - dt * (G[c] @ np.ravel(p))
        num += float(np.dot(r, r))
        den += float(np.dot(np.ravel(f[c]), np.ravel(f[c])))
    div = sum(D[c] @ np.ravel(vel[c]) for c in range(3))
    un = np.sqrt(sum(float(np.dot(np.ravel(vel[c]), np.ravel(vel[c]))) for c in range(3)))
    return float(np.sqrt(num / den)), float(np.linalg.norm(div) / max(un, 1e-300))


def pressure_matrix(faces, dt, Re):
    """Dense C = sum_c D_c H_c^{-1} G_c (Eq. 9), for tiny grids."""
    lam = dt / Re
    D, G = div_grad_3d(faces)
    C = None
    for c in range(3):
        Hc = asm.helmholtz(component_ops(faces, c), lam).tocsc()
        X = spla.splu(Hc).solve(G[c].toarray())
        term = D[c] @ X
        C = term if C is None else C + term
    return np.asarray(C)


def stokes_three_step_dense(faces, dt, Re, f):
    """The three steps of Sec. 2 with an explicitly formed dense C (tiny grids)."""
    lam = dt / Re
    D, G = div_grad_3d(faces)
    Hs = [spla.splu(asm.helmholtz(component_ops(faces, c), lam).tocsc()) for c in range(3)]
    uhat = [Hs[c].solve(np.ravel(f[c])) for c in range(3)]
    b = sum(D[c] @ uhat[c] for c in range(3))
    C = pressure_matrix(faces, dt, Re)
    vol = asm.volumes(pressure_ops(faces))
    N = C.shape[0]
    B = np.zeros((N + 1, N + 1))
    B[:N, :N] = C
    B[:N, N] = 1.0
    B[N, :N] = vol
    q = np.linalg.solve(B, np.concatenate([b, [0.0]]))[:N]
    vs, ps = shapes(faces)
    vel = [(uhat[c] - Hs[c].solve(G[c] @ q)).reshape(vs[c]) for c in range(3)]
    return tuple(vel), (q / dt).reshape(ps)


def bicgstab(apply_A, apply_Minv, b, tol, maxiter):
    """Right-preconditioned BiCGstab (van der Vorst 1992), FP64 scalars.

    Returns (x, iterations, ||b - A x|| / ||b||)."""
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    rel = 1.0
    while it < maxiter:
        it += 1
        rho = float(np.dot(rhat, r))
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = apply_Minv(p)
        v = apply_A(phat)
        alpha = rho / float(np.dot(rhat, v))
        s = r - alpha * v
        shat = apply_Minv(s)
        t = apply_A(shat)
        omega = float(np.dot(t, s)) / float(np.dot(t, t))
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho_old = rho
        rel = float(np.linalg.norm(r)) / bnorm
        if rel <= tol:
            break
    return x, it, rel


def pcg(apply_A, apply_B, b, weights, tol, maxiter):
    """Preconditioned conjugate gradients (Hestenes & Stiefel 1952) for A x = b
    with A and the preconditioner B self-adjoint and positive definite in the
    inner product <x, y> = sum(weights * x * y), FP64 scalars.

    Returns (x, iterations, ||b - A x|| / ||b||) (Euclidean norms)."""
    w = np.asarray(weights, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    p = np.zeros_like(b)
    rho = 1.0
    it = 0
    rel = 1.0
    while it < maxiter:
        z = apply_B(r)
        rho_new = float(np.sum(w * r * z))
        p = z if it == 0 else z + (rho_new / rho) * p
        rho = rho_new
        v = apply_A(p)
        alpha = rho / float(np.sum(w * p * v))
        x = x + alpha * p
        r = r - alpha * v
        it += 1
        rel = float(np.linalg.norm(r)) / bnorm
        if rel <= tol:
            break
    return x, it, rel


def bicgstab_l(apply_A, apply_Minv, b, ell, tol, maxiter):
    """Right-preconditioned BiCGstab(ell) (Sleijpen & Fokkema 1993), the Krylov
    solver of the paper (ell = 2, Sec. 2), FP64 scalars.

    The iteration runs on y for (A M^{-1}) y = b (so its residuals are the true
    residuals of x = M^{-1} y, returned at the end).  One outer iteration makes
    ell BiCG steps (2 ell operator applications) followed by a minimal-residual
    step over the ell + 1 vectors r_0 .. r_ell (modified Gram-Schmidt).
    Returns (x, outer iterations, ||b - A x|| / ||b||)."""
    op = lambda v: apply_A(apply_Minv(v))
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    y = np.zeros_like(b)
    r = [b.copy()] + [np.zeros_like(b) for _ in range(ell)]
    u = [np.zeros_like(b) for _ in range(ell + 1)]
    rhat = b.copy()
    rho0, alpha, omega = 1.0, 0.0, 1.0
    it = 0
    rel = 1.0
    while it < maxiter:
        it += 1
        rho0 = -omega * rho0
        # BiCG part: ell steps, each raising the degree of the u / r sequences
        for j in range(ell):
            rho1 = float(np.dot(rhat, r[j]))
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                u[i] = r[i] - beta * u[i]
            u[j + 1] = op(u[j])
            alpha = rho0 / float(np.dot(rhat, u[j + 1]))
            for i in range(j + 1):
                r[i] = r[i] - alpha * u[i + 1]
            r[j + 1] = op(r[j])
            y = y + alpha * u[0]
        # minimal-residual part: orthogonalise r_1 .. r_ell (MGS), then the
        # coefficients of the polynomial in the original basis
        tau = np.zeros((ell + 1, ell + 1))
        sigma = np.zeros(ell + 1)
        gp = np.zeros(ell + 1)
        for j in range(1, ell + 1):
            for i in range(1, j):
                tau[i, j] = float(np.dot(r[j], r[i])) / sigma[i]
                r[j] = r[j] - tau[i, j] * r[i]
            sigma[j] = float(np.dot(r[j], r[j]))
            gp[j] = float(np.dot(r[0], r[j])) / sigma[j]
        g = np.zeros(ell + 1)
        g[ell] = gp[ell]
        omega = g[ell]
        for j in range(ell - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, ell + 1))
        gpp = np.zeros(ell + 1)
        for j in range(1, ell):
            gpp[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, ell))
        y = y + g[1] * r[0]
        r[0] = r[0] - gp[ell] * r[ell]
        u[0] = u[0] - g[ell] * u[ell]
        for j in range(1, ell):
            u[0] = u[0] - g[j] * u[j]
            y = y + gpp[j] * r[j]
            r[0] = r[0] - gp[j] * r[j]
        rel = float(np.linalg.norm(r[0])) / bnorm
        if rel <= tol:
            break
    x = apply_Minv(y)
    return x, it, float(np.linalg.norm(b - apply_A(x))) / bnorm


def stokes_semi_direct(faces, dt, Re, f, tol=1e-11, maxiter=200, method="tpt", precond="laplace",
                       krylov="bicgstab"):
    """Three-step semi-direct Stokes inverse (Sec. 2): direct Helmholtz inverses by
    the decomposition solvers, BiCGstab on C preconditioned by L_p^{-1}
    (precond="laplace", the paper's choice) or by L_p^{-1} - lam*I
    (precond="cahouet-chabard": Cahouet & Chabard 1988, the exact inverse of
    C = L_p (I - lam L_p)^{-1} when the discrete operators commute).

    krylov: "bicgstab", "bicgstab2" (the paper's choice, Sec. 2) or "cg"
    (conjugate gradients on -C q = -b in the volume-weighted inner product,
    preconditioned by minus the chosen preconditioner).
    Returns ((u, v, w), p, iterations, relative C-residual)."""
    lam = dt / Re
    D, G = div_grad_3d(faces)
    vs, ps = shapes(faces)
    cops = [component_ops(faces, c) for c in range(3)]
    pops = pressure_ops(faces)

    def Hinv(c, g):
        return dec.solve(np.reshape(g, vs[c]), cops[c], lam, 1.0, method).ravel()

    def Lp_inv(g):
        # L_p = D G is the zero-flux Laplacian; -L_p^{-1} is the Laplace solve
        out = -dec.solve(np.reshape(g, ps), pops, 1.0, 0.0, method).ravel()
        if precond == "cahouet-chabard":
            out = out - lam * np.ravel(g)
        return out

    def C(q):
        return sum(D[c] @ Hinv(c, G[c] @ q) for c in range(3))

    uhat = [Hinv(c, f[c]) for c in range(3)]
    b = sum(D[c] @ uhat[c] for c in range(3))
    vol = asm.volumes(pops)
    if krylov == "bicgstab2":
        q, it, rel = bicgstab_l(C, Lp_inv, b, 2, tol, maxiter)
    elif krylov == "cg":
        q, it, rel = pcg(lambda v: -C(v), lambda v: -Lp_inv(v), -b, vol, tol, maxiter)
    else:
        q, it, rel = bicgstab(C, Lp_inv, b, tol, maxiter)
    q = q - np.dot(vol, q) / vol.sum()
    vel = tuple((uhat[c] - Hinv(c, G[c] @ q)).reshape(vs[c]) for c in range(3))
    return vel, (q / dt).reshape(ps), it, rel
