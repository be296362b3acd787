"""Time-stepper-based Newton solver for steady states (Sec. 2, Eq. 10-17), the
application the Stokes inverse is built for.

A steady state of the discretised equations F(U) = L U + N(U) + f = 0 (Eq. 10)
is a fixed point of the semi-implicit time step (Eq. 13),

    (u^{k+1} - u^k) / dt = (1/Re) Delta u^{k+1} - G p^{k+1} + N(u^k) + f,   D u^{k+1} = 0,

which is one Stokes inverse:  u^{k+1} = T(u^k) = S^{-1}(u^k + dt (N(u^k) + f)).
Newton's method (Eq. 11-12) is applied to the preconditioned system of Eq. 17,
R(u) = T(u) - u = 0: the right-hand side is the difference of two consecutive
time steps (Eq. 14), and the Jacobian action on a vector v is the difference
of two consecutive linearised time steps (Eq. 15-16),

    R'(u) v = S^{-1}(v + dt N_U(u) v) - v,

so the Newton correction is found by a Krylov method that needs only Stokes
inverses (BiCGstab here; the paper uses BiCGstab(2)).  Large dt makes
S^{-1} a good preconditioner of the steady Jacobian, which is why the Stokes
inverse must work at large time steps.

The Stokes inverse is a callable `stokes(g) -> (u, p)` solving
(I - (dt/Re) Delta) u + dt G p = g, D u = 0 for a velocity forcing g (three
face fields); `library_stokes_inverse` wraps fdi_stokes_solve.  Velocity
states are lists of three arrays (NumPy or CUDA tensors); the nonlinear term
and its Jacobian action are callables on such states.
"""
from __future__ import annotations

from dataclasses import dataclass, field


def _axpy(a, x, y):
    """a * x + y for states (lists of arrays)."""
    return [a * xi + yi for xi, yi in zip(x, y)]


def _scale(a, x):
    return [a * xi for xi in x]


def _dot(x, y):
    return float(sum(float((xi * yi).sum()) for xi, yi in zip(x, y)))


def _norm(x):
    return _dot(x, x) ** 0.5


@dataclass
class NewtonResult:
    u: list
    p: object
    iterations: int
    residuals: list = field(default_factory=list)  # ||R(u_n)|| per Newton iteration
    krylov_iterations: list = field(default_factory=list)
    stokes_solves: int = 0
    converged: bool = False


class TimeStepperNewton:
    """Newton iteration on R(u) = T(u) - u = 0 with matrix-free BiCGstab for the
    correction (Eq. 17).

    stokes     callable g -> (u, p): the Stokes inverse at the chosen dt, Re
    dt         the time step the Stokes inverse was built for
    N, N_U     callables: N(u) -> state, N_U(u, v) -> state (Jacobian action)
    f          forcing state (may be None)
    """

    def __init__(self, stokes, dt, N, N_U, f=None):
        self.stokes = stokes
        self.dt = float(dt)
        self.N = N
        self.N_U = N_U
        self.f = f
        self.solves = 0

    def step(self, u):
        """One time step T(u) (Eq. 13-14): returns (u_next, p_next)."""
        g = _axpy(self.dt, self.N(u), u)
        if self.f is not None:
            g = _axpy(self.dt, self.f, g)
        self.solves += 1
        return self.stokes(g)

    def jac(self, u, v):
        """R'(u) v: the linearised time step minus v (Eq. 15-16)."""
        g = _axpy(self.dt, self.N_U(u, v), v)
        self.solves += 1
        w, _ = self.stokes(g)
        return _axpy(-1.0, v, w)

    def _bicgstab(self, u, b, tol, maxiter):
        """BiCGstab (van der Vorst) for R'(u) x = b, x0 = 0; relative tolerance."""
        x = _scale(0.0, b)
        r = [bi + 0.0 for bi in b]
        bn = _norm(b)
        if bn == 0.0:
            return x, 0
        rhat = [ri + 0.0 for ri in r]
        rho_old = alpha = omega = 1.0
        v = _scale(0.0, b)
        p = _scale(0.0, b)
        for it in range(1, maxiter + 1):
            rho = _dot(rhat, r)
            beta = (rho / rho_old) * (alpha / omega)
            p = _axpy(beta, _axpy(-omega, v, p), r)
            v = self.jac(u, p)
            alpha = rho / _dot(rhat, v)
            s = _axpy(-alpha, v, r)
            t = self.jac(u, s)
            tt = _dot(t, t)
            omega = _dot(t, s) / tt if tt > 0.0 else 0.0
            x = _axpy(alpha, p, _axpy(omega, s, x))
            r = _axpy(-omega, t, s)
            rho_old = rho
            if _norm(r) <= tol * bn or omega == 0.0:
                return x, it
        return x, maxiter

    def solve(self, u0, tol=1e-10, max_newton=20, krylov_tol=1e-3, krylov_maxiter=100):
        """Newton iterations from u0 until ||T(u) - u|| <= tol * max(1, ||T(u)||)
        (Euclidean norms over the three face fields).  Each Newton step solves
        R'(u) du = -R(u) to the relative `krylov_tol` (inexact Newton: a loose
        tolerance trades Newton steps for Krylov iterations)."""
        self.solves = 0
        u = [x + 0.0 for x in u0]
        res = NewtonResult(u=u, p=None, iterations=0)
        for n in range(max_newton + 1):
            tu, tp = self.step(u)
            R = _axpy(-1.0, u, tu)
            rn = _norm(R)
            res.residuals.append(rn)
            res.u, res.p, res.iterations = u, tp, n
            if rn <= tol * max(1.0, _norm(tu)):
                # the converged state: one more time step changes nothing
                res.u = tu
                res.converged = True
                break
            if n == max_newton:
                break
            du, kit = self._bicgstab(u, _scale(-1.0, R), krylov_tol, krylov_maxiter)
            res.krylov_iterations.append(kit)
            u = _axpy(1.0, du, u)
        res.stokes_solves = self.solves
        return res


def library_stokes_inverse(plan, dt, Re, stream=None):
    """Stokes inverse g -> (u, p) through fdi_stokes_solve on a MAC plan; states
    are lists of three contiguous FP64 CUDA tensors of the face-field shapes."""
    import torch

    from . import fdi

    def stokes(g):
        g = [x.contiguous() for x in g]
        u = [torch.empty_like(x) for x in g]
        p = torch.empty(plan.field_shape(fdi.FIELD_CELL), dtype=torch.float64, device=g[0].device)
        if stream is not None:  # the solve on `stream` follows the work that made g, and precedes its readers
            stream.wait_stream(torch.cuda.current_stream())
        fdi.stokes_solve(plan, dt, Re, g, u, p, stream)
        if stream is not None:
            torch.cuda.current_stream().wait_stream(stream)
        return u, p

    return stokes
