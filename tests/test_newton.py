"""The time-stepper-based Newton solver (Sec. 2, Eq. 10-17) as a client of the
Stokes inverse, run on CPU with the oracle's direct Stokes solve standing in
for the library call (the host logic under test is the same)."""
import numpy as np
import pytest

from oracle import stokes as st
from paper_1107_2461_gb300.newton import TimeStepperNewton
from workloads import rhs_gaussian, tanh_faces


def _setup(dt, Re):
    faces = [tanh_faces(6, 1.5), tanh_faces(5, 1.5), tanh_faces(7, 2.0)]
    vs, ps = st.shapes(faces)

    def stokes(g):
        vel, p = st.stokes_direct(faces, dt, Re, [np.asarray(x) for x in g])
        return [np.asarray(v) for v in vel], p

    f = [rhs_gaussian(vs[c], 40 + c) for c in range(3)]
    return faces, vs, stokes, f


def test_linear_term_converges_in_one_newton_step():
    # N(u) = -c u: the steady state solves (c - Delta/Re) u + G p = f, which is
    # the Stokes system with dt' = 1/c and forcing f / c
    dt, Re, c = 10.0, 100.0, 2.0
    faces, vs, stokes, f = _setup(dt, Re)
    solver = TimeStepperNewton(stokes, dt, N=lambda u: [-c * x for x in u], N_U=lambda u, v: [-c * x for x in v], f=f)
    res = solver.solve([np.zeros(s) for s in vs], tol=1e-11, krylov_tol=1e-13, krylov_maxiter=200)
    assert res.converged and res.iterations == 1, res.residuals
    ref, pref = st.stokes_direct(faces, 1.0 / c, Re, [x / c for x in f])
    for c_ in range(3):
        assert np.abs(res.u[c_] - ref[c_]).max() <= 1e-9 * np.abs(ref[c_]).max()


def test_quadratic_term_converges_quadratically_to_a_steady_state():
    # N(u) = -gamma u * u (component-wise): a smooth nonlinearity whose Jacobian
    # action is -2 gamma u * v; exact Newton corrections give quadratic
    # convergence, and the limit is a fixed point of the time step, i.e. a
    # steady state of Eq. 10
    dt, Re, gamma = 5.0, 50.0, 0.3
    faces, vs, stokes, f = _setup(dt, Re)
    N = lambda u: [-gamma * x * x for x in u]  # noqa: E731
    N_U = lambda u, v: [-2.0 * gamma * x * y for x, y in zip(u, v)]  # noqa: E731
    solver = TimeStepperNewton(stokes, dt, N=N, N_U=N_U, f=f)
    res = solver.solve([np.zeros(s) for s in vs], tol=1e-12, krylov_tol=1e-13, krylov_maxiter=300)
    r = np.array(res.residuals)
    assert res.converged and res.iterations <= 8, r
    # quadratic: r_{n+1} <= C r_n^2 while above the rounding floor
    above = r[1:] > 1e-12 * r[0]
    assert np.sum(above) >= 3 and np.all((r[1:] <= 0.1 * r[:-1] ** 2)[above]), r
    # the limit satisfies the time step exactly: (I - dt/Re Delta) u + dt G p = u + dt (N(u) + f), D u = 0
    g = [u + dt * (n + fc) for u, n, fc in zip(res.u, N(res.u), f)]
    mom, div = st.saddle_residual(faces, dt, Re, g, res.u, res.p)
    assert mom <= 1e-10 and div <= 1e-10, (mom, div)


def test_inexact_newton_needs_more_steps_but_the_same_state():
    dt, Re, gamma = 5.0, 50.0, 0.3
    faces, vs, stokes, f = _setup(dt, Re)
    N = lambda u: [-gamma * x * x for x in u]  # noqa: E731
    N_U = lambda u, v: [-2.0 * gamma * x * y for x, y in zip(u, v)]  # noqa: E731
    exact = TimeStepperNewton(stokes, dt, N, N_U, f).solve([np.zeros(s) for s in vs], tol=1e-11, krylov_tol=1e-13,
                                                            krylov_maxiter=300)
    loose = TimeStepperNewton(stokes, dt, N, N_U, f).solve([np.zeros(s) for s in vs], tol=1e-11, krylov_tol=1e-2)
    assert loose.converged and loose.iterations >= exact.iterations
    for c in range(3):
        assert np.abs(loose.u[c] - exact.u[c]).max() <= 1e-9 * np.abs(exact.u[c]).max()
    assert loose.stokes_solves > 0 and sum(loose.krylov_iterations) > 0
