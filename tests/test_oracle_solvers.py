"""Pins of the oracle's 3D Helmholtz / Laplace solvers (Sec. 3, Eq. 25-29):
independent loop assembly, brute-force dense inverses, manufactured eigenmodes,
cross-method agreement (the paper's TPF/TPT/iterative agreement, Sec. 5) and the
Neumann null space (Eq. 28)."""
import itertools

import numpy as np
import pytest

from oracle import assembled as asm
from oracle import decomposition as dec
from oracle import operators1d as o1
from workloads import box_faces, rhs_uniform, tanh_faces

D, N = o1.DIRICHLET, o1.NEUMANN


def _ops(faces, lo, hi):
    return asm.cell_ops(faces, lo, hi)


@pytest.mark.parametrize("lo,hi", [((D, D, D), (D, D, D)), ((N, N, N), (N, N, N)),
                                   ((D, N, D), (N, D, N)), ((N, D, N), (N, D, D))])
@pytest.mark.parametrize("lam,sigma", [(1e-3, 1.0), (1.0, 1.0), (1e3, 1.0), (1.0, 0.0)])
def test_kron_assembly_matches_loop_assembly(lo, hi, lam, sigma):
    faces = [tanh_faces(3, 1.2), tanh_faces(4, 2.0), tanh_faces(5, 1.5)]
    A_k = asm.helmholtz(_ops(faces, lo, hi), lam, sigma).toarray()
    A_l = asm.stencil_matrix_by_loops(faces, lo, hi, lam, sigma)
    assert np.abs(A_k - A_l).max() <= 1e-13 * np.abs(A_l).max()


def _dense_reference(faces, lo, hi, lam, sigma, f):
    A = asm.stencil_matrix_by_loops(faces, lo, hi, lam, sigma)
    ops = _ops(faces, lo, hi)
    if asm.is_singular(ops, sigma):
        vol = asm.volumes(ops)
        n = A.shape[0]
        B = np.zeros((n + 1, n + 1))
        B[:n, :n] = A
        B[:n, n] = 1.0
        B[n, :n] = vol
        fp = f.ravel() - np.dot(vol, f.ravel()) / vol.sum()
        return np.linalg.solve(B, np.concatenate([fp, [0.0]]))[:n].reshape(f.shape)
    return np.linalg.solve(A, f.ravel()).reshape(f.shape)


BCS = [((D, D, D), (D, D, D)), ((N, N, N), (N, N, N)), ((D, N, N), (N, N, D)), ((N, D, N), (N, N, N))]


@pytest.mark.parametrize("lo,hi", BCS)
@pytest.mark.parametrize("lam,sigma", [(1e-5, 1.0), (1.0, 1.0), (1e3, 1.0), (1.0, 0.0)])
@pytest.mark.parametrize("method", ["tpf", "tpt0", "tpt1", "tpt2", "direct"])
def test_brute_force_dense_inverse(lo, hi, lam, sigma, method):
    faces = [tanh_faces(4, 1.5), tanh_faces(5, 2.0), tanh_faces(3, 1.0)]
    ops = _ops(faces, lo, hi)
    if sigma == 0.0 and not asm.is_singular(ops, 0.0) and all(b == N for b in lo + hi):
        pytest.skip("not applicable")
    f = rhs_uniform((3, 5, 4), seed=7)
    ref = _dense_reference(faces, lo, hi, lam, sigma, f)
    if method == "direct":
        got = asm.solve(ops, f, lam, sigma)
    elif method == "tpf":
        got = dec.tpf_solve(f, ops, lam, sigma)
    else:
        got = dec.tpt_solve(f, ops, lam, sigma, thomas_dir=int(method[-1]))
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_manufactured_eigenmode_product():
    # A (e_x (x) e_y (x) e_z) = (sigma - lam (Lx + Ly + Lz)) (e_x (x) e_y (x) e_z), with A
    # assembled by the loop route and the 1D eigenpairs of Eq. 24
    faces = [tanh_faces(6, 1.5), tanh_faces(5, 1.5), tanh_faces(7, 2.0)]
    lo, hi = (D, N, D), (D, D, N)
    lam = 0.37
    A = asm.stencil_matrix_by_loops(faces, lo, hi, lam, 1.0)
    eig = [dec.generalized_eig(*o1.cell_operator(faces[d], lo[d], hi[d])) for d in range(3)]
    for (a, b, c) in [(0, 0, 0), (5, 4, 6), (2, 3, 1)]:
        u = np.einsum("k,j,i->kji", eig[2][1][:, c], eig[1][1][:, b], eig[0][1][:, a]).ravel()
        mu = 1.0 - lam * (eig[0][0][a] + eig[1][0][b] + eig[2][0][c])
        assert np.abs(A @ u - mu * u).max() <= 1e-11 * abs(mu) * np.abs(u).max()
        x = dec.tpt_solve(u.reshape(7, 5, 6), [o1.cell_operator(faces[d], lo[d], hi[d]) for d in range(3)], lam)
        assert np.abs(x.ravel() - u / mu).max() <= 1e-12 * np.abs(u / mu).max()


def test_config1_cross_method_agreement():
    # 16^3, tanh factor 1.5, Dirichlet walls, lambda = dt/Re = 1e3/1e3; the paper reports
    # TPF, TPT and the iterative solver agreeing to at least ten digits (Sec. 5)
    faces = box_faces((16, 16, 16), 1.5)
    ops = _ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform((16, 16, 16), seed=0)
    lam = 1e3 / 1000.0
    ref = asm.solve(ops, f, lam)
    assert asm.relative_residual(ops, ref, f, lam) < 1e-13
    for x in (dec.tpf_solve(f, ops, lam), dec.tpt_solve(f, ops, lam, thomas_dir=2),
              dec.tpt_solve(f, ops, lam, thomas_dir=0)):
        assert np.abs(x - ref).max() <= 1e-11 * np.abs(ref).max()
        assert asm.relative_residual(ops, x, f, lam) < 1e-11


@pytest.mark.parametrize("method", ["tpf", "tpt"])
def test_neumann_null_space(method):
    # pure zero-flux Laplacian: A 1 = 0, V^T A = 0; the solve returns the zero-mean
    # solution and ignores the mean of f (Eq. 28 reading)
    faces = [tanh_faces(6, 1.5), tanh_faces(7, 2.0), tanh_faces(5, 1.2)]
    ops = _ops(faces, (N, N, N), (N, N, N))
    A = asm.stencil_matrix_by_loops(faces, (N, N, N), (N, N, N), 1.0, 0.0)
    vol = asm.volumes(ops)
    assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-10 * np.abs(A).max()
    assert np.abs(vol @ A).max() < 1e-12 * np.abs(A).max()
    f = rhs_uniform((5, 7, 6), seed=3)
    u1 = dec.solve(f, ops, 1.0, 0.0, method)
    u2 = dec.solve(f + 5.0, ops, 1.0, 0.0, method)
    assert abs(np.dot(vol, u1.ravel())) < 1e-13 * np.abs(u1).max()
    assert np.abs(u1 - u2).max() < 1e-11 * np.abs(u1).max()
    fp = asm.project_zero_mean(f, vol)
    assert np.abs(A @ u1.ravel() - fp).max() < 1e-10 * np.abs(fp).max()


def test_3d_continuum_convergence():
    # -Delta u = f with u = sin(pi x) sin(2 pi y) sin(pi z): second-order convergence
    errs = []
    for n in (16, 32, 64):
        faces = box_faces((n, n, n), 1.5)
        ops = _ops(faces, (D, D, D), (D, D, D))
        c = [0.5 * (fc[:-1] + fc[1:]) for fc in faces]
        Z, Y, X = np.meshgrid(c[2], c[1], c[0], indexing="ij")
        u = np.sin(np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(np.pi * Z)
        f = 6 * np.pi**2 * u
        got = dec.tpt_solve(f, ops, 1.0, 0.0)
        errs.append(np.abs(got - u).max())
    errs = np.array(errs)
    assert np.all(errs[:-1] / errs[1:] > 3.5), errs


def test_transposed_inverse_is_caught():
    # a plausible mistake (E^{-1} transposed) fails the brute-force pin
    faces = [tanh_faces(4, 1.5), tanh_faces(5, 2.0), tanh_faces(3, 1.0)]
    ops = _ops(faces, (D, D, D), (D, D, D))
    f = rhs_uniform((3, 5, 4), seed=7)
    ref = _dense_reference(faces, (D, D, D), (D, D, D), 1.0, 1.0, f)
    orig = dec.generalized_eig

    def wrong(m, K):
        lam, E, Einv = orig(m, K)
        return lam, E, E.T.copy()

    dec.generalized_eig = wrong
    try:
        bad = dec.tpf_solve(f, ops, 1.0, 1.0)
    finally:
        dec.generalized_eig = orig
    assert np.abs(bad - ref).max() > 1e-6 * np.abs(ref).max()
