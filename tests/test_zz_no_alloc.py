"""The allocation-free eigen entry point (fdi_eigen_noalloc), for callers that
may not allocate device memory, reproduces the plan-creation eigen
decomposition (fdi_plan_eigen), called twice in a row through the C ABI.

Kept in a file that sorts last so that a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest

from workloads import tanh_faces

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fdi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2461_gb300 import build
    build.build()
    import paper_1107_2461_gb300 as pkg
    return pkg


def _noalloc(fdi, faces, face_kind, bc_lo, bc_hi, with_flag=True):
    import torch
    n = len(faces) - 1
    m = n - 1 if face_kind else n
    lam = torch.empty(m, dtype=torch.float64, device="cuda")
    E = torch.empty(m * m, dtype=torch.float64, device="cuda")
    Einv = torch.empty(m * m, dtype=torch.float64, device="cuda")
    f = np.ascontiguousarray(faces, dtype=np.float64)
    conv = C.c_int(-1)
    lib = fdi.fdi.load()
    stream = torch.cuda.current_stream()
    st = lib.fdi_eigen_noalloc(f.ctypes.data_as(C.POINTER(C.c_double)), n, face_kind, bc_lo, bc_hi,
                               lam.data_ptr(), E.data_ptr(), Einv.data_ptr(), C.byref(conv) if with_flag else None,
                               stream.cuda_stream)
    assert st == 0, fdi.status_string(st)
    if with_flag:
        assert conv.value == 1
    else:
        # without the flag the call returns at once; the caller synchronises
        stream.synchronize()
    return lam.cpu().numpy(), E.cpu().numpy().reshape(m, m), Einv.cpu().numpy().reshape(m, m)


def _compare(a, b):
    lam_a, E_a, Ei_a = a
    lam_b, E_b, Ei_b = b
    scale = np.abs(lam_b).max()
    # the same kernel on the same operator: agreement to the eigen tests' tolerance
    assert np.abs(lam_a - lam_b).max() <= 1e-13 * scale
    assert np.abs(E_a - E_b).max() <= 1e-12 * np.abs(E_b).max()
    assert np.abs(Ei_a - Ei_b).max() <= 1e-12 * np.abs(Ei_b).max()


def test_noalloc_eigen_matches_plan_twice(fdi):
    # call 1: zero-flux cell operator (exact null pair), n = 64
    fx = tanh_faces(64, 2.0)
    faces = [fx, tanh_faces(6, 1.0), tanh_faces(6, 1.0)]
    plan = fdi.plan_create(faces, (64, 6, 6), (1, 0, 0), (1, 0, 0))
    ref1 = plan.eigen(fdi.FIELD_CELL, 0)
    plan.destroy()
    got1 = _noalloc(fdi, fx, 0, 1, 1)
    _compare(got1, ref1)
    # call 2, on the same scratch array: staggered face operator, n = 200
    fx = tanh_faces(200, 1.5)
    faces = [fx, tanh_faces(5, 1.0), tanh_faces(5, 1.0)]
    plan = fdi.plan_create(faces, (200, 5, 5), grid=fdi.GRID_MAC)
    ref2 = plan.eigen(fdi.FIELD_U, 0)
    plan.destroy()
    got2 = _noalloc(fdi, fx, 1, 0, 0)
    _compare(got2, ref2)


def test_noalloc_rejects_sizes_beyond_its_scratch(fdi):
    lib = fdi.fdi.load()
    f = np.linspace(0.0, 1.0, 258)
    st = lib.fdi_eigen_noalloc(f.ctypes.data_as(C.POINTER(C.c_double)), 257, 0, 0, 0, 1, 1, 1, None, None)
    assert st == fdi.fdi.ERR_INVALID_ARG


@pytest.mark.parametrize("bc,with_flag", [((0, 0), True), ((0, 1), False), ((1, 0), True)])
def test_noalloc_eigen_wall_kinds(fdi, bc, with_flag):
    # Dirichlet walls on both sides, and mixed walls (one side zero-flux), of a
    # cell operator: the wall terms of the operator assembled by the call; the
    # second case passes no convergence flag and synchronises afterwards
    n = 97
    fx = tanh_faces(n, 1.7)
    faces = [fx, tanh_faces(4, 1.0), tanh_faces(4, 1.0)]
    plan = fdi.plan_create(faces, (n, 4, 4), (bc[0], 0, 0), (bc[1], 0, 0))
    ref = plan.eigen(fdi.FIELD_CELL, 0)
    plan.destroy()
    for _ in range(2):
        _compare(_noalloc(fdi, fx, 0, bc[0], bc[1], with_flag), ref)


def test_noalloc_rejects_walls_of_a_face_operator(fdi):
    # the staggered velocity operator has no-slip walls only
    lib = fdi.fdi.load()
    f = np.linspace(0.0, 1.0, 11)
    st = lib.fdi_eigen_noalloc(f.ctypes.data_as(C.POINTER(C.c_double)), 10, 1, 1, 0, 1, 1, 1, None, None)
    assert st == fdi.fdi.ERR_INVALID_ARG
