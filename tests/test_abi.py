"""The C-ABI library builds, loads and exports every entry point declared in
include/fdi.h; host-side argument checks answer without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1107_2461_gb300 import build
    build.build()
    from paper_1107_2461_gb300 import fdi
    return fdi.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "fdi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdi_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for req in ["fdi_plan_create", "fdi_plan_destroy", "fdi_helmholtz_solve", "fdi_laplace_solve",
                "fdi_stokes_solve", "fdi_helmholtz_solve_batched", "fdi_last_result", "fdi_status_string"]:
        assert req in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1107_2461_gb300 import fdi
    assert set(_declared()) <= set(fdi.SIGNATURES)


def test_status_strings(lib):
    from paper_1107_2461_gb300 import fdi
    assert fdi.status_string(0) == "FDI_OK"
    assert fdi.status_string(4) == "FDI_ERR_NOT_CONVERGED"
    assert fdi.status_string(99) == "FDI_ERR_UNKNOWN"


def test_invalid_arguments_rejected_without_touching_the_gpu(lib):
    from paper_1107_2461_gb300 import fdi
    import numpy as np
    faces = [np.linspace(0, 1, 9)] * 3
    # n out of range
    with pytest.raises(fdi.FdiError) as e:
        fdi.plan_create(faces, (8, 8, 300))
    assert e.value.status == fdi.ERR_INVALID_ARG
    # non-ascending faces
    bad = [np.linspace(0, 1, 9), np.linspace(1, 0, 9), np.linspace(0, 1, 9)]
    with pytest.raises(fdi.FdiError) as e:
        fdi.plan_create(bad, (8, 8, 8))
    assert e.value.status == fdi.ERR_INVALID_ARG
    # Thomas axis out of range; a staggered plan with its Thomas axis not z
    for axis in (3, -3):
        with pytest.raises(fdi.FdiError) as e:
            fdi.plan_create(faces, (8, 8, 8), thomas_axis=axis)
        assert e.value.status == fdi.ERR_UNSUPPORTED
    with pytest.raises(fdi.FdiError) as e:
        fdi.plan_create(faces, (8, 8, 8), grid=fdi.GRID_MAC, thomas_axis=1)
    assert e.value.status == fdi.ERR_UNSUPPORTED
    # the two reserved precision modes are not built and are refused at creation
    for prec in (fdi.PREC_MIXED_TF32, fdi.PREC_MIXED_BF16):
        with pytest.raises(fdi.FdiError) as e:
            fdi.plan_create(faces, (8, 8, 8), prec=prec)
        assert e.value.status == fdi.ERR_UNSUPPORTED
    # null plan handles
    assert lib.fdi_helmholtz_solve(None, 1.0, None, None, None) == fdi.ERR_INVALID_ARG
    assert lib.fdi_plan_destroy(None) == fdi.ERR_INVALID_ARG
    assert lib.fdi_last_result(None, None, None, None) == fdi.ERR_INVALID_ARG
    assert lib.fdi_helmholtz_solve_batched(None, None, None, None, -1, None) == fdi.ERR_INVALID_ARG
    assert lib.fdi_field_solve_host(None, 0, 1.0, 1.0, None, None, 1, None, None) == fdi.ERR_INVALID_ARG
    assert lib.fdi_stokes_solve(None, 1.0, 1.0, None, None, None, None) == fdi.ERR_INVALID_ARG
    for setter in ("fdi_plan_set_krylov", "fdi_plan_set_stokes_preconditioner", "fdi_plan_set_graphs",
                   "fdi_plan_set_thomas_config", "fdi_plan_enable_timing"):
        assert getattr(lib, setter)(None, 0) == fdi.ERR_INVALID_ARG, setter
    assert lib.fdi_plan_set_tolerances(None, 1e-10, 2, 1e-10, 10) == fdi.ERR_INVALID_ARG
    assert lib.fdi_last_launch_count(None, None) == fdi.ERR_INVALID_ARG


def test_stokes_plan_bytes_estimate_scales_with_the_grid(lib):
    # host-only sizing used by the serving runtime's admission: grows with the
    # number of cells (about x8 from 128^3 to 256^3), mixed plans hold the extra
    # FP32 planes, and permuting the extents changes little
    from paper_1107_2461_gb300 import fdi
    est = fdi.stokes_plan_bytes_estimate
    for prec in (fdi.PREC_FP64, fdi.PREC_MIXED_F16):
        sizes = [est((n, n, n), prec) for n in (16, 32, 64, 128, 256)]
        assert all(b > a for a, b in zip(sizes, sizes[1:]))
        assert 7.0 < sizes[-1] / sizes[-2] < 8.5
        a, b = est((64, 128, 256), prec), est((256, 128, 64), prec)
        assert abs(a - b) <= 0.05 * max(a, b)
    assert est((128, 128, 128), fdi.PREC_MIXED_F16) > est((128, 128, 128), fdi.PREC_FP64)
    # 256^3 Stokes plans fit many times over in a GB300's 288 GB
    assert est((256, 256, 256), fdi.PREC_MIXED_F16) < 16e9


def test_later_entry_points_reject_null_handles_and_bad_sizes(lib):
    # every check below answers on the host, before any CUDA call
    import numpy as np
    from paper_1107_2461_gb300 import fdi
    bad = fdi.ERR_INVALID_ARG
    assert lib.fdi_field_solve(None, 0, 1.0, 1.0, None, None, None) == bad
    assert lib.fdi_laplace_solve(None, None, None, None) == bad
    assert lib.fdi_apply_transform(None, 0, 0, 0, None, None, 1, None) == bad
    assert lib.fdi_plan_eigen(None, 0, 0, None, None, None, None) == bad
    assert lib.fdi_plan_autotune(None, 1.0, None, None, 1, None, None) == bad
    cnt = C.c_int(0)
    assert lib.fdi_plan_kernel_times(None, 0, None, None, None, C.byref(cnt)) == bad
    assert lib.fdi_plan_reset_kernel_times(None) == bad
    assert lib.fdi_plan_set_resident(None, 1) == bad
    assert lib.fdi_plan_set_wait_limit(None, 0) == bad
    # serving runtime: null handles, and a server that could hold nothing
    h = C.c_void_p()
    assert lib.fdi_server_create(0, 4, C.byref(h)) == bad
    assert lib.fdi_server_create(1 << 30, 0, C.byref(h)) == bad
    assert lib.fdi_server_create(1 << 30, 65, C.byref(h)) == bad
    assert lib.fdi_server_create(1 << 30, 4, None) == bad
    t = C.c_longlong(0)
    assert lib.fdi_server_submit(None, None, C.byref(t)) == bad
    assert lib.fdi_server_poll(None, 1, 0, None) == bad
    assert lib.fdi_server_drain(None) == bad
    assert lib.fdi_server_stats(None, None) == bad
    assert lib.fdi_server_destroy(None) == bad
    # cylindrical plans: extents, radial faces below zero, descending faces
    dp = C.POINTER(C.c_double)
    r = np.linspace(0.0, 1.0, 9)
    z = np.linspace(0.0, 1.0, 9)
    out = C.c_void_p()

    def cyl(rf, nr, nth, zf, nz):
        return lib.fdi_plan_create_cyl(rf.ctypes.data_as(dp), nr, nth, zf.ctypes.data_as(dp), nz,
                                       0, 0, 0, 0, fdi.PREC_FP64, 0, C.byref(out))
    assert cyl(r, 8, 2, z, 8) == bad
    assert cyl(r, 8, 300, z, 8) == bad
    assert cyl(r, 1, 8, z, 8) == bad
    assert cyl(r - 0.5, 8, 8, z, 8) == bad
    assert cyl(r[::-1].copy(), 8, 8, z, 8) == bad
    assert cyl(r, 8, 8, z[::-1].copy(), 8) == bad
    assert not out.value
    assert lib.fdi_plan_create_cyl(None, 8, 8, None, 8, 0, 0, 0, 0, fdi.PREC_FP64, 0, C.byref(out)) == bad


def test_binding_refuses_arrays_it_cannot_pass():
    # argument marshalling only, on the host: CPU, strided or non-FP64 tensors
    # never reach the C ABI as device pointers, nor device or mistyped arrays
    # as host buffers
    torch = pytest.importorskip("torch")
    import numpy as np
    from paper_1107_2461_gb300 import fdi
    with pytest.raises(ValueError):
        fdi._ptr(torch.zeros(8, dtype=torch.float64))  # not on the device
    with pytest.raises(TypeError):
        fdi._ptr(np.zeros(8))
    assert fdi._ptr(None) is None and fdi._ptr(1234) == 1234
    with pytest.raises(ValueError):
        fdi._host_ptr(np.zeros(8, dtype=np.float32), 8)
    with pytest.raises(ValueError):
        fdi._host_ptr(np.zeros((4, 4))[:, ::2], 8)
    with pytest.raises(ValueError):
        fdi._host_ptr(np.zeros(9), 8)
    with pytest.raises(ValueError):
        fdi._host_ptr(torch.zeros(8, dtype=torch.float32), 8)
    a = np.zeros(8)
    assert fdi._host_ptr(a, 8) == a.ctypes.data
    t = torch.zeros(8, dtype=torch.float64)
    assert fdi._host_ptr(t, 8) == t.data_ptr()
