"""Thin ctypes binding over libfdi.so (argument marshalling only).

Every numerical step runs in the CUDA kernels behind the C ABI declared in
include/fdi.h; this module converts Python arguments (torch CUDA tensors or raw
device pointers, host face arrays) into the C types and turns a non-OK status
into an exception.  There is no fallback: if libfdi.so is missing the import
fails with an explanation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfdi.so")

OK = 0
ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_SINGULAR, ERR_UNSUPPORTED = range(1, 8)
BC_DIRICHLET, BC_NEUMANN = 0, 1
GRID_CELL, GRID_MAC = 0, 1
PREC_FP64, PREC_MIXED_TF32, PREC_MIXED_BF16, PREC_MIXED_F16 = 0, 1, 2, 3
FIELD_CELL, FIELD_U, FIELD_V, FIELD_W = 0, 1, 2, 3

class StokesRequest(C.Structure):
    """fdi_stokes_request (host arrays in the MAC shapes)."""
    _fields_ = [("n", C.c_int * 3), ("beta", C.c_double), ("dt", C.c_double), ("Re", C.c_double),
                ("prec", C.c_int), ("f", C.c_void_p * 3), ("u", C.c_void_p * 3), ("p", C.c_void_p)]


class StokesResult(C.Structure):
    """fdi_stokes_result."""
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("iters", C.c_int), ("rel_residual", C.c_double),
                ("queue_ms", C.c_double), ("latency_ms", C.c_double)]


class ServerReport(C.Structure):
    """fdi_server_report."""
    _fields_ = [("completed", C.c_longlong), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("throughput_rps", C.c_double), ("peak_bytes", C.c_size_t), ("bytes_in_use", C.c_size_t),
                ("plans_created", C.c_longlong), ("plans_evicted", C.c_longlong), ("plans_cached", C.c_longlong)]


# every function declared in include/fdi.h: name -> (restype, argtypes)
_vp = C.c_void_p
_i = C.c_int
_d = C.c_double
SIGNATURES = {
    "fdi_plan_create": (_i, [C.POINTER(C.POINTER(_d)), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), _i, _i, _i,
                             C.POINTER(_vp)]),
    "fdi_plan_destroy": (_i, [_vp]),
    "fdi_plan_set_tolerances": (_i, [_vp, _d, _i, _d, _i]),
    "fdi_helmholtz_solve": (_i, [_vp, _d, _vp, _vp, _vp]),
    "fdi_laplace_solve": (_i, [_vp, _vp, _vp, _vp]),
    "fdi_field_solve": (_i, [_vp, _i, _d, _d, _vp, _vp, _vp]),
    "fdi_stokes_solve": (_i, [_vp, _d, _d, C.POINTER(_vp), C.POINTER(_vp), _vp, _vp]),
    "fdi_helmholtz_solve_batched": (_i, [C.POINTER(_vp), C.POINTER(_d), C.POINTER(_vp), C.POINTER(_vp), _i, _vp]),
    "fdi_field_solve_host": (_i, [_vp, _i, _d, _d, C.POINTER(_vp), C.POINTER(_vp), _i, C.POINTER(_d), _vp]),
    "fdi_last_result": (_i, [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_d)]),
    "fdi_plan_eigen": (_i, [_vp, _i, _i, C.POINTER(_d), C.POINTER(_d), C.POINTER(_d), C.POINTER(_i)]),
    "fdi_last_launch_count": (_i, [_vp, C.POINTER(C.c_longlong)]),
    "fdi_apply_transform": (_i, [_vp, _i, _i, _i, _vp, _vp, C.c_longlong, _vp]),
    "fdi_plan_set_stokes_preconditioner": (_i, [_vp, _i]),
    "fdi_plan_set_krylov": (_i, [_vp, _i]),
    "fdi_eigen_noalloc": (_i, [C.POINTER(_d), _i, _i, _i, _i, _vp, _vp, _vp, C.POINTER(_i), _vp]),
    "fdi_plan_set_graphs": (_i, [_vp, _i]),
    "fdi_plan_create_cyl": (_i, [C.POINTER(_d), _i, _i, C.POINTER(_d), _i, _i, _i, _i, _i, _i, _i, C.POINTER(_vp)]),
    "fdi_plan_set_thomas_config": (_i, [_vp, _i]),
    "fdi_plan_set_wait_limit": (_i, [_vp, C.c_longlong]),
    "fdi_plan_set_resident": (_i, [_vp, C.c_int]),
    "fdi_plan_autotune": (_i, [_vp, _d, _vp, _vp, _i, C.POINTER(_i), _vp]),
    "fdi_plan_enable_timing": (_i, [_vp, _i]),
    "fdi_plan_kernel_times": (_i, [_vp, _i, C.POINTER(C.c_char_p), C.POINTER(_d), C.POINTER(C.c_longlong),
                                   C.POINTER(_i)]),
    "fdi_plan_reset_kernel_times": (_i, [_vp]),
    "fdi_stokes_plan_bytes_estimate": (C.c_size_t, [C.POINTER(_i), _i]),
    "fdi_server_create": (_i, [C.c_size_t, _i, C.POINTER(_vp)]),
    "fdi_server_submit": (_i, [_vp, C.POINTER(StokesRequest), C.POINTER(C.c_longlong)]),
    "fdi_server_poll": (_i, [_vp, C.c_longlong, _i, C.POINTER(StokesResult)]),
    "fdi_server_drain": (_i, [_vp]),
    "fdi_server_stats": (_i, [_vp, C.POINTER(ServerReport)]),
    "fdi_server_destroy": (_i, [_vp]),
    "fdi_last_error_message": (C.c_char_p, []),
    "fdi_status_string": (C.c_char_p, [_i]),
}

_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libfdi.so and declare the C signatures; raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(
            f"libfdi.so not found at {_LIB_PATH}: build it with "
            "`python -m paper_1107_2461_gb300.build` (nvcc, sm_103a); there is no CPU fallback")
    lib = C.CDLL(_LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FdiError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        self.status = status
        msg = lib.fdi_last_error_message().decode(errors="replace")
        super().__init__(f"{where}: {lib.fdi_status_string(status).decode()} {msg}")


def _check(status, where):
    if status != OK:
        raise FdiError(status, where)


def _ptr(x):
    """Device pointer of a torch tensor (must be contiguous FP64 on CUDA) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("tensor must live on the CUDA device")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(x.dtype) != "torch.float64":
            raise ValueError("tensor must be float64")
        return x.data_ptr()
    raise TypeError(f"expected a CUDA tensor or a device pointer, got {type(x)}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """Owning handle of an fdi_plan (fdi_plan_create / fdi_plan_destroy)."""

    def __init__(self, faces, n=None, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), grid=GRID_CELL, prec=PREC_FP64,
                 thomas_axis=2):
        lib = load()
        self._faces = [np.ascontiguousarray(np.asarray(f, dtype=np.float64)) for f in faces]
        if n is None:
            n = [f.size - 1 for f in self._faces]
        self.n = tuple(int(v) for v in n)
        self.grid, self.prec, self.thomas_axis = grid, prec, thomas_axis
        fptrs = (C.POINTER(C.c_double) * 3)(*[f.ctypes.data_as(C.POINTER(C.c_double)) for f in self._faces])
        nn = (C.c_int * 3)(*self.n)
        lo = (C.c_int * 3)(*[int(b) for b in bc_lo])
        hi = (C.c_int * 3)(*[int(b) for b in bc_hi])
        h = C.c_void_p()
        _check(lib.fdi_plan_create(fptrs, nn, lo, hi, grid, prec, thomas_axis, C.byref(h)), "fdi_plan_create")
        self.handle = h.value

    def destroy(self):
        if self.handle:
            _check(load().fdi_plan_destroy(self.handle), "fdi_plan_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def set_tolerances(self, tol, max_refine, krylov_tol=1e-11, max_iters=200):
        _check(load().fdi_plan_set_tolerances(self.handle, tol, max_refine, krylov_tol, max_iters),
               "fdi_plan_set_tolerances")

    def field_shape(self, field=FIELD_CELL):
        nx, ny, nz = self.n
        return {FIELD_CELL: (nz, ny, nx), FIELD_U: (nz, ny, nx - 1), FIELD_V: (nz, ny - 1, nx),
                FIELD_W: (nz - 1, ny, nx)}[field]

    def eigen(self, field=FIELD_CELL, d=0):
        """(lam, E, Einv) of direction d of a field, copied to host."""
        lib = load()
        m = C.c_int()
        _check(lib.fdi_plan_eigen(self.handle, field, d, None, None, None, C.byref(m)), "fdi_plan_eigen")
        lam = np.empty(m.value)
        E = np.empty((m.value, m.value))
        Einv = np.empty((m.value, m.value))
        dp = C.POINTER(C.c_double)
        _check(lib.fdi_plan_eigen(self.handle, field, d, lam.ctypes.data_as(dp), E.ctypes.data_as(dp),
                                  Einv.ctypes.data_as(dp), C.byref(m)), "fdi_plan_eigen")
        return lam, E, Einv


def plan_create(faces, n=None, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), grid=GRID_CELL, prec=PREC_FP64, thomas_axis=2):
    return Plan(faces, n, bc_lo, bc_hi, grid, prec, thomas_axis)


class CylPlan(Plan):
    """Owning handle of a cylindrical plan (fdi_plan_create_cyl): fields in C
    order [n_z][n_theta][n_r], r fastest."""

    def __init__(self, rfaces, ntheta, zfaces, bc_r=(0, 0), bc_z=(0, 0), prec=PREC_FP64, tpf=False):
        lib = load()
        self._faces = [np.ascontiguousarray(np.asarray(f, dtype=np.float64)) for f in (rfaces, zfaces)]
        nr, nz = self._faces[0].size - 1, self._faces[1].size - 1
        self.n = (nr, int(ntheta), nz)
        self.grid, self.prec, self.thomas_axis = GRID_CELL, prec, -1 if tpf else 0
        dp = C.POINTER(C.c_double)
        h = C.c_void_p()
        _check(lib.fdi_plan_create_cyl(self._faces[0].ctypes.data_as(dp), nr, int(ntheta),
                                       self._faces[1].ctypes.data_as(dp), nz, int(bc_r[0]), int(bc_r[1]),
                                       int(bc_z[0]), int(bc_z[1]), prec, 1 if tpf else 0, C.byref(h)),
               "fdi_plan_create_cyl")
        self.handle = h.value


def plan_create_cyl(rfaces, ntheta, zfaces, bc_r=(0, 0), bc_z=(0, 0), prec=PREC_FP64, tpf=False):
    """Cylindrical plan (Sec. 6): radial faces (rfaces[0] = 0: the axis),
    ntheta uniform periodic cells, axial faces; bc_r = (inner, outer),
    bc_z = (low, high) wall types; tpf: eigen decomposition along r per theta
    mode (Eq. 45-46, FP64 only) instead of the radial Thomas sweep (Eq. 44)."""
    return CylPlan(rfaces, ntheta, zfaces, bc_r, bc_z, prec, tpf)


def plan_destroy(plan: Plan):
    plan.destroy()


def helmholtz_solve(plan: Plan, lam, rhs, out, stream=None):
    _check(load().fdi_helmholtz_solve(plan.handle, float(lam), _ptr(rhs), _ptr(out), _stream(stream)),
           "fdi_helmholtz_solve")


def laplace_solve(plan: Plan, rhs, out, stream=None):
    _check(load().fdi_laplace_solve(plan.handle, _ptr(rhs), _ptr(out), _stream(stream)), "fdi_laplace_solve")


def field_solve(plan: Plan, field, sigma, lam, rhs, out, stream=None):
    _check(load().fdi_field_solve(plan.handle, int(field), float(sigma), float(lam), _ptr(rhs), _ptr(out),
                                  _stream(stream)), "fdi_field_solve")


def stokes_solve(plan: Plan, dt, Re, f, u, p, stream=None):
    fa = (C.c_void_p * 3)(*[_ptr(t) for t in f])
    ua = (C.c_void_p * 3)(*[_ptr(t) for t in u])
    _check(load().fdi_stokes_solve(plan.handle, float(dt), float(Re), fa, ua, _ptr(p), _stream(stream)),
           "fdi_stokes_solve")


def helmholtz_solve_batched(plans, lambdas, rhs, out, stream=None):
    k = len(plans)
    pa = (C.c_void_p * k)(*[p.handle for p in plans])
    la = (C.c_double * k)(*[float(v) for v in lambdas])
    ra = (C.c_void_p * k)(*[_ptr(t) for t in rhs])
    oa = (C.c_void_p * k)(*[_ptr(t) for t in out])
    _check(load().fdi_helmholtz_solve_batched(pa, la, ra, oa, k, _stream(stream)), "fdi_helmholtz_solve_batched")


def _host_ptr(x, count):
    """Address of a C-contiguous FP64 host array (numpy array or CPU torch tensor)."""
    if hasattr(x, "data_ptr"):
        if x.is_cuda or not x.is_contiguous() or str(x.dtype) != "torch.float64":
            raise ValueError("host arrays must be contiguous float64 CPU tensors")
        if x.numel() != count:
            raise ValueError(f"host array has {x.numel()} values, the field {count}")
        return x.data_ptr()
    if not (x.dtype == "float64" and x.flags["C_CONTIGUOUS"]):
        raise ValueError("host arrays must be C-contiguous float64")
    if x.size != count:
        raise ValueError(f"host array has {x.size} values, the field {count}")
    return x.ctypes.data


def field_solve_host(plan: Plan, field, sigma, lam, rhs, out, stream=None):
    """Solves for each host right-hand side rhs[i] into the host array out[i]
    (pipelined host-device copies; pinned CPU tensors overlap best).  Returns
    the relative residual of every solve; raises if one missed its tolerance."""
    k = len(rhs)
    if len(out) != k:
        raise ValueError("rhs and out must have the same length")
    count = int(np.prod(plan.field_shape(field)))
    for o in out:
        if not hasattr(o, "data_ptr") and not o.flags["WRITEABLE"]:
            raise ValueError("output host array is read-only")
    ra = (C.c_void_p * max(k, 1))(*[_host_ptr(t, count) for t in rhs])
    oa = (C.c_void_p * max(k, 1))(*[_host_ptr(t, count) for t in out])
    rel = (C.c_double * max(k, 1))()
    _check(load().fdi_field_solve_host(plan.handle, int(field), float(sigma), float(lam), ra, oa, k, rel,
                                       _stream(stream)), "fdi_field_solve_host")
    return [rel[i] for i in range(k)]


def last_result(plan: Plan):
    """(iters, refine_steps, rel_residual) of the last solve; synchronise first."""
    it, rs, rr = C.c_int(), C.c_int(), C.c_double()
    st = load().fdi_last_result(plan.handle, C.byref(it), C.byref(rs), C.byref(rr))
    if st not in (OK, ERR_NOT_CONVERGED):
        _check(st, "fdi_last_result")
    return it.value, rs.value, rr.value, st


def last_launch_count(plan: Plan) -> int:
    v = C.c_longlong()
    _check(load().fdi_last_launch_count(plan.handle, C.byref(v)), "fdi_last_launch_count")
    return v.value


def _fptr(x):
    """Device pointer of a contiguous float32 CUDA tensor."""
    if not (x.is_cuda and x.is_contiguous() and str(x.dtype) == "torch.float32"):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return x.data_ptr()


def apply_transform(plan: Plan, field, d, inverse, inp, out, rows, stream=None):
    _check(load().fdi_apply_transform(plan.handle, int(field), int(d), 1 if inverse else 0, _fptr(inp), _fptr(out),
                                      int(rows), _stream(stream)), "fdi_apply_transform")


def set_krylov(plan: Plan, method: int):
    """0: BiCGstab, 1: BiCGstab(2) (the paper's solver), 2: conjugate gradients in
    the volume-weighted inner product, for the Stokes pressure system."""
    _check(load().fdi_plan_set_krylov(plan.handle, int(method)), "fdi_plan_set_krylov")


def set_stokes_preconditioner(plan: Plan, mode: int):
    _check(load().fdi_plan_set_stokes_preconditioner(plan.handle, int(mode)), "fdi_plan_set_stokes_preconditioner")


def set_wait_limit(plan: Plan, cycles: int):
    """Bound (SM cycles, 0 = default) on the waits inside the tensor-core
    kernels; also clears the plan's sticky wait-limit flag."""
    _check(load().fdi_plan_set_wait_limit(plan.handle, int(cycles)), "fdi_plan_set_wait_limit")


def set_resident(plan: Plan, enable: bool):
    """Resident small-grid solve (one cooperative launch per solve) on or off
    for the plan's fields with x and y extents <= 128 (mixed plans)."""
    _check(load().fdi_plan_set_resident(plan.handle, 1 if enable else 0), "fdi_plan_set_resident")


def set_thomas_config(plan: Plan, lines_per_cta: int):
    _check(load().fdi_plan_set_thomas_config(plan.handle, int(lines_per_cta)), "fdi_plan_set_thomas_config")


def autotune(plan: Plan, lam, rhs, out, reps=3, stream=None):
    """Time the Thomas configurations on this plan, keep the fastest; returns the
    chosen lines per CTA (2, 64 or 128)."""
    t = C.c_int(0)
    _check(load().fdi_plan_autotune(plan.handle, float(lam), _ptr(rhs), _ptr(out), int(reps), C.byref(t),
                                    _stream(stream)), "fdi_plan_autotune")
    return t.value


def set_graphs(plan: Plan, on=True):
    """Enable / disable CUDA-graph replay of repeated field solves on this plan."""
    _check(load().fdi_plan_set_graphs(plan.handle, 1 if on else 0), "fdi_plan_set_graphs")


def enable_timing(plan: Plan, on=True):
    _check(load().fdi_plan_enable_timing(plan.handle, 1 if on else 0), "fdi_plan_enable_timing")


def kernel_times(plan: Plan, max_entries=64):
    """{kernel name: (total device ms, launches)} accumulated since the last reset."""
    names = (C.c_char_p * max_entries)()
    ms = (C.c_double * max_entries)()
    cnt = (C.c_longlong * max_entries)()
    c = C.c_int()
    _check(load().fdi_plan_kernel_times(plan.handle, max_entries, names, ms, cnt, C.byref(c)),
           "fdi_plan_kernel_times")
    return {names[i].decode(): (ms[i], cnt[i]) for i in range(c.value)}


def reset_kernel_times(plan: Plan):
    _check(load().fdi_plan_reset_kernel_times(plan.handle), "fdi_plan_reset_kernel_times")


def status_string(s: int) -> str:
    return load().fdi_status_string(int(s)).decode()


class Server:
    """Stokes-inverse serving loop (fdi_server_*): resident plan cache, admission
    by device-memory footprint, `slots` concurrent workers.  Requests take host
    NumPy arrays; the arrays are kept referenced until the request is done."""

    def __init__(self, budget_bytes, slots=4):
        h = C.c_void_p()
        _check(load().fdi_server_create(int(budget_bytes), int(slots), C.byref(h)), "fdi_server_create")
        self.handle = h.value
        self._keep = {}

    def submit(self, n, beta, dt, Re, f, u, p, prec=PREC_MIXED_F16):
        """n: (nx, ny, nz); f, u: three contiguous float64 arrays (MAC shapes); p: cell array."""
        for a in list(f) + list(u) + [p]:
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
                raise ValueError("server requests take contiguous float64 NumPy arrays")
        r = StokesRequest()
        r.n = (C.c_int * 3)(*[int(v) for v in n])
        r.beta, r.dt, r.Re, r.prec = float(beta), float(dt), float(Re), int(prec)
        r.f = (C.c_void_p * 3)(*[a.ctypes.data for a in f])
        r.u = (C.c_void_p * 3)(*[a.ctypes.data for a in u])
        r.p = p.ctypes.data
        t = C.c_longlong()
        _check(load().fdi_server_submit(self.handle, C.byref(r), C.byref(t)), "fdi_server_submit")
        self._keep[t.value] = (f, u, p)
        return t.value

    def poll(self, ticket, wait=False):
        res = StokesResult()
        _check(load().fdi_server_poll(self.handle, int(ticket), 1 if wait else 0, C.byref(res)), "fdi_server_poll")
        if res.state == 2:
            self._keep.pop(ticket, None)
        return {"state": res.state, "status": res.status, "iters": res.iters, "rel_residual": res.rel_residual,
                "queue_ms": res.queue_ms, "latency_ms": res.latency_ms}

    def drain(self):
        _check(load().fdi_server_drain(self.handle), "fdi_server_drain")

    def stats(self):
        r = ServerReport()
        _check(load().fdi_server_stats(self.handle, C.byref(r)), "fdi_server_stats")
        return {k: getattr(r, k) for k, _ in ServerReport._fields_}

    def close(self):
        if self.handle:
            _check(load().fdi_server_destroy(self.handle), "fdi_server_destroy")
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stokes_plan_bytes_estimate(n, prec=PREC_MIXED_F16) -> int:
    arr = (C.c_int * 3)(*[int(v) for v in n])
    return int(load().fdi_stokes_plan_bytes_estimate(arr, int(prec)))
