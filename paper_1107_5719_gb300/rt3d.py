"""Thin ctypes binding of librt3d.so (C ABI in include/rt3d.h).

The functions carry the C names and only marshal arguments: numpy arrays
for the host-pointer calls, CUDA torch tensors (or raw device addresses)
for the ``*_dev`` calls.  Every step of the computation runs in the CUDA
library; there is no fallback.  Loading fails loudly if ``librt3d.so`` is
missing or cannot be loaded.

``Solver`` bundles a context with one problem for convenience.
"""

from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

(RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ENOTCONV, RT_ETIMEOUT, RT_ESTATE, RT_ESCRATCH,
 RT_EBOUNDS) = range(9)
RT_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024
RT_FP64, RT_FP32_SWEEP, RT_DF64 = 0, 1, 2
RT_BC_ZERO, RT_BC_PLANCK, RT_BC_DIFFUSION = 0, 1, 2
RT_OS_JACOBI, RT_OS_GAUSS_SEIDEL = 0, 1
RT_FS_LONG, RT_FS_SHORT = 0, 1
RT_SRC_LINEAR, RT_SRC_PARABOLIC = 0, 1

_NAMES = {0: "RT_OK", 1: "RT_EINVAL", 2: "RT_ENOMEM", 3: "RT_ECUDA", 4: "RT_ENOTCONV",
          5: "RT_ETIMEOUT", 6: "RT_ESTATE", 7: "RT_ESCRATCH", 8: "RT_EBOUNDS"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librt3d.so")
# RT3D_CHECKED=1 loads the checked build (bounds tests in the kernels,
# RT_EBOUNDS on a bad index) instead.
LIB_PATH_CHECKED = os.path.join(_HERE, "librt3d_checked.so")
_lib = None
_lock = threading.Lock()

P = C.POINTER(C.c_double)
VP = C.c_void_p


class RtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class rt_stats(C.Structure):
    _fields_ = [("launches", C.c_ulonglong), ("fs_launches", C.c_ulonglong),
                ("fs_ms", C.c_double), ("jacobi_launches", C.c_ulonglong),
                ("jacobi_ms", C.c_double), ("steps", C.c_ulonglong),
                ("lstar_launches", C.c_ulonglong), ("iterations", C.c_ulonglong),
                ("host_syncs", C.c_ulonglong)]


class rt_problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("dy", C.c_double), ("dz", C.c_double), ("chi", VP), ("eps", VP), ("B", VP)]


# name -> (restype, argtypes); pointers to data are passed as void*
_SIGS = {
    "rt_version": (C.c_char_p, []),
    "rt_create": (C.c_int, [C.POINTER(VP), C.c_int, C.c_int]),
    "rt_destroy": (C.c_int, [VP]),
    "rt_last_error": (C.c_char_p, [VP]),
    "rt_set_stream": (C.c_int, [VP, VP]),
    "rt_set_grid": (C.c_int, [VP, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]),
    "rt_set_boundary": (C.c_int, [VP, C.c_int, C.c_int]),
    "rt_set_quadrature": (C.c_int, [VP, C.c_int, VP, VP, VP]),
    "rt_set_opacity": (C.c_int, [VP, VP]),
    "rt_set_epsilon": (C.c_int, [VP, VP]),
    "rt_set_planck": (C.c_int, [VP, VP]),
    "rt_set_opacity_dev": (C.c_int, [VP, VP]),
    "rt_set_epsilon_dev": (C.c_int, [VP, VP]),
    "rt_set_planck_dev": (C.c_int, [VP, VP]),
    "rt_formal_solution": (C.c_int, [VP, VP, VP, VP]),
    "rt_formal_solution_dev": (C.c_int, [VP, VP, VP, VP]),
    "rt_os_step": (C.c_int, [VP, VP, VP, VP, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "rt_os_step_dev": (C.c_int, [VP, VP, VP, VP, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "rt_solve": (C.c_int, [VP, C.c_double, C.c_int, C.c_double, C.c_int, VP,
                           C.POINTER(C.c_int), P, VP, VP]),
    "rt_solve_dev": (C.c_int, [VP, C.c_double, C.c_int, C.c_double, C.c_int, VP,
                               C.POINTER(C.c_int), P, VP, VP]),
    "rt_get_J": (C.c_int, [VP, VP]),
    "rt_set_J": (C.c_int, [VP, VP]),
    "rt_last_step_count": (C.c_int, [VP, C.POINTER(C.c_ulonglong)]),
    "rt_fs32_branch_counts": (C.c_int, [VP, VP, C.POINTER(C.c_ulonglong),
                                        C.POINTER(C.c_ulonglong)]),
    "rt_set_fs_record": (C.c_int, [VP, C.c_longlong]),
    "rt_batch_set_fs_record": (C.c_int, [VP, C.c_longlong]),
    "rt_fs_record_info": (C.c_int, [VP, C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    "rt_set_direction_groups": (C.c_int, [VP, C.c_int]),
    "rt_set_cutoff": (C.c_int, [VP, C.c_double]),
    "rt_set_profiling": (C.c_int, [VP, C.c_int]),
    "rt_set_ng": (C.c_int, [VP, C.c_int, C.c_double]),
    "rt_batch_set_ng": (C.c_int, [VP, C.c_int, C.c_double]),
    "rt_set_os_method": (C.c_int, [VP, C.c_int]),
    "rt_set_fs_method": (C.c_int, [VP, C.c_int]),
    "rt_set_source_order": (C.c_int, [VP, C.c_int]),
    "rt_set_precision": (C.c_int, [VP, C.c_int]),
    "rt_set_df_finish": (C.c_int, [VP, C.c_double]),
    "rt_set_graphs": (C.c_int, [VP, C.c_int]),
    "rt_batch_set_df_finish": (C.c_int, [VP, C.c_double]),
    "rt_checked_build": (C.c_int, []),
    "rt_bounds_selftest": (C.c_int, [VP]),
    "rt_get_plane_order": (C.c_int, [VP, VP]),
    "rt_batch_set_precision": (C.c_int, [VP, C.c_int]),
    "rt_batch_set_os_method": (C.c_int, [VP, C.c_int]),
    "rt_get_stats": (C.c_int, [VP, C.POINTER(rt_stats)]),
    "rt_reset_stats": (C.c_int, [VP]),
    "rt_batch_create": (C.c_int, [C.POINTER(VP), C.c_int, C.c_int, C.c_int, C.POINTER(rt_problem),
                                  C.c_int, C.c_int, C.c_int, VP, VP, VP]),
    "rt_batch_destroy": (C.c_int, [VP]),
    "rt_batch_last_error": (C.c_char_p, [VP]),
    "rt_batch_set_stream": (C.c_int, [VP, VP]),
    "rt_batch_reset": (C.c_int, [VP, C.c_int]),
    "rt_batch_solve": (C.c_int, [VP, C.c_double, C.c_int, C.c_double, C.c_int, VP, VP,
                                 C.POINTER(C.c_int)]),
    "rt_batch_get_J": (C.c_int, [VP, C.c_int, VP]),
    "rt_batch_get_J_dev": (C.c_int, [VP, C.c_int, VP]),
    "rt_batch_set_direction_groups": (C.c_int, [VP, C.c_int]),
    "rt_batch_set_graphs": (C.c_int, [VP, C.c_int]),
    "rt_set_block_threads": (C.c_int, [VP, C.c_int]),
    "rt_set_block_order": (C.c_int, [VP, C.c_int]),
    "rt_batch_set_block_threads": (C.c_int, [VP, C.c_int]),
    "rt_batch_set_block_order": (C.c_int, [VP, C.c_int]),
    "rt_probe_peaks": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "rt_batch_set_profiling": (C.c_int, [VP, C.c_int]),
    "rt_batch_get_stats": (C.c_int, [VP, C.POINTER(rt_stats)]),
    "rt_batch_reset_stats": (C.c_int, [VP]),
    "rt_segment_weights": (C.c_int, [C.c_int, C.c_longlong, VP, VP, VP, VP, VP]),
    "rt_formal_solution_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                             C.c_double, C.c_int, C.c_int, C.c_int, VP, VP, VP,
                                             VP, VP, VP, VP, VP]),
}


def load(path: Optional[str] = None):
    """Load librt3d.so (built by ``paper_1107_5719_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or (LIB_PATH_CHECKED if os.environ.get("RT3D_CHECKED") == "1" else LIB_PATH)
            if not os.path.exists(p):
                raise ImportError(f"{p} is missing: build it with paper_1107_5719_gb300.build.build()")
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def exported_names():
    return list(_SIGS)


def _check(ctx, rc, allow=()):
    if rc != RT_OK and rc not in allow:
        msg = load().rt_last_error(ctx).decode() if ctx else ""
        raise RtError(rc, msg)
    return rc


def _host(a, dtype=np.float64):
    """C-contiguous float64 host array and its address."""
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _dev(t):
    """Device address of a CUDA tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device calls need contiguous CUDA tensors")
    return t.data_ptr()


# ---- C-named wrappers -----------------------------------------------------

def rt_version() -> str:
    return load().rt_version().decode()


def rt_create(device: int = 0, precision: int = RT_FP64):
    h = VP()
    rc = load().rt_create(C.byref(h), device, precision)
    if rc != RT_OK:
        raise RtError(rc, f"rt_create(device={device}, precision={precision}) failed")
    return h.value


def rt_destroy(ctx):
    return load().rt_destroy(ctx)


def rt_last_error(ctx) -> str:
    return load().rt_last_error(ctx).decode()


def rt_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t address, or None."""
    h = getattr(stream, "cuda_stream", stream)
    return _check(ctx, load().rt_set_stream(ctx, h))


def rt_set_grid(ctx, nx, ny, nz, dx=1.0, dy=1.0, dz=1.0):
    return _check(ctx, load().rt_set_grid(ctx, nx, ny, nz, dx, dy, dz))


def rt_set_boundary(ctx, top, bottom):
    return _check(ctx, load().rt_set_boundary(ctx, top, bottom))


def rt_set_quadrature(ctx, mu, phi, w):
    mu, pm = _host(mu)
    phi, pp = _host(phi)
    w, pw = _host(w)
    return _check(ctx, load().rt_set_quadrature(ctx, len(mu), pm, pp, pw))


def _setter(name):
    def f(ctx, arr):
        a, p = _host(arr)
        return _check(ctx, getattr(load(), name)(ctx, p))
    f.__name__ = name
    return f


def _setter_dev(name):
    def f(ctx, t):
        return _check(ctx, getattr(load(), name)(ctx, _dev(t)))
    f.__name__ = name
    return f


rt_set_opacity = _setter("rt_set_opacity")
rt_set_epsilon = _setter("rt_set_epsilon")
rt_set_planck = _setter("rt_set_planck")
rt_set_opacity_dev = _setter_dev("rt_set_opacity_dev")
rt_set_epsilon_dev = _setter_dev("rt_set_epsilon_dev")
rt_set_planck_dev = _setter_dev("rt_set_planck_dev")


def rt_formal_solution(ctx, S, shape, want_lstar=True):
    """Host call: returns (J_fs, Lambda* [27, *shape] or None)."""
    J = np.empty(shape)
    L = np.empty((27, *shape)) if want_lstar else None
    Sp = None
    if S is not None:
        S, Sp = _host(S)
    _check(ctx, load().rt_formal_solution(ctx, Sp, J.ctypes.data, L.ctypes.data if want_lstar else None))
    return J, L


def rt_formal_solution_dev(ctx, S, J_fs, lstar=None):
    return _check(ctx, load().rt_formal_solution_dev(ctx, _dev(S), _dev(J_fs), _dev(lstar)))


def rt_os_step(ctx, J_fs, J_old, tol_inner=1e-12, max_sweeps=1000):
    J_fs, pf = _host(J_fs)
    J_old, po = _host(J_old)
    Jn = np.empty_like(J_old)
    ns = C.c_int()
    _check(ctx, load().rt_os_step(ctx, pf, po, Jn.ctypes.data, tol_inner, max_sweeps, C.byref(ns)))
    return Jn, ns.value


def rt_os_step_dev(ctx, J_fs, J_old, J_new, tol_inner=1e-12, max_sweeps=1000):
    ns = C.c_int()
    _check(ctx, load().rt_os_step_dev(ctx, _dev(J_fs), _dev(J_old), _dev(J_new), tol_inner,
                                      max_sweeps, C.byref(ns)))
    return ns.value


def rt_solve(ctx, shape, tol=1e-8, max_iter=500, tol_inner=1e-12, max_sweeps=1000):
    """Host call: returns dict(J, iters, delta, deltas, sweeps, converged)."""
    J = np.empty(shape)
    it = C.c_int()
    last = C.c_double()
    deltas = np.zeros(max_iter)
    sweeps = np.zeros(max_iter, dtype=np.int32)
    rc = _check(ctx, load().rt_solve(ctx, tol, max_iter, tol_inner, max_sweeps, J.ctypes.data,
                                     C.byref(it), C.byref(last), deltas.ctypes.data,
                                     sweeps.ctypes.data), allow=(RT_ENOTCONV,))
    n = it.value
    return dict(J=J, iters=n, delta=last.value, deltas=deltas[:n], sweeps=sweeps[:n],
                converged=(rc == RT_OK))


def rt_solve_dev(ctx, J_out=None, tol=1e-8, max_iter=500, tol_inner=1e-12, max_sweeps=1000,
                 deltas=None, sweeps=None):
    """Device call (J_out a CUDA tensor or None): returns (iters, delta, converged)."""
    it = C.c_int()
    last = C.c_double()
    pd = deltas.ctypes.data if deltas is not None else None
    ps = sweeps.ctypes.data if sweeps is not None else None
    rc = _check(ctx, load().rt_solve_dev(ctx, tol, max_iter, tol_inner, max_sweeps, _dev(J_out),
                                         C.byref(it), C.byref(last), pd, ps), allow=(RT_ENOTCONV,))
    return it.value, last.value, rc == RT_OK


def rt_get_J(ctx, shape):
    J = np.empty(shape)
    _check(ctx, load().rt_get_J(ctx, J.ctypes.data))
    return J


def rt_set_J(ctx, J):
    J, p = _host(J)
    return _check(ctx, load().rt_set_J(ctx, p))


def rt_last_step_count(ctx) -> int:
    n = C.c_ulonglong()
    _check(ctx, load().rt_last_step_count(ctx, C.byref(n)))
    return n.value


def rt_fs32_branch_counts(ctx, S=None):
    """(steps, series steps) of one counting FP32 march of S (None: from
    the current iterate)."""
    p = None
    if S is not None:
        S, p = _host(S)
    n, s = C.c_ulonglong(), C.c_ulonglong()
    _check(ctx, load().rt_fs32_branch_counts(ctx, p, C.byref(n), C.byref(s)))
    return n.value, s.value


def rt_set_fs_record(ctx, max_bytes=-1):
    return _check(ctx, load().rt_set_fs_record(ctx, int(max_bytes)))


def rt_batch_set_fs_record(b, max_bytes=-1):
    return _bcheck(b, load().rt_batch_set_fs_record(b, int(max_bytes)))


def rt_fs_record_info(ctx):
    """(bytes held, recording valid) of the recorded FP64 march."""
    n, v = C.c_longlong(), C.c_int()
    _check(ctx, load().rt_fs_record_info(ctx, C.byref(n), C.byref(v)))
    return n.value, bool(v.value)


def rt_set_direction_groups(ctx, groups):
    return _check(ctx, load().rt_set_direction_groups(ctx, groups))


def rt_set_cutoff(ctx, cut):
    return _check(ctx, load().rt_set_cutoff(ctx, cut))


def rt_set_ng(ctx, period, min_delta=0.0):
    return _check(ctx, load().rt_set_ng(ctx, period, min_delta))


def rt_batch_set_ng(b, period, min_delta=0.0):
    return _bcheck(b, load().rt_batch_set_ng(b, period, min_delta))


def rt_set_os_method(ctx, method):
    return _check(ctx, load().rt_set_os_method(ctx, method))


def rt_set_fs_method(ctx, method):
    return _check(ctx, load().rt_set_fs_method(ctx, method))


def rt_set_source_order(ctx, order):
    return _check(ctx, load().rt_set_source_order(ctx, order))


def rt_set_precision(ctx, precision):
    return _check(ctx, load().rt_set_precision(ctx, precision))


def rt_checked_build() -> bool:
    return bool(load().rt_checked_build())


def rt_bounds_selftest(ctx):
    """Raw status: RT_EBOUNDS from the checked build, RT_OK otherwise."""
    return load().rt_bounds_selftest(ctx)


def rt_get_plane_order(ctx, nz):
    """Dispatch order of the planes in the march launches (order[r] = plane)."""
    out = np.empty(nz, dtype=np.int32)
    _check(ctx, load().rt_get_plane_order(ctx, out.ctypes.data))
    return out


def rt_batch_set_precision(b, precision):
    return _bcheck(b, load().rt_batch_set_precision(b, precision))


def rt_set_df_finish(ctx, delta_switch):
    return _check(ctx, load().rt_set_df_finish(ctx, delta_switch))


def rt_set_graphs(ctx, on):
    return _check(ctx, load().rt_set_graphs(ctx, 1 if on else 0))


def rt_batch_set_df_finish(b, delta_switch):
    return _bcheck(b, load().rt_batch_set_df_finish(b, delta_switch))


def rt_batch_set_os_method(b, method):
    return _bcheck(b, load().rt_batch_set_os_method(b, method))


def rt_set_profiling(ctx, on=True):
    return _check(ctx, load().rt_set_profiling(ctx, 1 if on else 0))


def rt_get_stats(ctx) -> dict:
    s = rt_stats()
    _check(ctx, load().rt_get_stats(ctx, C.byref(s)))
    return {k: getattr(s, k) for k, _ in rt_stats._fields_}


def rt_reset_stats(ctx):
    return _check(ctx, load().rt_reset_stats(ctx))


def rt_segment_weights(precision, x, w_cur, w_up, e, stream=None):
    """Diagnostic: device segment weights at optical depths x (CUDA tensors)."""
    h = getattr(stream, "cuda_stream", stream)
    return load().rt_segment_weights(precision, x.numel(), _dev(x), _dev(w_cur), _dev(w_up),
                                     _dev(e), h)


def rt_formal_solution_noalloc(nx, ny, nz, dx, dy, dz, top, bottom, mu, phi, w, chi, S, B, J_fs,
                               stream=None):
    """Allocation-free formal solution for callers that may not allocate
    device memory while running.  mu, phi, w: host arrays; chi, S, B, J_fs:
    CUDA tensors (or device addresses).  Returns the status code; the work
    is enqueued on `stream` (torch stream, raw handle, or None)."""
    mu, pm = _host(mu)
    phi, pp = _host(phi)
    w, pw = _host(w)
    h = getattr(stream, "cuda_stream", stream)
    return load().rt_formal_solution_noalloc(nx, ny, nz, dx, dy, dz, top, bottom, len(mu), pm, pp,
                                             pw, _dev(chi), _dev(S), _dev(B), _dev(J_fs), h)


def _bcheck(b, rc, allow=()):
    if rc != RT_OK and rc not in allow:
        raise RtError(rc, load().rt_batch_last_error(b).decode() if b else "")
    return rc


def rt_batch_create(problems, device=0, precision=RT_FP32_SWEEP):
    """Batch of ``workloads.Problem``-like problems sharing quadrature and
    boundary modes (taken from the first problem)."""
    p0 = problems[0]
    keep = []
    arr = (rt_problem * len(problems))()
    for i, p in enumerate(problems):
        chi, pc = _host(p.chi)
        eps, pe = _host(p.eps)
        B, pb = _host(p.B)
        keep += [chi, eps, B]
        arr[i] = rt_problem(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, pc, pe, pb)
    mu, pm = _host(p0.mu)
    phi, pp = _host(p0.phi)
    w, pw = _host(p0.w)
    h = VP()
    rc = load().rt_batch_create(C.byref(h), device, precision, len(problems), arr, p0.top_bc,
                                p0.bottom_bc, len(mu), pm, pp, pw)
    if rc != RT_OK:
        msg = load().rt_batch_last_error(h.value).decode() if h.value else ""
        if h.value:
            load().rt_batch_destroy(h.value)
        raise RtError(rc, msg)
    return h.value


def rt_batch_destroy(b):
    return load().rt_batch_destroy(b)


def rt_batch_last_error(b) -> str:
    return load().rt_batch_last_error(b).decode()


def rt_batch_set_stream(b, stream):
    h = getattr(stream, "cuda_stream", stream)
    return _bcheck(b, load().rt_batch_set_stream(b, h))


def rt_batch_reset(b, rebuild_lstar=False):
    return _bcheck(b, load().rt_batch_reset(b, 1 if rebuild_lstar else 0))


def rt_batch_solve(b, nprob, tol=1e-8, max_iter=1000, tol_inner=1e-12, max_sweeps=1000):
    """Returns dict(iters, deltas, n_converged, converged)."""
    it = np.zeros(nprob, dtype=np.int32)
    dl = np.zeros(nprob)
    nc = C.c_int()
    rc = _bcheck(b, load().rt_batch_solve(b, tol, max_iter, tol_inner, max_sweeps, it.ctypes.data,
                                          dl.ctypes.data, C.byref(nc)), allow=(RT_ENOTCONV,))
    return dict(iters=it, deltas=dl, n_converged=nc.value, converged=(rc == RT_OK))


def rt_batch_get_J(b, p, shape):
    J = np.empty(shape)
    _bcheck(b, load().rt_batch_get_J(b, p, J.ctypes.data))
    return J


def rt_batch_get_J_dev(b, p, J):
    return _bcheck(b, load().rt_batch_get_J_dev(b, p, _dev(J)))


def rt_batch_set_direction_groups(b, groups):
    return _bcheck(b, load().rt_batch_set_direction_groups(b, groups))


def rt_probe_peaks(device: int = 0) -> dict:
    """Measured FP64 and FP32 FMA throughput of the device (TFLOP/s)."""
    a, b = C.c_double(), C.c_double()
    rc = load().rt_probe_peaks(device, C.byref(a), C.byref(b))
    if rc:
        raise RtError(rc, "rt_probe_peaks failed")
    return {"fp64_tflops": a.value, "fp32_tflops": b.value}


def rt_set_block_threads(ctx, threads):
    return _check(ctx, load().rt_set_block_threads(ctx, threads))


def rt_set_block_order(ctx, order):
    return _check(ctx, load().rt_set_block_order(ctx, order))


def rt_batch_set_block_threads(b, threads):
    return _bcheck(b, load().rt_batch_set_block_threads(b, threads))


def rt_batch_set_block_order(b, order):
    return _bcheck(b, load().rt_batch_set_block_order(b, order))


def rt_batch_set_graphs(b, on=True):
    return _bcheck(b, load().rt_batch_set_graphs(b, 1 if on else 0))


def rt_batch_set_profiling(b, on=True):
    return _bcheck(b, load().rt_batch_set_profiling(b, 1 if on else 0))


def rt_batch_get_stats(b) -> dict:
    s = rt_stats()
    _bcheck(b, load().rt_batch_get_stats(b, C.byref(s)))
    return {k: getattr(s, k) for k, _ in rt_stats._fields_}


def rt_batch_reset_stats(b):
    return _bcheck(b, load().rt_batch_reset_stats(b))


# ---- convenience ----------------------------------------------------------

class Solver:
    """One context holding one problem (a ``workloads.Problem``-like object)."""

    def __init__(self, problem, device: int = 0, precision: int = RT_FP64, groups: int = 0,
                 cutoff: Optional[float] = None, ng_period: int = 0, ng_min_delta: float = 0.0,
                 os_method: int = RT_OS_JACOBI, fs_method: int = RT_FS_LONG,
                 record: Optional[int] = None):
        self.p = problem
        self.precision = precision
        self.ctx = rt_create(device, precision)
        self.shape = (problem.nz, problem.ny, problem.nx)
        rt_set_grid(self.ctx, problem.nx, problem.ny, problem.nz, problem.dx, problem.dy, problem.dz)
        rt_set_boundary(self.ctx, problem.top_bc, problem.bottom_bc)
        rt_set_quadrature(self.ctx, problem.mu, problem.phi, problem.w)
        rt_set_opacity(self.ctx, problem.chi)
        rt_set_epsilon(self.ctx, problem.eps)
        rt_set_planck(self.ctx, problem.B)
        if groups:
            rt_set_direction_groups(self.ctx, groups)
        if cutoff is not None:
            rt_set_cutoff(self.ctx, cutoff)
        if ng_period:
            rt_set_ng(self.ctx, ng_period, ng_min_delta)
        if os_method != RT_OS_JACOBI:
            rt_set_os_method(self.ctx, os_method)
        if fs_method != RT_FS_LONG:
            rt_set_fs_method(self.ctx, fs_method)
        if getattr(problem, "src_order", 0):
            rt_set_source_order(self.ctx, problem.src_order)
        if record is not None:
            rt_set_fs_record(self.ctx, record)

    def formal_solution(self, S=None, want_lstar=True):
        return rt_formal_solution(self.ctx, S, self.shape, want_lstar)

    def os_step(self, J_fs, J_old, tol_inner=1e-12, max_sweeps=1000):
        return rt_os_step(self.ctx, J_fs, J_old, tol_inner, max_sweeps)

    def solve(self, tol=None, max_iter=500, tol_inner=1e-12, max_sweeps=1000):
        tol = self.p.tol if tol is None else tol
        return rt_solve(self.ctx, self.shape, tol, max_iter, tol_inner, max_sweeps)

    def close(self):
        if self.ctx:
            rt_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
