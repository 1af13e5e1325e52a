"""FP64 CPU oracle for the 3DRT hot path (test infrastructure only).

The arithmetic lives in ``rt_oracle.c`` (plain C, FP64, no FMA contraction),
compiled here with gcc; this module only builds it and marshals numpy
arrays through ctypes.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import it; the GPU library never does.

Sections of Hauschildt & Baron (2011) that each function follows:
  formal_solution     Sect. 2.2 (formal solution, J and Lambda*; long or
                      short characteristics)
  mean_intensity_at,  Sect. 2.2 (J, Lambda* at sampled voxels only)
  lstar_at
  intensity           Sect. 2.2 (intensity along one characteristic)
  os_step             Sect. 2.3 (operator splitting, Jordan iterations or
                      red-black Gauss-Seidel)
  solve               Sect. 2 (outer iteration, optional Ng acceleration),
                      Sect. 3.1 item 5 (S)
  ng_step             Sect. 2 (Ng acceleration of the outer iteration)
  weights             segment weights of the linear-source integral
  weights_parabolic   segment weights of the parabolic-source integral
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, NOTCONV = 0, 1, 2, 3


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("top_bc", C.c_int), ("bottom_bc", C.c_int), ("src_order", C.c_int)]


def build(force: bool = False) -> str:
    """Compile rt_oracle.c into liboracle.so (gcc, -O2, OpenMP, no FMA
    contraction so x86 and Arm hosts give the same rounding)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the argument types of the exported oracle functions."""
    P = C.POINTER(C.c_double)
    G = C.POINTER(Grid)
    lib.orc_weights.argtypes = [C.c_double, P, P]
    lib.orc_weights.restype = None
    lib.orc_weights_parabolic.argtypes = [C.c_double, C.c_double, P, P, P]
    lib.orc_weights_parabolic.restype = None
    lib.orc_intensity.argtypes = [G, P, P, P, C.c_double, C.c_double,
                                  C.c_long, C.c_long, C.c_long]
    lib.orc_intensity.restype = C.c_double
    lib.orc_formal_solution.argtypes = [G, P, P, P, C.c_int, P, P, P, P, P, C.c_int]
    lib.orc_mean_intensity_at.argtypes = [G, P, P, P, C.c_int, P, P, P, C.c_long,
                                          C.POINTER(C.c_long), P, C.c_int]
    lib.orc_lstar_at.argtypes = [G, P, C.c_int, P, P, P, C.c_long, C.POINTER(C.c_long), P,
                                 C.c_int]
    lib.orc_os_step.argtypes = [G, P, P, P, P, P, C.c_double, C.c_int,
                                C.POINTER(C.c_int)]
    lib.orc_solve.argtypes = [G, P, P, P, C.c_int, P, P, P, C.c_double, C.c_int,
                              C.c_double, C.c_int, C.c_int, P, P,
                              C.POINTER(C.c_int), P, C.POINTER(C.c_int), C.c_int]
    lib.orc_solve_ng.argtypes = lib.orc_solve.argtypes + [C.c_int, C.c_double]
    lib.orc_solve_ex.argtypes = lib.orc_solve_ng.argtypes + [C.c_int, C.c_int]
    lib.orc_formal_solution_sc.argtypes = lib.orc_formal_solution.argtypes
    lib.orc_os_step_method.argtypes = lib.orc_os_step.argtypes + [C.c_int]
    lib.orc_ng_step.argtypes = [C.c_long, P, P, P, P, P, P, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(C.CDLL(_LIB))
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _grid(p) -> Grid:
    return Grid(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, p.top_bc, p.bottom_bc,
                getattr(p, "src_order", 0))


def weights(x: float):
    """(w_cur, w_up) of one segment with optical depth x."""
    lib = _load()
    a, b = C.c_double(), C.c_double()
    lib.orc_weights(float(x), C.byref(a), C.byref(b))
    return a.value, b.value


def weights_parabolic(a: float, b: float):
    """(P_up, P_cur, P_down) of a segment with optical depth a whose
    downstream neighbour segment has optical depth b."""
    lib = _load()
    u, c, d = C.c_double(), C.c_double(), C.c_double()
    lib.orc_weights_parabolic(float(a), float(b), C.byref(u), C.byref(c), C.byref(d))
    return u.value, c.value, d.value


def intensity(p, S, mu, phi, i, j, k) -> float:
    """Intensity at voxel (i,j,k) in direction (mu, phi) for source S."""
    lib = _load()
    g = _grid(p)
    chi, pc = _d(p.chi)
    S, ps = _d(S)
    B, pb = _d(p.B)
    return lib.orc_intensity(C.byref(g), pc, ps, pb, float(mu), float(phi), i, j, k)


def formal_solution(p, S, lstar: bool = True, nthreads: int = 0, method: int = 0):
    """Return (J_fs, Lambda* [27][nz][ny][nx] or None) for source S; method
    LONG (long characteristics) or SHORT (short characteristics)."""
    lib = _load()
    g = _grid(p)
    chi, pc = _d(p.chi)
    S, ps = _d(S)
    B, pb = _d(p.B)
    mu, pm = _d(p.mu)
    phi, pp = _d(p.phi)
    w, pw = _d(p.w)
    J = np.empty((p.nz, p.ny, p.nx))
    L = np.empty((27, p.nz, p.ny, p.nx)) if lstar else None
    fn = lib.orc_formal_solution_sc if method == SHORT else lib.orc_formal_solution
    rc = fn(C.byref(g), pc, ps, pb, len(mu), pm, pp, pw,
            J.ctypes.data_as(C.POINTER(C.c_double)),
            L.ctypes.data_as(C.POINTER(C.c_double)) if lstar else None, nthreads)
    if rc:
        raise ValueError(f"oracle formal_solution rejected its input ({rc})")
    return J, L


def mean_intensity_at(p, S, voxels, nthreads: int = 0):
    """J at the given flat voxel indices only."""
    lib = _load()
    g = _grid(p)
    chi, pc = _d(p.chi)
    S, ps = _d(S)
    B, pb = _d(p.B)
    mu, pm = _d(p.mu)
    phi, pp = _d(p.phi)
    w, pw = _d(p.w)
    vox = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.empty(vox.shape[0])
    rc = lib.orc_mean_intensity_at(C.byref(g), pc, ps, pb, len(mu), pm, pp, pw,
                                   vox.shape[0], vox.ctypes.data_as(C.POINTER(C.c_long)),
                                   out.ctypes.data_as(C.POINTER(C.c_double)), nthreads)
    if rc:
        raise ValueError(f"oracle mean_intensity_at rejected its input ({rc})")
    return out


def lstar_at(p, voxels, nthreads: int = 0):
    """Lambda* rows [len(voxels)][27] at the given flat voxel indices only
    (the same contributions as formal_solution's Lambda*)."""
    lib = _load()
    g = _grid(p)
    chi, pc = _d(p.chi)
    mu, pm = _d(p.mu)
    phi, pp = _d(p.phi)
    w, pw = _d(p.w)
    vox = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.empty((vox.shape[0], 27))
    rc = lib.orc_lstar_at(C.byref(g), pc, len(mu), pm, pp, pw, vox.shape[0],
                          vox.ctypes.data_as(C.POINTER(C.c_long)),
                          out.ctypes.data_as(C.POINTER(C.c_double)), nthreads)
    if rc:
        raise ValueError(f"oracle lstar_at rejected its input ({rc})")
    return out


JACOBI, GAUSS_SEIDEL = 0, 1
LONG, SHORT = 0, 1


def os_step(p, lstar, J_fs, J_old, tol_inner=1e-12, max_sweeps=1000, method=JACOBI):
    """Return (J_new, sweeps); method JACOBI or GAUSS_SEIDEL (red-black)."""
    lib = _load()
    g = _grid(p)
    L, pl = _d(lstar)
    eps, pe = _d(p.eps)
    Jf, pf = _d(J_fs)
    Jo, po = _d(J_old)
    Jn = np.empty_like(Jo)
    ns = C.c_int()
    rc = lib.orc_os_step_method(C.byref(g), pl, pe, pf, po,
                                Jn.ctypes.data_as(C.POINTER(C.c_double)),
                                float(tol_inner), int(max_sweeps), C.byref(ns), int(method))
    if rc:
        raise ValueError(f"oracle os_step rejected its input ({rc})")
    return Jn, ns.value


def ng_step(x0, x1, x2, x3):
    """Second-order Ng extrapolation of four iterates (x0 newest); returns
    (x, a, b, singular)."""
    lib = _load()
    a0, p0 = _d(x0)
    a1, p1 = _d(x1)
    a2, p2 = _d(x2)
    a3, p3 = _d(x3)
    out = np.empty_like(a0)
    a, b = C.c_double(), C.c_double()
    rc = lib.orc_ng_step(a0.size, p0, p1, p2, p3, out.ctypes.data_as(C.POINTER(C.c_double)),
                         C.byref(a), C.byref(b))
    return out, a.value, b.value, bool(rc)


def solve(p, tol=None, max_iter=500, tol_inner=1e-12, max_sweeps=1000, J0=None,
          nthreads: int = 0, want_lstar: bool = False, ng_period: int = 0,
          ng_min_delta: float = 0.0, os_method: int = JACOBI, fs_method: int = 0):
    """Outer iteration (Ng acceleration every ng_period iterations if > 0;
    operator splitting by os_method, JACOBI or GAUSS_SEIDEL; formal solution
    by fs_method, LONG or SHORT characteristics).
    Returns a dict with J, iters, deltas, sweeps, converged (and lstar if
    asked)."""
    lib = _load()
    g = _grid(p)
    chi, pc = _d(p.chi)
    eps, pe = _d(p.eps)
    B, pb = _d(p.B)
    mu, pm = _d(p.mu)
    phi, pp = _d(p.phi)
    w, pw = _d(p.w)
    J = np.array(J0 if J0 is not None else p.B, dtype=np.float64, order="C")
    L = np.empty((27, p.nz, p.ny, p.nx)) if want_lstar else None
    deltas = np.zeros(max_iter)
    sweeps = np.zeros(max_iter, dtype=np.int32)
    iters = C.c_int()
    tol = p.tol if tol is None else tol
    rc = lib.orc_solve_ex(C.byref(g), pc, pe, pb, len(mu), pm, pp, pw, float(tol),
                          int(max_iter), float(tol_inner), int(max_sweeps),
                          1 if J0 is not None else 0, J.ctypes.data_as(C.POINTER(C.c_double)),
                          L.ctypes.data_as(C.POINTER(C.c_double)) if want_lstar else None,
                          C.byref(iters), deltas.ctypes.data_as(C.POINTER(C.c_double)),
                          sweeps.ctypes.data_as(C.POINTER(C.c_int)), nthreads, int(ng_period),
                          float(ng_min_delta), int(os_method), int(fs_method))
    if rc not in (OK, NOTCONV):
        raise ValueError(f"oracle solve rejected its input ({rc})")
    n = iters.value
    out = dict(J=J, iters=n, deltas=deltas[:n].copy(), sweeps=sweeps[:n].copy(),
               converged=(rc == OK))
    if want_lstar:
        out["lstar"] = L
    return out
