"""FP64 CPU oracle for two-stage multisplitting on the 3D Laplace 7-point stencil.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_2009_12638_gb300``) and the library never
imports it.

The arithmetic lives in ``ms_oracle.c`` (plain C, FP64, built with
``-O2 -ffp-contract=off``); this module compiles it on first use and wraps it
with ctypes and numpy.  Paper sections followed (Brown, Bull and Bethune,
"A highly scalable approach to solving linear systems using two-stage
multisplitting"):

* ``apply_A`` -- the 7-point operator of section 2.1 (the Jacobi listing weights
  the six neighbours by 1/6, i.e. point Jacobi for A = 6 I - adjacency).
* ``lift`` / ``residual`` -- right-hand side with Dirichlet data moved to it, and
  the global residual used by the stop rule ||Ax - b||_2 < tol (section 2.1).
* ``block_cg`` -- the inner Krylov stage (section 2.2, section 3), CG from zero.
* ``solve`` -- block Jacobi X_i = A_ii^{-1}(B_i - sum_j A_ij X_j) (section 3,
  Listing 1), correction form, with the global norm assembled from block
  partial sums (section 3).
* ``solve_delayed`` -- the asynchronous variant with bounded delays (sections
  2.1, 2.3 and 3): each block reads its neighbours' values from a sweep that
  may lag by a given delay.

Pins (tests/test_oracle.py): Kronecker-sum operator, sine eigenpairs,
symmetry, discretely harmonic closed forms, the point-Jacobi formula for 1^3
blocks, dense LU for one block and for converged solves, exact block Jacobi
against dense block solves, the truncated inner CG against the Krylov-space
A-norm minimiser with its exact stop index, and ``solve_delayed`` (with exact
inner solves) against dense block solves whose face layers come from the
delayed iterates, sweep by sweep, plus zero delays = synchronous and
convergence to the LU solution.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ms_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libms_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = 1
ERR_NOT_CONVERGED = 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ms_oracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.POINTER(ctypes.c_int)
        ll = ctypes.POINTER(ctypes.c_longlong)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        lib.or_set_threads.argtypes = [c_int]
        lib.or_get_max_threads.restype = c_int
        lib.or_boundary_size.argtypes = [c_int, c_int, c_int]
        lib.or_boundary_size.restype = ctypes.c_longlong
        lib.or_apply_A.argtypes = [c_int, c_int, c_int, d, d]
        lib.or_lift.argtypes = [c_int, c_int, c_int, d, d, d]
        lib.or_residual.argtypes = [c_int, c_int, c_int, d, d, d]
        lib.or_block_cg.argtypes = [c_int, c_int, c_int, d, d, d, c_double, c_int]
        lib.or_block_cg.restype = c_int
        lib.or_solve.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, i, i, i, d, d, d, c_double, c_int,
                                 c_double, c_int, i, ll, d, d]
        lib.or_solve.restype = c_int
        lib.or_solve_overlap.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, i, i, i, c_int, d, d, d, c_double,
                                         c_int, c_double, c_int, i, ll, d, d]
        lib.or_solve_overlap.restype = c_int
        lib.or_solve_ex.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, i, i, i, c_int, c_int, d, d, d, c_double,
                                    c_int, c_double, c_int, i, ll, d, d]
        lib.or_solve_ex.restype = c_int
        lib.or_block_gmres.argtypes = [c_int, c_int, c_int, d, d, c_double, c_int, c_int]
        lib.or_block_gmres.restype = c_int
        lib.or_solve_delayed.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, i, i, i, d, d, d, c_double,
                                         c_int, c_double, c_int, c_int, i, i, d]
        lib.or_solve_delayed.restype = c_int
        _lib = lib
        return lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n: int) -> None:
    """Threads for the loop over blocks inside one sweep (results do not depend on it)."""
    _load().or_set_threads(int(n))


def max_threads() -> int:
    return int(_load().or_get_max_threads())


def boundary_size(nx: int, ny: int, nz: int) -> int:
    return int(_load().or_boundary_size(nx, ny, nz))


def apply_A(u: np.ndarray) -> np.ndarray:
    """A u on an (nz, ny, nx) interior grid, u zero outside (section 2.1)."""
    u = _f64(u)
    nz, ny, nx = u.shape
    y = np.empty_like(u)
    _load().or_apply_A(nx, ny, nz, _dp(u), _dp(y))
    return y


def lift(nx, ny, nz, f=None, bnd=None) -> np.ndarray:
    """bhat = f + lift(g) for one right-hand side; returns shape (nz, ny, nx)."""
    out = np.empty((nz, ny, nx), dtype=np.float64)
    f = None if f is None else _f64(f, (nz, ny, nx))
    bnd = None if bnd is None else _f64(bnd).ravel()
    if bnd is not None and bnd.size != boundary_size(nx, ny, nz):
        raise ValueError("boundary array has the wrong size")
    _load().or_lift(nx, ny, nz, _dp(f), _dp(bnd), _dp(out))
    return out


def residual(bhat: np.ndarray, x: np.ndarray) -> np.ndarray:
    bhat = _f64(bhat)
    x = _f64(x, bhat.shape)
    nz, ny, nx = bhat.shape
    r = np.empty_like(bhat)
    _load().or_residual(nx, ny, nz, _dp(bhat), _dp(x), _dp(r))
    return r


def block_cg(r: np.ndarray, inner_rtol: float, inner_maxit: int):
    """CG on one block system A_ii d = r from d = 0; returns (d, r_final, iterations)."""
    r = _f64(r).copy()
    bz, by, bx = r.shape
    d = np.empty_like(r)
    work = np.empty(2 * r.size, dtype=np.float64)
    m = _load().or_block_cg(bx, by, bz, _dp(r), _dp(d), _dp(work), float(inner_rtol), int(inner_maxit))
    return d, r, int(m)


def block_gmres(r: np.ndarray, inner_rtol: float, inner_maxit: int, restart: int):
    """Restarted GMRES on one block system A_ii d = r from d = 0; returns (d, r_final, iterations)."""
    r = _f64(r).copy()
    bz, by, bx = r.shape
    d = np.empty_like(r)
    m = _load().or_block_gmres(bx, by, bz, _dp(r), _dp(d), float(inner_rtol), int(inner_maxit), int(restart))
    return d, r, int(m)


def _cuts(c):
    return np.ascontiguousarray(c, dtype=np.int32)


def solve(nx, ny, nz, cx, cy, cz, f=None, bnd=None, x0=None, inner_rtol=1e-6, inner_maxit=50,
          outer_tol=1e-8, outer_maxit=100000, history=False, overlap=None, inner="cg", restart=10):
    """Block Jacobi with inner CG for ONE right-hand side.

    Returns a dict: x (nz, ny, nx), status, outer_its, inner_its, rel_residual,
    and history (relative residual of every iterate x^0..x^K) if requested.
    overlap: None = or_solve; o >= 0 = or_solve_overlap with blocks extended
    by o points per face (o = 0 gives or_solve's result).
    inner: "cg" or "gmres" (restarted GMRES(restart), or_block_gmres).
    """
    cx, cy, cz = _cuts(cx), _cuts(cy), _cuts(cz)
    px, py, pz = len(cx) - 1, len(cy) - 1, len(cz) - 1
    x = np.zeros((nz, ny, nx)) if x0 is None else _f64(x0, (nz, ny, nx)).copy()
    f = None if f is None else _f64(f, (nz, ny, nx))
    bnd = None if bnd is None else _f64(bnd).ravel()
    if bnd is not None and bnd.size != boundary_size(nx, ny, nz):
        raise ValueError("boundary array has the wrong size")
    outer = ctypes.c_int(0)
    inner_its_c = ctypes.c_longlong(0)
    rel = ctypes.c_double(0.0)
    hist = np.zeros(outer_maxit + 1) if history else None
    if inner not in ("cg", "gmres"):
        raise ValueError("inner must be 'cg' or 'gmres'")
    if inner == "gmres":
        st = _load().or_solve_ex(nx, ny, nz, px, py, pz, _ip(cx), _ip(cy), _ip(cz), int(overlap or 0), int(restart),
                                 _dp(f), _dp(bnd), _dp(x), float(inner_rtol), int(inner_maxit), float(outer_tol),
                                 int(outer_maxit), ctypes.byref(outer), ctypes.byref(inner_its_c), _dp(hist),
                                 ctypes.byref(rel))
    elif overlap is None:
        st = _load().or_solve(nx, ny, nz, px, py, pz, _ip(cx), _ip(cy), _ip(cz), _dp(f), _dp(bnd), _dp(x),
                              float(inner_rtol), int(inner_maxit), float(outer_tol), int(outer_maxit),
                              ctypes.byref(outer), ctypes.byref(inner_its_c), _dp(hist), ctypes.byref(rel))
    else:
        st = _load().or_solve_overlap(nx, ny, nz, px, py, pz, _ip(cx), _ip(cy), _ip(cz), int(overlap), _dp(f),
                                      _dp(bnd), _dp(x), float(inner_rtol), int(inner_maxit), float(outer_tol),
                                      int(outer_maxit), ctypes.byref(outer), ctypes.byref(inner_its_c), _dp(hist),
                                      ctypes.byref(rel))
    if st == ERR_ARG:
        raise ValueError("oracle rejected the arguments")
    out = dict(x=x, status=int(st), outer_its=int(outer.value), inner_its=int(inner_its_c.value),
               rel_residual=float(rel.value))
    if history:
        out["history"] = hist[: outer.value + 1].copy()
    return out


def solve_delayed(nx, ny, nz, cx, cy, cz, delays, max_delay, f=None, bnd=None, x0=None, inner_rtol=1e-6,
                  inner_maxit=50, outer_tol=1e-8, outer_maxit=1000):
    """Asynchronous block Jacobi with the given per-(sweep, block, face) delays (int array)."""
    cx, cy, cz = _cuts(cx), _cuts(cy), _cuts(cz)
    px, py, pz = len(cx) - 1, len(cy) - 1, len(cz) - 1
    nblocks = px * py * pz
    delays = np.ascontiguousarray(delays, dtype=np.int32).reshape(-1)
    if delays.size < (outer_maxit + 1) * nblocks * 6:
        raise ValueError("need (outer_maxit+1)*nblocks*6 delays")
    x = np.zeros((nz, ny, nx)) if x0 is None else _f64(x0, (nz, ny, nx)).copy()
    f = None if f is None else _f64(f, (nz, ny, nx))
    bnd = None if bnd is None else _f64(bnd).ravel()
    outer = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    st = _load().or_solve_delayed(nx, ny, nz, px, py, pz, _ip(cx), _ip(cy), _ip(cz), _dp(f), _dp(bnd), _dp(x),
                                  float(inner_rtol), int(inner_maxit), float(outer_tol), int(outer_maxit),
                                  int(max_delay), _ip(delays), ctypes.byref(outer), ctypes.byref(rel))
    if st == ERR_ARG:
        raise ValueError("oracle rejected the arguments")
    return dict(x=x, status=int(st), outer_its=int(outer.value), rel_residual=float(rel.value))
