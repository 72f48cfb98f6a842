"""GB300-native two-stage multisplitting for the 3D Laplace 7-point stencil.

Outer block Jacobi (synchronous or asynchronous) with an inner CG per block,
after Brown, Bull and Bethune, "A highly scalable approach to solving linear
systems using two-stage multisplitting" (sections 2.1, 2.2, 3; Listing 1).

This package is a thin layer over the CUDA library libms.so and its C ABI
(include/ms.h): PyTorch supplies device memory and the current stream, every
step of the solve runs in the library's sm_103a kernels.  There is no CPU
fallback; if the library is missing, importing the solver raises.

    grid = Grid(nx, ny, nz, nrhs)
    grid.partition(px, py, pz)                 # or explicit cut arrays
    x, stats = grid.solve(f=None, bnd=g, precision="mixed", mode="sync")
    u = MsSolve.apply(f, g, grid, opts)        # differentiable in f and g
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib

__all__ = ["Grid", "SolveStats", "MsSolve", "boundary_size", "MsError"]

MsError = _lib.MsError


def boundary_size(nx: int, ny: int, nz: int) -> int:
    return 2 * nz * ny + 2 * nz * nx + 2 * ny * nx


def resident_variants():
    """Rows of the resident engine's layout table (ms_resident_variant): a list
    of dicts with threads, strips (4-point x-strips per thread and plane),
    planes (z-planes per CTA at most), d_smem, q_regs, one_reduction."""
    lib = _lib.load()
    n = ctypes.c_int(0)
    lib.ms_resident_variant(-1, ctypes.byref(n), None, None, None, None, None, None)
    rows = []
    for v in range(n.value):
        f = [ctypes.c_int(0) for _ in range(6)]
        rc = lib.ms_resident_variant(v, None, *[ctypes.byref(x) for x in f])
        if rc != _lib.MS_OK:
            raise MsError(f"ms_resident_variant({v}) returned {rc}")
        rows.append(dict(zip(("threads", "strips", "planes", "d_smem", "q_regs", "one_reduction"),
                             (x.value for x in f))))
    return rows


@dataclass
class SolveStats:
    status: int
    outer_its: int
    inner_its: int
    lups: int
    rel_residual: float
    time_ms: float
    launches: int
    cluster: int
    threads: int
    slots: int
    per_rhs_outer_its: list
    per_rhs_rel: list
    sweep_ms: float = 0.0
    sweep_launches: int = 0
    engine: int = 0
    variant: int = -1
    inner_rtol_final: float = 0.0
    history_ms: np.ndarray | None = None
    history: np.ndarray | None = None
    trace: np.ndarray | None = None
    trace_count: int = 0

    @property
    def status_name(self):
        return _lib.STATUS_NAMES.get(self.status, str(self.status))


# numpy view of ms_trace_rec (include/ms.h): one record per block solve
TRACE_DTYPE = np.dtype([("sweep", "<i4"), ("block", "<i4"), ("rhs", "<i4"), ("inner_its", "<i4"),
                        ("block_rr", "<f8"), ("t_ns", "<u8")])


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream_handle(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _make_opts(lib, mode="sync", precision="mixed", inner_rtol=1e-6, inner_maxit=50, outer_tol=1e-8,
               outer_maxit=100000, time_limit_ms=0.0, cluster=0, threads=0, slots=0, check_every=0, use_graph=True,
               slow_block=-1, slow_ns=0, profile=False, engine="auto", persistent="auto", variant=-1,
               inner_adapt=False, overlap=0, inner="cg", gmres_restart=10, wait_polls=0, sum_polls=0):
    o = _lib.Opts()
    lib.ms_default_opts(ctypes.byref(o))
    o.mode = _lib.MODE[mode] if isinstance(mode, str) else int(mode)
    o.precision = _lib.PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.inner_rtol = float(inner_rtol)
    o.inner_maxit = int(inner_maxit)
    o.outer_tol = float(outer_tol)
    o.outer_maxit = int(outer_maxit)
    o.time_limit_ms = float(time_limit_ms)
    o.cluster = int(cluster)
    o.threads = int(threads)
    o.slots = int(slots)
    o.check_every = int(check_every)
    o.use_graph = 1 if use_graph else 0
    o.slow_block = int(slow_block)
    o.slow_ns = int(slow_ns)
    o.profile = 1 if profile else 0
    o.persistent = {"auto": 1, True: 2, False: 0}[persistent] if not isinstance(persistent, int) or isinstance(
        persistent, bool) else int(persistent)
    o.engine = {"auto": 0, "streaming": 1, "resident": 2}[engine] if isinstance(engine, str) else int(engine)
    o.variant = int(variant)
    o.inner_adapt = 1 if inner_adapt else 0
    o.overlap = int(overlap)
    o.inner_method = {"cg": 0, "gmres": 1}[inner] if isinstance(inner, str) else int(inner)
    o.gmres_restart = int(gmres_restart)
    o.wait_polls = int(wait_polls)
    o.sum_polls = int(sum_polls)
    return o


class Grid:
    """A grid handle (ms_create_grid) with its block partition and workspace."""

    def __init__(self, nx: int, ny: int, nz: int, nrhs: int = 1, device=None):
        self._lib = _lib.load()
        self.nx, self.ny, self.nz, self.nrhs = int(nx), int(ny), int(nz), int(nrhs)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.ms_create_grid(self.nx, self.ny, self.nz, self.nrhs, ctypes.byref(h))
        if rc != _lib.MS_OK:
            raise _lib.MsError(rc, self._lib.ms_last_error(None).decode())
        self._h = h
        self.px = self.py = self.pz = 1

    # ------------------------------------------------------------------ housekeeping
    def close(self):
        if getattr(self, "_h", None):
            self._lib.ms_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc not in (_lib.MS_OK,):
            raise _lib.MsError(rc, self._lib.ms_last_error(self._h).decode())

    @property
    def shape(self):
        return (self.nrhs, self.nz, self.ny, self.nx)

    @property
    def npts(self):
        return self.nx * self.ny * self.nz

    @property
    def nbnd(self):
        return boundary_size(self.nx, self.ny, self.nz)

    def partition(self, px, py, pz, cx=None, cy=None, cz=None):
        arr = []
        for c in (cx, cy, cz):
            arr.append(None if c is None else (ctypes.c_int * len(c))(*[int(v) for v in c]))
        self._check(self._lib.ms_partition(self._h, int(px), int(py), int(pz), *arr))
        self.px, self.py, self.pz = int(px), int(py), int(pz)
        return self

    def cuts(self):
        cx = (ctypes.c_int * (self.px + 1))()
        cy = (ctypes.c_int * (self.py + 1))()
        cz = (ctypes.c_int * (self.pz + 1))()
        self._check(self._lib.ms_get_cuts(self._h, cx, cy, cz))
        return list(cx), list(cy), list(cz)

    def _field(self, t, name, shape, allow_none=True):
        if t is None:
            if allow_none:
                return None
            raise ValueError(f"{name} is required")
        if not isinstance(t, torch.Tensor):
            t = torch.as_tensor(np.asarray(t, dtype=np.float64))
        if t.dtype != torch.float64:
            raise TypeError(f"{name} must be float64")
        if t.device != self.device:
            t = t.to(self.device)
        t = t.contiguous()
        if t.numel() != int(np.prod(shape)):
            raise ValueError(f"{name} must have {int(np.prod(shape))} elements, got {t.numel()}")
        return t.view(shape)

    # ------------------------------------------------------------------ solver calls
    def solve(self, f=None, bnd=None, x0=None, out=None, history=False, **opts):
        """Solve A x = f + lift(bnd) for every rhs; returns (x, SolveStats).

        f: (nrhs, nz, ny, nx) or None; bnd: (nrhs, nbnd) or None;
        x0: initial guess (default zero); out: optional result tensor (may be x0).
        opts: mode ('sync'|'async'), precision ('mixed'|'fp64'), inner_rtol,
        inner_maxit, outer_tol, outer_maxit, time_limit_ms, cluster, threads,
        slots, check_every, use_graph, slow_block, slow_ns, profile,
        engine ('auto'|'streaming'|'resident'), persistent, variant (resident
        layout row, see resident_variants(); -1 = tuned), inner_adapt (sync:
        choose the inner tolerance at run time), overlap (sync: blocks extended
        by this many points per face, streaming engine), inner ('cg'|'gmres'),
        gmres_restart (GMRES basis size per cycle, 1..50), wait_polls
        (persistent sync launch: poll budget of its bounded waits, 0 = default),
        sum_polls (resident engine: polls before a cluster sum without a
        cluster barrier gives up, 0 = default; for tests of that wait),
        trace (N > 0: keep the last N block-solve records, returned as
        stats.trace, a numpy array of TRACE_DTYPE, with stats.trace_count).
        """
        return self._call(self._lib.ms_solve, f, bnd, x0, out, history, opts)

    def gcg_solve(self, f=None, bnd=None, x0=None, out=None, **opts):
        """ms_gcg_solve: one global FP64 CG solve of A x = f + lift(bnd) on the
        whole grid (no blocks), the comparison method; returns (x, SolveStats).
        Uses opts outer_tol, outer_maxit (iteration cap) and time_limit_ms;
        stats.outer_its is the iteration count."""
        return self._call(self._lib.ms_gcg_solve, f, bnd, x0, out, False, opts)

    def _call(self, fn, f, bnd, x0, out, history, opts):
        trace_n = int(opts.pop("trace", 0) or 0)
        f = self._field(f, "f", self.shape)
        bnd = self._field(bnd, "bnd", (self.nrhs, self.nbnd))
        if out is None:
            out = torch.zeros(self.shape, dtype=torch.float64, device=self.device)
            if x0 is not None:
                out.copy_(self._field(x0, "x0", self.shape, allow_none=False))
        else:
            if out.dtype != torch.float64 or not out.is_contiguous() or out.device != self.device:
                raise ValueError("out must be a contiguous float64 tensor on the grid's device")
            if x0 is not None and x0.data_ptr() != out.data_ptr():
                out.copy_(self._field(x0, "x0", self.shape, allow_none=False))
        o = _make_opts(self._lib, **opts)
        hist = thist = None
        if history:
            hist = np.zeros((self.nrhs, o.outer_maxit + 1))
            o.res_hist = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            thist = np.zeros(o.outer_maxit + 1)
            o.time_hist = thist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        trace = None
        if trace_n > 0:
            trace = np.zeros(trace_n, dtype=TRACE_DTYPE)
            o.trace_cap = trace_n
            o.trace = trace.ctypes.data_as(ctypes.POINTER(_lib.TraceRec))
        st = _lib.Stats()
        per_its = (ctypes.c_int * self.nrhs)()
        per_rel = (ctypes.c_double * self.nrhs)()
        st.per_rhs_outer_its = per_its
        st.per_rhs_rel = per_rel
        with torch.cuda.device(self.device):
            rc = fn(self._h, _ptr(f), _ptr(bnd), _ptr(out), ctypes.byref(o), ctypes.byref(st),
                    _stream_handle(self.device))
        if rc not in (_lib.MS_OK, _lib.MS_ERR_NOT_CONVERGED, _lib.MS_ERR_TIMEOUT):
            self._check(rc)
        stats = SolveStats(rc, st.outer_its, st.inner_its, st.lups, st.rel_residual, st.time_ms, st.launches,
                           st.cluster, st.threads, st.slots, list(per_its), list(per_rel), st.sweep_ms,
                           st.sweep_launches, st.engine, st.variant, st.inner_rtol_final)
        if hist is not None:
            stats.history = hist
            stats.history_ms = thist
        if trace is not None:
            stats.trace_count = int(st.trace_count)
            stats.trace = trace[:min(trace_n, stats.trace_count)]
        return out, stats

    def solve_host(self, f=None, bnd=None, x=None, **opts):
        """ms_solve_host: numpy (host) arrays in, solution written into x (host)."""
        def host(a, shape):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            if a.size != int(np.prod(shape)):
                raise ValueError("wrong size")
            return a
        f = host(f, self.shape)
        bnd = host(bnd, (self.nrhs, self.nbnd))
        if x is None:
            x = np.zeros(self.shape)
        if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
            raise ValueError("x must be a C-contiguous float64 numpy array")
        o = _make_opts(self._lib, **opts)
        st = _lib.Stats()
        p = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)  # noqa: E731
        with torch.cuda.device(self.device):
            rc = self._lib.ms_solve_host(self._h, p(f), p(bnd), p(x), ctypes.byref(o), ctypes.byref(st),
                                         _stream_handle(self.device))
        if rc not in (_lib.MS_OK, _lib.MS_ERR_NOT_CONVERGED, _lib.MS_ERR_TIMEOUT):
            self._check(rc)
        return x, SolveStats(rc, st.outer_its, st.inner_its, st.lups, st.rel_residual, st.time_ms, st.launches,
                             st.cluster, st.threads, st.slots, [], [], st.sweep_ms, st.sweep_launches, st.engine,
                             st.variant, st.inner_rtol_final)

    def residual(self, x, f=None, bnd=None):
        """True relative residual per rhs (absolute where ||bhat|| = 0), computed on the GPU."""
        f = self._field(f, "f", self.shape)
        bnd = self._field(bnd, "bnd", (self.nrhs, self.nbnd))
        x = self._field(x, "x", self.shape, allow_none=False)
        out = (ctypes.c_double * self.nrhs)()
        with torch.cuda.device(self.device):
            self._check(self._lib.ms_residual(self._h, _ptr(f), _ptr(bnd), _ptr(x), out,
                                              _stream_handle(self.device)))
        return np.array(list(out))

    def norms(self, x, f=None, bnd=None):
        """ms_norms: (rr, bb) device tensors [nrhs] -- sum of (bhat - A x)^2 and of
        bhat^2 over this grid's points (FP64, fixed summation order)."""
        f = self._field(f, "f", self.shape)
        bnd = self._field(bnd, "bnd", (self.nrhs, self.nbnd))
        x = self._field(x, "x", self.shape, allow_none=False)
        rr = torch.empty(self.nrhs, dtype=torch.float64, device=self.device)
        bb = torch.empty(self.nrhs, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            self._check(self._lib.ms_norms(self._h, _ptr(f), _ptr(bnd), _ptr(x), _ptr(rr), _ptr(bb),
                                           _stream_handle(self.device)))
        return rr, bb

    def sweep(self, x_in, x_out, f=None, bnd=None, rr=None, stats=False, **opts):
        """ms_sweep: one synchronous outer sweep, x_out = x^{k+1} from x_in = x^k.
        Returns rr (device [nrhs], sum of (bhat - A x^k)^2 over this grid) and,
        with stats=True, a SolveStats (that call waits for the GPU)."""
        f = self._field(f, "f", self.shape)
        bnd = self._field(bnd, "bnd", (self.nrhs, self.nbnd))
        x_in = self._field(x_in, "x_in", self.shape, allow_none=False)
        if (x_out.dtype != torch.float64 or not x_out.is_contiguous() or x_out.device != self.device
                or x_out.numel() != self.nrhs * self.npts):
            raise ValueError("x_out must be a contiguous float64 tensor of the grid's shape on its device")
        if rr is None:
            rr = torch.empty(self.nrhs, dtype=torch.float64, device=self.device)
        o = _make_opts(self._lib, **opts)
        st = _lib.Stats() if stats else None
        with torch.cuda.device(self.device):
            self._check(self._lib.ms_sweep(self._h, _ptr(f), _ptr(bnd), _ptr(x_in), _ptr(x_out), _ptr(rr),
                                           ctypes.byref(o), ctypes.byref(st) if st is not None else None,
                                           _stream_handle(self.device)))
        if st is None:
            return rr
        return rr, SolveStats(st.status, st.outer_its, st.inner_its, st.lups, st.rel_residual, st.time_ms,
                              st.launches, st.cluster, st.threads, st.slots, [], [], st.sweep_ms, st.sweep_launches,
                              st.engine, st.variant, st.inner_rtol_final)

    def face_gather(self, lam):
        """grad_bnd[s][p] = lam[s][q(p)] (the adjoint of the boundary lift)."""
        lam = self._field(lam, "lam", self.shape, allow_none=False)
        out = torch.empty((self.nrhs, self.nbnd), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            self._check(self._lib.ms_face_gather(self._h, _ptr(lam), _ptr(out), _stream_handle(self.device)))
        return out


class MsSolve(torch.autograd.Function):
    """u = A^{-1}(f + lift(bnd)) with a hand-written adjoint.

    A is symmetric (the 7-point Laplacian), so the backward pass solves
    A lam = dL/du with the same block solver and returns dL/df = lam and
    dL/dbnd = lam at the interior point next to each boundary point.  The
    forward solution is saved (checkpointed) for reuse as the caller needs it.
    """

    @staticmethod
    def forward(ctx, f, bnd, grid: Grid, opts: dict):
        opts = dict(opts or {})
        u, st = grid.solve(f=f, bnd=bnd, **opts)
        if st.status not in (_lib.MS_OK,):
            raise _lib.MsError(st.status, "forward solve did not converge")
        ctx.grid = grid
        ctx.opts = opts
        ctx.save_for_backward(u)
        ctx.forward_stats = st
        return u

    @staticmethod
    def backward(ctx, grad_u):
        grid = ctx.grid
        lam, st = grid.solve(f=grad_u.contiguous(), bnd=None, **ctx.opts)
        if st.status not in (_lib.MS_OK,):
            raise _lib.MsError(st.status, "adjoint solve did not converge")
        grad_f = lam if ctx.needs_input_grad[0] else None
        grad_b = grid.face_gather(lam) if ctx.needs_input_grad[1] else None
        return grad_f, grad_b, None, None
