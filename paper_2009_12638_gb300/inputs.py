"""Seeded synthetic inputs for the multisplitting solver (numpy only).

This module produces problem data -- boundary values, sources, block cuts,
probe vectors, delay schedules -- and nothing of the solver's arithmetic.  The
CUDA path, the CPU oracle, the tests and the benchmark all draw their inputs
from here, so that both sides of every parity check see identical bytes.

Grid conventions (the paper's model problem, section 2.1: Laplace's equation
on a box with Dirichlet data):

* interior point (i, j, k), 0 <= i < nx, stored x-fastest, arrays shaped
  (nrhs, nz, ny, nx) or (nz, ny, nx);
* coordinates x_i = (i + 1) / (nx + 1), so the boundary sits at 0 and 1;
* Dirichlet data packed per right-hand side as the faces
  x-(nz*ny), x+(nz*ny), y-(nz*nx), y+(nz*nx), z-(ny*nx), z+(ny*nx)
  (edges and corners are never used by a 7-point stencil).
"""
from __future__ import annotations

import math

import numpy as np


def boundary_size(nx: int, ny: int, nz: int) -> int:
    return 2 * nz * ny + 2 * nz * nx + 2 * ny * nx


def coords(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 1.0) / (n + 1.0)


def interior_from_function(nx, ny, nz, u) -> np.ndarray:
    """Samples u(x, y, z) at the interior points, shape (nz, ny, nx)."""
    z, y, x = np.meshgrid(coords(nz), coords(ny), coords(nx), indexing="ij")
    return np.ascontiguousarray(u(x, y, z), dtype=np.float64)


def boundary_from_function(nx, ny, nz, u) -> np.ndarray:
    """Packed Dirichlet faces sampled from u(x, y, z) on the box boundary."""
    xs, ys, zs = coords(nx), coords(ny), coords(nz)
    zz, yy = np.meshgrid(zs, ys, indexing="ij")  # (nz, ny)
    zx, xx = np.meshgrid(zs, xs, indexing="ij")  # (nz, nx)
    yx, xy = np.meshgrid(ys, xs, indexing="ij")  # (ny, nx)
    faces = [
        u(np.zeros_like(zz), yy, zz), u(np.ones_like(zz), yy, zz),
        u(xx, np.zeros_like(zx), zx), u(xx, np.ones_like(zx), zx),
        u(xy, yx, np.zeros_like(yx)), u(xy, yx, np.ones_like(yx)),
    ]
    return np.concatenate([np.asarray(f, dtype=np.float64).ravel() for f in faces])


def face_slices(nx, ny, nz):
    """(offset, shape) of each packed face: x-, x+, y-, y+, z-, z+."""
    shapes = [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]
    out, off = [], 0
    for s in shapes:
        out.append((off, s))
        off += s[0] * s[1]
    return out


def boundary_uniform(nx, ny, nz, nrhs, seed, lo=-1.0, hi=1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(nrhs, boundary_size(nx, ny, nz)))


def boundary_normal(nx, ny, nz, nrhs, seed) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(nrhs, boundary_size(nx, ny, nz)))


def equal_cuts(n: int, p: int) -> np.ndarray:
    """p nearly equal pieces of n; the remainder goes to the leading blocks."""
    if p < 1 or p > n:
        raise ValueError("need 1 <= p <= n")
    q, rem = divmod(n, p)
    sizes = [q + (1 if a < rem else 0) for a in range(p)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)


def uneven_cuts(n: int, p: int, lo: int, hi: int, rng: np.random.Generator, max_tries: int = 10_000_000):
    """Cut n into p edges, each drawn iid uniform from [lo, hi], kept in the
    order drawn; all p are redrawn until they sum to n."""
    if not (p * lo <= n <= p * hi):
        raise ValueError("n cannot be cut into p edges within [lo, hi]")
    tries = 0
    batch = 4096
    while tries < max_tries:
        draws = rng.integers(lo, hi + 1, size=(batch, p))
        ok = np.nonzero(draws.sum(axis=1) == n)[0]
        if ok.size:
            sizes = draws[ok[0]]
            return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
        tries += batch
    raise RuntimeError("no cut found")


def gaussian_probes(shape, count, seed) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(count,) + tuple(shape))


def delay_schedule(outer_maxit, nblocks, max_delay, seed) -> np.ndarray:
    """Per (sweep, block, face) staleness in [0, max_delay] for the
    bounded-delay asynchronous model."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, max_delay + 1, size=(outer_maxit + 1, nblocks, 6)).astype(np.int32)


def harmonic_linear(x, y, z):
    return x + 2.0 * y + 3.0 * z


def harmonic_xyz(x, y, z):
    return x * y * z


def adjoint_target(x, y, z):
    s2 = math.sqrt(2.0) * math.pi
    return np.sin(math.pi * x) * np.sin(math.pi * y) * np.sinh(s2 * z) / math.sinh(s2)


def make_config(name: str, scale: int = 1) -> dict:
    """The standard workloads.  ``scale`` > 1 shrinks every block edge by that
    factor while keeping the block counts (for quick checks).

    keys: nx, ny, nz, nrhs, cx, cy, cz, bnd (nrhs, nb), f (None or array),
    opts (solver options), and per-workload extras.
    """
    if name == "laplace32_linear":
        n = 32 // scale
        return dict(nx=n, ny=n, nz=n, nrhs=1, cx=equal_cuts(n, 2), cy=equal_cuts(n, 2), cz=equal_cuts(n, 2),
                    bnd=boundary_from_function(n, n, n, harmonic_linear)[None, :], f=None,
                    exact=interior_from_function(n, n, n, harmonic_linear)[None],
                    opts=dict(inner_rtol=1e-6, inner_maxit=50, outer_tol=1e-8))
    if name == "laplace256_u11":
        n = 256 // scale
        return dict(nx=n, ny=n, nz=n, nrhs=1, cx=equal_cuts(n, 4), cy=equal_cuts(n, 4), cz=equal_cuts(n, 4),
                    bnd=boundary_uniform(n, n, n, 1, 2009), f=None,
                    opts=dict(inner_rtol=1e-6, inner_maxit=50, outer_tol=1e-8))
    if name == "batched_uneven":
        nx, ny, nz = 384, 320, 256
        rng = np.random.default_rng(12638)
        cx = uneven_cuts(nx, 5, 40, 96, rng)
        cy = uneven_cuts(ny, 6, 40, 96, rng)
        cz = uneven_cuts(nz, 4, 40, 96, rng)
        if scale > 1:
            cx, cy, cz = (np.asarray(c) // scale for c in (cx, cy, cz))
            nx, ny, nz = int(cx[-1]), int(cy[-1]), int(cz[-1])
        return dict(nx=nx, ny=ny, nz=nz, nrhs=16, cx=cx, cy=cy, cz=cz,
                    bnd=boundary_normal(nx, ny, nz, 16, 12639), f=None,
                    opts=dict(inner_rtol=1e-6, inner_maxit=50, outer_tol=1e-8))
    if name == "adjoint128":
        n = 128 // scale
        return dict(nx=n, ny=n, nz=n, nrhs=1, cx=equal_cuts(n, 4), cy=equal_cuts(n, 4), cz=equal_cuts(n, 4),
                    bnd=boundary_uniform(n, n, n, 1, 4), f=None,
                    target=interior_from_function(n, n, n, adjoint_target),
                    probe_seed=5, nprobes=64,
                    opts=dict(inner_rtol=1e-6, inner_maxit=50, outer_tol=1e-12))
    if name == "laplace512_async":
        n = 512 // scale
        return dict(nx=n, ny=n, nz=n, nrhs=4, cx=equal_cuts(n, 8), cy=equal_cuts(n, 8), cz=equal_cuts(n, 8),
                    bnd=boundary_uniform(n, n, n, 4, 512), f=None,
                    opts=dict(inner_rtol=1e-6, inner_maxit=50, outer_tol=1e-8))
    raise KeyError(name)


CONFIG_NAMES = ("laplace32_linear", "laplace256_u11", "batched_uneven", "adjoint128", "laplace512_async")
