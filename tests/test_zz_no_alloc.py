"""ms_residual_noalloc: the residual entry point for callers that cannot
allocate device memory at the point of the call (in a latency-critical loop
that cannot absorb cudaMalloc's implicit synchronisation, or with all device
memory owned by their own pool allocator).  It must
give the same numbers as ms_residual, call after call, although its scratch
is one fixed device array shared by every call.

This file is collected last on purpose (tests/test_zz_*) so that a run that
stops at the first failure has already run every other test; it also passes
on its own in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2009_12638_gb300 import Grid, _lib, inputs

pytestmark = pytest.mark.gpu


def _call(grid, f, bnd, x, out):
    lib = _lib.load()
    p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.ms_residual_noalloc(grid._h, p(f), p(bnd), p(x), p(out), stream)


def test_noalloc_residual_matches_ms_residual_twice():
    nx, ny, nz, nrhs = 37, 29, 23, 3
    grid = Grid(nx, ny, nz, nrhs)
    rng = np.random.default_rng(60)
    for call in range(2):  # the second call must not see the first call's scratch
        x = torch.from_numpy(rng.standard_normal((nrhs, nz, ny, nx))).cuda()
        bnd = torch.from_numpy(rng.uniform(-1, 1, size=(nrhs, inputs.boundary_size(nx, ny, nz)))).cuda()
        f = torch.from_numpy(rng.standard_normal((nrhs, nz, ny, nx))).cuda() if call else None
        out = torch.full((nrhs,), np.nan, dtype=torch.float64, device="cuda")
        assert _call(grid, f, bnd, x, out) == _lib.MS_OK
        torch.cuda.synchronize()
        want = grid.residual(x, f=f, bnd=bnd)
        np.testing.assert_allclose(out.cpu().numpy(), want, rtol=1e-12, atol=0)


def test_noalloc_residual_rejects_too_many_rhs():
    grid = Grid(2, 2, 2, _lib.NOALLOC_MAX_RHS + 1)
    x = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    out = torch.zeros(grid.nrhs, dtype=torch.float64, device="cuda")
    assert _call(grid, None, None, x, out) == _lib.MS_ERR_ARG
    assert b"MS_NOALLOC_MAX_RHS" in _lib.load().ms_last_error(grid._h)
