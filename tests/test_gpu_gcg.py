"""Parity of the global FP64 CG (ms_gcg_solve, the single-matrix comparison
method) with the oracle.  With one block covering the grid, the oracle's
block-Jacobi sweep from x0 = 0 is exactly m iterations of CG on A (the inner
method of sections 2.2 and 3), a case already pinned to dense LU in the CPU
tests; both sides are FP64, so iterates agree up to summation order
(1e-11 relative in the inf-norm)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12638_gb300 import Grid, inputs

pytestmark = pytest.mark.gpu


def cuda(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def oracle_cg(nx, ny, nz, bnd, f=None, iters=None, rtol=0.0, maxit=100000):
    """CG on the whole grid: one oracle sweep with a single block."""
    return oracle.solve(nx, ny, nz, [0, nx], [0, ny], [0, nz], f=f, bnd=bnd, inner_rtol=rtol,
                        inner_maxit=iters if iters is not None else maxit, outer_tol=0.0, outer_maxit=1)


@pytest.mark.parametrize("shape", [(16, 16, 16), (13, 11, 9), (40, 7, 22), (1, 1, 30)])
@pytest.mark.parametrize("iters", [1, 7, 25])
def test_gcg_iterates_match_oracle(shape, iters):
    nx, ny, nz = shape
    rng = np.random.default_rng(60 + iters)
    bnd = rng.uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    f = rng.uniform(-1, 1, size=(1, nz, ny, nx))
    g = Grid(nx, ny, nz, 1)
    x, st = g.gcg_solve(f=cuda(f), bnd=cuda(bnd), outer_tol=0.0, outer_maxit=iters)
    ref = oracle_cg(nx, ny, nz, bnd[0], f=f[0], iters=iters)
    assert st.status_name == "ERR_NOT_CONVERGED" and st.outer_its == iters
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 1e-11


def test_gcg_stop_rule_matches_oracle_count():
    """Stop on ||r_k|| < tol ||bhat||: the same iteration count as the oracle's
    single-block CG with inner tolerance tol (+-1: the oracle tests <= after
    each step, both on recurrence residuals whose rounding differs)."""
    nx, ny, nz = 24, 20, 18
    bnd = np.random.default_rng(61).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = Grid(nx, ny, nz, 1)
    for tol in (1e-4, 1e-8, 1e-12):
        x, st = g.gcg_solve(bnd=cuda(bnd), outer_tol=tol)
        ref = oracle_cg(nx, ny, nz, bnd[0], rtol=tol)
        assert st.status == 0 and abs(st.outer_its - ref["inner_its"]) <= 1, (tol, st.outer_its, ref["inner_its"])
        assert st.rel_residual < 2 * tol
        assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= max(1e-10, 10 * tol * 0.5 * (nx + 1) ** 2)


def test_gcg_reproduces_discretely_harmonic_closed_form():
    cfg = inputs.make_config("laplace32_linear")
    n = cfg["nx"]
    g = Grid(n, n, n, 1)
    x, st = g.gcg_solve(bnd=cuda(cfg["bnd"]), outer_tol=1e-13)
    assert st.status == 0
    assert rel_inf(x.cpu().numpy()[0], cfg["exact"][0]) <= 1e-9


def test_gcg_rhs_are_independent_and_warm_start():
    nx, ny, nz = 20, 18, 16
    rng = np.random.default_rng(62)
    bnd = rng.uniform(-1, 1, size=(3, inputs.boundary_size(nx, ny, nz)))
    bnd[1] *= 0.0  # a zero right-hand side stops at k = 0 with x = x0 = 0
    g3 = Grid(nx, ny, nz, 3)
    x3, s3 = g3.gcg_solve(bnd=cuda(bnd), outer_tol=1e-10)
    assert s3.status == 0 and s3.per_rhs_outer_its[1] == 0
    assert not x3[1].any()
    g1 = Grid(nx, ny, nz, 1)
    x1, s1 = g1.gcg_solve(bnd=cuda(bnd[2:3]), outer_tol=1e-10)
    np.testing.assert_array_equal(x3[2].cpu().numpy(), x1[0].cpu().numpy())
    assert s1.outer_its == s3.per_rhs_outer_its[2]
    # warm start from a perturbed solution converges to the same tolerance in fewer iterations
    x0 = x1 + 1e-6 * torch.from_numpy(rng.standard_normal(x1.shape)).cuda()
    xw, sw = g1.gcg_solve(bnd=cuda(bnd[2:3]), x0=x0, outer_tol=1e-10)
    assert sw.status == 0 and sw.rel_residual < 1e-10 * 1.01 + 1e-12 and sw.outer_its < s1.outer_its


def test_gcg_iteration_cap():
    g = Grid(12, 12, 12, 2)
    bnd = np.random.default_rng(63).uniform(-1, 1, size=(2, g.nbnd))
    x, st = g.gcg_solve(bnd=cuda(bnd), outer_tol=1e-14, outer_maxit=5)
    assert st.status_name == "ERR_NOT_CONVERGED" and st.outer_its == 5 and st.per_rhs_outer_its == [5, 5]
    x, st = g.gcg_solve(bnd=cuda(bnd), outer_tol=1e-14, outer_maxit=0)
    assert st.outer_its == 0 and not x.any()


def test_gcg_full_size_256_true_residual():
    """The 256^3 workload: global FP64 CG to 1e-8 (the comparison line of the bench)."""
    cfg = inputs.make_config("laplace256_u11")
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], 1)
    b = cuda(cfg["bnd"])
    x, st = g.gcg_solve(bnd=b, outer_tol=1e-8)
    assert st.status == 0 and st.rel_residual < 1e-8
    assert g.residual(x, bnd=b)[0] < 1e-8
