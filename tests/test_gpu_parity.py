"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances, derived from the arithmetic:
* FP64 path, same algorithm, different rounding order: iterates after a few
  sweeps agree to ~1e-13 relative; converged solutions must agree within
  1e-9 relative in the inf-norm with the same outer count +-1.
* Mixed path (FP32 inner CG, FP64 outer): it is a different inner
  arithmetic, so iterates are not compared; the converged solution must reach
  the same true relative residual (< tol) and lie within kappa(A) * tol of the
  oracle's converged solution.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12638_gb300 import Grid, MsError, inputs

pytestmark = pytest.mark.gpu


def cuda(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def make_grid(nx, ny, nz, nrhs, cx, cy, cz):
    g = Grid(nx, ny, nz, nrhs)
    g.partition(len(cx) - 1, len(cy) - 1, len(cz) - 1, cx, cy, cz)
    return g


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def oracle_all(cfg, **kw):
    outs = []
    for s in range(cfg["nrhs"]):
        f = None if cfg.get("f") is None else cfg["f"][s]
        outs.append(oracle.solve(cfg["nx"], cfg["ny"], cfg["nz"], cfg["cx"], cfg["cy"], cfg["cz"], f=f,
                                 bnd=cfg["bnd"][s], **kw))
    return outs


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(min(16, oracle.max_threads()))
    yield
    oracle.set_threads(1)


# ---------------------------------------------------------------- converged parity
@pytest.mark.parametrize("cluster,threads", [(0, 0), (1, 256), (4, 512), (8, 1024)])
def test_laplace32_fp64_sync_matches_oracle(cluster, threads):
    cfg = inputs.make_config("laplace32_linear")
    ref = oracle_all(cfg, history=True, **cfg["opts"])[0]
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    x, st = g.solve(bnd=cuda(cfg["bnd"]), precision="fp64", cluster=cluster, threads=threads, history=True,
                    **cfg["opts"])
    assert st.status == 0 and ref["status"] == 0
    assert abs(st.outer_its - ref["outer_its"]) <= 1
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 1e-9
    k = min(st.outer_its, ref["outer_its"])
    np.testing.assert_allclose(st.history[0][: k + 1], ref["history"][: k + 1], rtol=1e-7)
    # the closed form: u = x + 2y + 3z sampled on the grid solves the discrete problem
    assert rel_inf(x.cpu().numpy()[0], cfg["exact"][0]) <= 440 * 1e-8


def test_laplace32_mixed_sync_reaches_tolerance():
    cfg = inputs.make_config("laplace32_linear")
    ref = oracle_all(cfg, **cfg["opts"])[0]
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    x, st = g.solve(bnd=cuda(cfg["bnd"]), precision="mixed", **cfg["opts"])
    assert st.status == 0 and st.rel_residual < 1e-8
    # independent re-check of the residual through ms_residual
    assert g.residual(x, bnd=cuda(cfg["bnd"]))[0] < 1e-8
    # kappa(A) ~ 440 at 32^3: both solutions lie within kappa * tol of the exact one
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 2 * 440 * 1e-8
    assert abs(st.outer_its - ref["outer_its"]) <= max(3, ref["outer_its"] // 20)


# ---------------------------------------------------------------- first sweeps, bit-close
def first_sweeps_case(nx, ny, nz, cx, cy, cz, nrhs, sweeps, seed, f=False, x0=False, inner_maxit=50, inner_rtol=1e-6,
                      **solve_kw):
    r = np.random.default_rng(seed)
    bnd = r.uniform(-1, 1, size=(nrhs, inputs.boundary_size(nx, ny, nz)))
    ff = r.standard_normal((nrhs, nz, ny, nx)) if f else None
    xx = r.standard_normal((nrhs, nz, ny, nx)) if x0 else np.zeros((nrhs, nz, ny, nx))
    g = make_grid(nx, ny, nz, nrhs, cx, cy, cz)
    x, st = g.solve(f=cuda(ff), bnd=cuda(bnd), x0=cuda(xx), precision="fp64", outer_tol=0.0, outer_maxit=sweeps,
                    inner_maxit=inner_maxit, inner_rtol=inner_rtol, **solve_kw)
    assert st.status == 4 and st.outer_its == sweeps
    xg = x.cpu().numpy()
    for s in range(nrhs):
        ref = oracle.solve(nx, ny, nz, cx, cy, cz, f=None if ff is None else ff[s], bnd=bnd[s], x0=xx[s],
                           outer_tol=0.0, outer_maxit=sweeps, inner_maxit=inner_maxit, inner_rtol=inner_rtol)
        assert rel_inf(xg[s], ref["x"]) <= 1e-11, s


@pytest.mark.parametrize("threads", [256, 512, 1024])
def test_fp64_first_sweeps_on_both_streaming_engines(threads):
    """The plain FP64 path runs on the scalar streaming engine (256 threads
    here) or on the vectorised strip engine in FP64 (512 / 1024 threads: 4-point
    strips of doubles, FP64 cluster sums): both must give the oracle's sweeps."""
    first_sweeps_case(64, 48, 40, [0, 40, 64], [0, 17, 48], [0, 13, 27, 40], 2, 3, 22, f=True, x0=True,
                      engine="streaming", threads=threads)


@pytest.mark.parametrize("case", [
    # (nx, ny, nz, cx, cy, cz): several tiles, ragged tails, thin and single blocks
    (37, 29, 23, [0, 13, 37], [0, 10, 20, 29], [0, 23]),
    (20, 20, 20, [0, 7, 14, 20], [0, 20], [0, 1, 2, 19, 20]),
    (9, 8, 7, list(range(10)), list(range(9)), list(range(8))),   # 1^3 blocks: point Jacobi
    (33, 1, 1, [0, 16, 33], [0, 1], [0, 1]),                       # 1-D
    (64, 48, 40, [0, 40, 64], [0, 17, 48], [0, 13, 27, 40]),
])
def test_first_sweeps_match_oracle_ragged(case):
    nx, ny, nz, cx, cy, cz = case
    first_sweeps_case(nx, ny, nz, cx, cy, cz, 1, 3, 21, f=True, x0=True)


@pytest.mark.parametrize("cluster,threads", [(1, 256), (2, 512), (3, 256), (8, 512), (16, 256)])
def test_first_sweeps_every_launch_shape(cluster, threads):
    first_sweeps_case(24, 20, 33, [0, 11, 24], [0, 20], [0, 5, 33], 1, 2, 22, f=True, cluster=cluster,
                      threads=threads)


def test_first_sweeps_multi_rhs_uneven():
    cfg = inputs.make_config("batched_uneven", scale=4)
    first_sweeps_case(cfg["nx"], cfg["ny"], cfg["nz"], cfg["cx"], cfg["cy"], cfg["cz"], 3, 2, 23)


def test_first_sweeps_without_graph_and_small_chunks():
    first_sweeps_case(16, 16, 16, [0, 8, 16], [0, 8, 16], [0, 8, 16], 2, 5, 24, use_graph=False, check_every=1)
    first_sweeps_case(16, 16, 16, [0, 8, 16], [0, 8, 16], [0, 8, 16], 2, 5, 24, use_graph=True, check_every=3)


def test_inner_maxit_zero_and_one():
    first_sweeps_case(12, 12, 12, [0, 6, 12], [0, 12], [0, 12], 1, 2, 25, inner_maxit=1)
    g = make_grid(8, 8, 8, 1, [0, 4, 8], [0, 8], [0, 8])
    bnd = np.random.default_rng(26).uniform(-1, 1, size=(1, inputs.boundary_size(8, 8, 8)))
    x, st = g.solve(bnd=cuda(bnd), precision="fp64", inner_maxit=0, outer_maxit=3, outer_tol=1e-8)
    assert st.status == 4 and not x.any()


# ---------------------------------------------------------------- stop rule edges
def test_zero_rhs_returns_zero_at_k0():
    g = make_grid(10, 10, 10, 2, [0, 5, 10], [0, 10], [0, 10])
    for prec in ("fp64", "mixed"):
        x, st = g.solve(bnd=torch.zeros(2, g.nbnd, dtype=torch.float64, device="cuda"), precision=prec)
        assert st.status == 0 and st.outer_its == 0 and not x.any()


def test_exact_start_stops_at_k0():
    n = 12
    bnd = inputs.boundary_from_function(n, n, n, inputs.harmonic_xyz)[None]
    x0 = inputs.interior_from_function(n, n, n, inputs.harmonic_xyz)[None]
    g = make_grid(n, n, n, 1, [0, 6, 12], [0, 6, 12], [0, 12])
    x, st = g.solve(bnd=cuda(bnd), x0=cuda(x0), precision="mixed")
    assert st.status == 0 and st.outer_its == 0
    np.testing.assert_array_equal(x.cpu().numpy(), x0)


@pytest.mark.parametrize("prec,threads", [("fp64", 512), ("fp64", 1024), ("mixed", 512), ("mixed", 1024)])
@pytest.mark.parametrize("case", [(6, 6, 6, [0, 3, 6], [0, 6], [0, 6]), (8, 8, 8, [0, 4, 8], [0, 8], [0, 8]),
                                  (13, 7, 9, [0, 1, 5, 9, 13], [0, 7], [0, 4, 9])])
def test_strip_engine_blocks_one_strip_wide(case, prec, threads):
    """Blocks at most 4 points wide hold one x-strip per row: the strip
    engine's strip-to-row mapping must stay exact there (the relative residual
    of x0 = 0 is 1, and two sweeps are the oracle's)."""
    nx, ny, nz, cx, cy, cz = case
    bnd = np.random.default_rng(28).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make_grid(nx, ny, nz, 1, cx, cy, cz)
    shape = dict(precision=prec, engine="streaming", threads=threads)
    x, st = g.solve(bnd=cuda(bnd), outer_maxit=0, history=True, **shape)
    assert st.history[0][0] == pytest.approx(1.0, rel=1e-12)
    x, st = g.solve(bnd=cuda(bnd), outer_tol=0.0, outer_maxit=2, **shape)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], outer_tol=0.0, outer_maxit=2)
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= (1e-11 if prec == "fp64" else 2e-4)


def test_outer_maxit_zero():
    g = make_grid(6, 6, 6, 1, [0, 3, 6], [0, 6], [0, 6])
    bnd = np.random.default_rng(27).uniform(-1, 1, size=(1, inputs.boundary_size(6, 6, 6)))
    x, st = g.solve(bnd=cuda(bnd), precision="fp64", outer_maxit=0, history=True)
    assert st.status == 4 and st.outer_its == 0 and not x.any()
    assert st.history[0][0] == pytest.approx(1.0, rel=1e-14)


def test_per_rhs_independent_stopping():
    """Two rhs: one already solved by x0, one not; each stops on its own."""
    n = 12
    c = inputs.equal_cuts(n, 2)
    b0 = inputs.boundary_from_function(n, n, n, inputs.harmonic_linear)
    b1 = inputs.boundary_uniform(n, n, n, 1, 28)[0]
    x0 = np.zeros((2, n, n, n))
    x0[0] = inputs.interior_from_function(n, n, n, inputs.harmonic_linear)
    g = make_grid(n, n, n, 2, c, c, c)
    x, st = g.solve(bnd=cuda(np.stack([b0, b1])), x0=cuda(x0), precision="fp64")
    ref = oracle.solve(n, n, n, c, c, c, bnd=b1)
    assert st.per_rhs_outer_its[0] == 0
    assert abs(st.per_rhs_outer_its[1] - ref["outer_its"]) <= 1
    assert rel_inf(x.cpu().numpy()[1], ref["x"]) <= 1e-9
    np.testing.assert_array_equal(x.cpu().numpy()[0], x0[0])


# ---------------------------------------------------------------- residual / face gather
def test_residual_matches_oracle():
    nx, ny, nz = 19, 17, 13
    r = np.random.default_rng(29)
    bnd = r.standard_normal((2, inputs.boundary_size(nx, ny, nz)))
    f = r.standard_normal((2, nz, ny, nx))
    x = r.standard_normal((2, nz, ny, nx))
    g = Grid(nx, ny, nz, 2)
    got = g.residual(cuda(x), f=cuda(f), bnd=cuda(bnd))
    for s in range(2):
        bh = oracle.lift(nx, ny, nz, f[s], bnd[s])
        want = np.linalg.norm(oracle.residual(bh, x[s])) / np.linalg.norm(bh)
        assert got[s] == pytest.approx(want, rel=1e-12)
    # zero bhat: absolute norm
    got0 = g.residual(cuda(x))
    for s in range(2):
        assert got0[s] == pytest.approx(np.linalg.norm(oracle.apply_A(x[s])), rel=1e-12)


def test_face_gather_is_lift_transpose():
    """<lift(g), lam> = <g, gather(lam)> for all g, lam (the gather is the adjoint of the lift)."""
    nx, ny, nz = 7, 6, 5
    r = np.random.default_rng(30)
    lam = r.standard_normal((1, nz, ny, nx))
    gb = Grid(nx, ny, nz, 1).face_gather(cuda(lam)).cpu().numpy()[0]
    nb = inputs.boundary_size(nx, ny, nz)
    for _ in range(5):
        gv = r.standard_normal(nb)
        lhs = np.vdot(oracle.lift(nx, ny, nz, None, gv), lam[0])
        assert np.vdot(gv, gb) == pytest.approx(lhs, rel=1e-12)


# ---------------------------------------------------------------- host-buffer entry point
def test_solve_host_matches_device():
    n = 16
    c = inputs.equal_cuts(n, 2)
    bnd = inputs.boundary_uniform(n, n, n, 2, 31)
    g = make_grid(n, n, n, 2, c, c, c)
    # tune the launch shape first: the tuning sweeps try several engines, whose
    # FP64 sums round differently; the two solves compared below use one shape
    g.solve(bnd=cuda(bnd), precision="fp64")
    xd, sd = g.solve(bnd=cuda(bnd), precision="fp64")
    xh = np.zeros((2, n, n, n))
    xh, sh = g.solve_host(bnd=bnd, x=xh, precision="fp64")
    assert sd.status == 0 and sh.status == 0 and sd.outer_its == sh.outer_its
    np.testing.assert_array_equal(xh, xd.cpu().numpy())


# ---------------------------------------------------------------- asynchronous mode
@pytest.mark.parametrize("prec,engine", [("fp64", "auto"), ("mixed", "streaming"), ("mixed", "resident")])
def test_async_converges_to_oracle_solution(prec, engine):
    cfg = inputs.make_config("laplace32_linear")
    ref = oracle_all(cfg, **cfg["opts"])[0]
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    x, st = g.solve(bnd=cuda(cfg["bnd"]), precision=prec, mode="async", engine=engine, **cfg["opts"])
    assert st.engine == (2 if engine == "resident" else 1)
    assert st.status == 0 and st.rel_residual < 1e-8
    assert g.residual(x, bnd=cuda(cfg["bnd"]))[0] < 1e-8
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 2 * 440 * 1e-8


@pytest.mark.parametrize("engine", ["streaming", "resident"])
def test_async_multi_rhs_uneven(engine):
    cfg = inputs.make_config("batched_uneven", scale=4)
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 16, cfg["cx"], cfg["cy"], cfg["cz"])
    x, st = g.solve(bnd=cuda(cfg["bnd"]), precision="mixed", mode="async", engine=engine)
    assert st.status == 0 and max(st.per_rhs_rel) < 1e-8
    assert (g.residual(x, bnd=cuda(cfg["bnd"])) < 1e-8).all()


@pytest.mark.parametrize("engine", ["streaming", "resident"])
def test_async_tolerates_a_slow_block(engine):
    """Section 5: asynchronous block Jacobi keeps progressing when one block is slow."""
    n = 24
    c = inputs.equal_cuts(n, 2)
    bnd = inputs.boundary_uniform(n, n, n, 1, 32)
    g = make_grid(n, n, n, 1, c, c, c)
    x, st = g.solve(bnd=cuda(bnd), precision="mixed", mode="async", slow_block=3, slow_ns=200_000, engine=engine)
    assert st.status == 0 and st.rel_residual < 1e-8


def test_async_time_limit_returns_timeout():
    n = 32
    c = inputs.equal_cuts(n, 4)
    bnd = inputs.boundary_uniform(n, n, n, 1, 33)
    g = make_grid(n, n, n, 1, c, c, c)
    x, st = g.solve(bnd=cuda(bnd), precision="fp64", mode="async", outer_tol=1e-14, time_limit_ms=20.0,
                    slow_block=0, slow_ns=1_000_000)
    assert st.status == 5
    assert np.isfinite(x.cpu().numpy()).all()


def test_persistent_wait_budget_runs_out_returns_timeout():
    """Failure detection by bounded device waits (section 5: progress despite
    slow cores): in the persistent synchronous launch a cluster waits for its
    neighbours' progress flags and for each sweep's stop decision.  One block
    made slow (1 ms per task) and a budget of 4 polls make such a wait run out:
    the solve must end with MS_ERR_TIMEOUT promptly (every other cluster leaves
    its own wait), with x the last complete iterate -- finite, and with the true
    residual the stats report.  The default budget rides out the same slow block."""
    import time
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    b = cuda(cfg["bnd"])
    shape = dict(cluster=4, threads=512, precision="mixed", engine="resident", persistent=True)
    t0 = time.perf_counter()
    x, st = g.solve(bnd=b, slow_block=5, slow_ns=1_000_000, wait_polls=4, **shape)
    elapsed = time.perf_counter() - t0
    assert st.status == 5
    assert elapsed < 20.0
    xh = x.cpu().numpy()
    assert np.isfinite(xh).all()
    assert g.residual(x, bnd=b)[0] == pytest.approx(st.rel_residual, rel=1e-12)
    x2, s2 = g.solve(bnd=b, slow_block=5, slow_ns=100_000, **shape)
    assert s2.status == 0 and s2.rel_residual < 1e-8


@pytest.mark.parametrize("mode,persistent", [("sync", False), ("sync", True), ("async", False)])
def test_tagged_sum_wait_runs_out_returns_timeout(mode, persistent):
    """The resident CG forms p.Ap without a cluster barrier: each CTA polls for
    the other CTAs' tagged totals, a wait bounded by opts.sum_polls.  With a
    budget of one poll the wait runs out (a total takes far longer than one
    poll to arrive from another SM): the solve must end by itself with
    MS_ERR_TIMEOUT in every launch form (no CTA leaves the CG loop or a
    cluster barrier out of step with the others), and the GPU stays usable --
    the same solve with the default budget converges."""
    import time
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    b = cuda(cfg["bnd"])
    shape = dict(cluster=4, threads=512, precision="mixed", engine="resident", mode=mode, persistent=persistent)
    t0 = time.perf_counter()
    x, st = g.solve(bnd=b, sum_polls=1, outer_maxit=20, outer_tol=0.0, **shape)
    assert time.perf_counter() - t0 < 30.0
    assert st.status == 5
    x2, s2 = g.solve(bnd=b, **shape)
    assert s2.status == 0 and s2.rel_residual < 1e-8
    assert g.residual(x2, bnd=b)[0] < 1e-8


def test_sync_time_limit_returns_timeout():
    n = 32
    c = inputs.equal_cuts(n, 4)
    bnd = inputs.boundary_uniform(n, n, n, 1, 34)
    g = make_grid(n, n, n, 1, c, c, c)
    x, st = g.solve(bnd=cuda(bnd), precision="fp64", outer_tol=1e-15, time_limit_ms=5.0, check_every=1)
    assert st.status == 5
    # the returned iterate is a complete sweep: its true residual is what the stats say
    assert g.residual(x, bnd=cuda(bnd))[0] == pytest.approx(st.rel_residual, rel=1e-12)


# ---------------------------------------------------------------- on-chip (resident) engine
RES_CASES = [
    (32, 32, 32, [0, 16, 32], [0, 16, 32], [0, 16, 32]),
    (37, 29, 23, [0, 13, 37], [0, 10, 20, 29], [0, 11, 23]),            # ragged strips and slabs
    (64, 64, 64, [0, 64], [0, 64], [0, 64]),                             # one 64^3 block
    (21, 19, 40, [0, 5, 21], [0, 1, 19], [0, 9, 40]),                     # 1-wide rows
]


@pytest.mark.parametrize("case", RES_CASES)
@pytest.mark.parametrize("engine,threads", [("resident", 0), ("streaming", 512), ("streaming", 1024),
                                            ("streaming", 256)])
def test_mixed_one_sweep_close_to_oracle(case, engine, threads):
    """One sweep from x0 = 0 is one FP32 CG solve per block: it must match the
    FP64 oracle's sweep to FP32-CG accuracy.  Streaming with 512/1024 threads
    is the vectorised strip engine, with 256 the scalar one."""
    nx, ny, nz, cx, cy, cz = case
    bnd = np.random.default_rng(50).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make_grid(nx, ny, nz, 1, cx, cy, cz)
    x, st = g.solve(bnd=cuda(bnd), precision="mixed", engine=engine, threads=threads, outer_tol=0.0, outer_maxit=1)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], outer_tol=0.0, outer_maxit=1)
    assert st.outer_its == 1
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 2e-4
    assert st.inner_its == ref["inner_its"] or abs(st.inner_its - ref["inner_its"]) <= 2 * len(cx) * len(cy) * len(cz)


def resident_vs_streaming(case, cluster=0, persistent=True):
    nx, ny, nz, cx, cy, cz = case
    bnd = np.random.default_rng(51).uniform(-1, 1, size=(2, inputs.boundary_size(nx, ny, nz)))
    g = make_grid(nx, ny, nz, 2, cx, cy, cz)
    xr, sr = g.solve(bnd=cuda(bnd), precision="mixed", engine="resident", cluster=cluster, persistent=persistent)
    xs, ss = g.solve(bnd=cuda(bnd), precision="mixed", engine="streaming")
    assert sr.status == 0 and max(sr.per_rhs_rel) < 1e-8
    assert (g.residual(xr, bnd=cuda(bnd)) < 1e-8).all()
    assert abs(sr.outer_its - ss.outer_its) <= max(2, ss.outer_its // 50)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[1])
    kappa = 0.5 * (max(nx, ny, nz) + 1) ** 2
    assert rel_inf(xr.cpu().numpy()[1], ref["x"]) <= 2 * kappa * 1e-8


@pytest.mark.parametrize("case", RES_CASES)
@pytest.mark.parametrize("persistent", [True, False])
def test_resident_converges_like_streaming(case, persistent):
    resident_vs_streaming(case, 0, persistent)


@pytest.mark.parametrize("cluster", [2, 4, 8, 16])
def test_resident_cluster_sizes(cluster):
    resident_vs_streaming(RES_CASES[0], cluster)


@pytest.mark.parametrize("magnitude", [1e-30, 1e30])
@pytest.mark.parametrize("engine", ["resident", "streaming"])
def test_mixed_is_scale_invariant(magnitude, engine):
    """The FP32 inner solve works on the residual scaled by a power of two near
    1/||bhat||, so data of any magnitude converges exactly like O(1) data."""
    n = 24
    c = inputs.equal_cuts(n, 2)
    bnd = np.random.default_rng(53).uniform(-1, 1, size=(1, inputs.boundary_size(n, n, n)))
    g = make_grid(n, n, n, 1, c, c, c)
    x1, s1 = g.solve(bnd=cuda(bnd), precision="mixed", engine=engine)
    xm, sm = g.solve(bnd=cuda(bnd * magnitude), precision="mixed", engine=engine)
    assert s1.status == 0 and sm.status == 0 and sm.rel_residual < 1e-8
    assert abs(sm.outer_its - s1.outer_its) <= 1
    assert rel_inf(xm.cpu().numpy() / magnitude, x1.cpu().numpy()) <= 2 * 0.5 * (n + 1) ** 2 * 1e-8


@pytest.mark.parametrize("persistent", [True, False])
def test_resident_persistent_and_per_sweep_agree(persistent):
    """The persistent dataflow launch runs exactly the strict-Jacobi sweeps of
    the per-sweep launches: same sweeps, same inner iterations, same x."""
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    b = cuda(cfg["bnd"])
    shape = dict(cluster=4, threads=512)  # one explicit shape: no tuning sweeps in either run
    x1, s1 = g.solve(bnd=b, precision="mixed", engine="resident", persistent=True, outer_tol=0.0, outer_maxit=25,
                     **shape)
    x2, s2 = g.solve(bnd=b, precision="mixed", engine="resident", persistent=False, outer_tol=0.0, outer_maxit=25,
                     **shape)
    assert s1.outer_its == s2.outer_its == 25 and s1.inner_its == s2.inner_its
    np.testing.assert_array_equal(x1.cpu().numpy(), x2.cpu().numpy())
    xc, sc = g.solve(bnd=b, precision="mixed", engine="resident", persistent=persistent, history=True)
    assert sc.status == 0 and sc.rel_residual < 1e-8


@pytest.mark.parametrize("case", RES_CASES[:2] + RES_CASES[3:])
def test_resident_q_in_registers_is_bit_identical(case):
    """Keeping q = A p in registers (one stencil per CG iteration) and moving
    d += alpha p to the next pass performs the same FMAs in the same order as
    recomputing the stencil: every layout and its q-in-registers twin give
    the same iterates bit for bit, sweep after sweep."""
    from paper_2009_12638_gb300 import resident_variants
    nx, ny, nz, cx, cy, cz = case
    bnd = np.random.default_rng(54).uniform(-1, 1, size=(2, inputs.boundary_size(nx, ny, nz)))
    g = make_grid(nx, ny, nz, 2, cx, cy, cz)
    rows = resident_variants()
    key = lambda r: (r["threads"], r["strips"], r["planes"], r["d_smem"])  # noqa: E731
    plain = {key(r): v for v, r in enumerate(rows) if not r["q_regs"] and not r["one_reduction"]}
    compared = 0
    for w, r in enumerate(rows):
        if not r["q_regs"]:
            continue
        v = plain[key(r)]
        res = []
        for var in (v, w):
            try:
                x, st = g.solve(bnd=cuda(bnd), precision="mixed", variant=var, persistent=False, outer_tol=0.0,
                                outer_maxit=4)
            except MsError:
                break  # this layout does not fit the blocks
            assert st.variant == var and st.outer_its == 4
            res.append((x.cpu().numpy(), st.inner_its))
        if len(res) == 2:
            np.testing.assert_array_equal(res[0][0], res[1][0])
            assert res[0][1] == res[1][1]
            compared += 1
    assert compared >= 2


def test_resident_uneven_multi_rhs():
    cfg = inputs.make_config("batched_uneven", scale=4)
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 4, cfg["cx"], cfg["cy"], cfg["cz"])
    x, st = g.solve(bnd=cuda(cfg["bnd"][:4]), precision="mixed", engine="resident")
    assert st.status == 0 and max(st.per_rhs_rel) < 1e-8


def test_resident_refuses_blocks_that_do_not_fit():
    g = make_grid(8, 8, 3, 1, [0, 8], [0, 8], [0, 3])  # bz = 3 < any cluster of 4: still fits with c <= 3
    bnd = np.random.default_rng(52).uniform(-1, 1, size=(1, g.nbnd))
    x, st = g.solve(bnd=cuda(bnd), precision="mixed", engine="resident")
    assert st.status == 0
    big = make_grid(200, 200, 8, 1, [0, 200], [0, 200], [0, 8])  # 50x200 strips per plane: too many
    with pytest.raises(Exception):
        big.solve(bnd=torch.zeros(1, big.nbnd, dtype=torch.float64, device="cuda"), precision="mixed",
                  engine="resident", outer_maxit=1)


@pytest.mark.parametrize("persistent", [True, False])
def test_residual_versus_time_history(persistent):
    """history=True records rho_k and the device time of its stop test
    (measured from the first one): the residual-versus-time curve."""
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    x, st = g.solve(bnd=cuda(cfg["bnd"]), precision="mixed", engine="resident", persistent=persistent, history=True)
    k = st.outer_its
    t = st.history_ms[: k + 1]
    h = st.history[0][: k + 1]
    assert st.status == 0 and h[-1] < 1e-8 <= h[-2]
    assert t[0] == 0.0 and (np.diff(t) >= 0.0).all() and t[-1] > 0.0
    assert t[-1] <= st.time_ms
