"""GPU tests of the one-sweep entry points (ms_sweep, ms_norms) and of the
block-Jacobi split over shards (paper sections 3 and 4.1), run as several
shards in one process on one GPU (LocalComm: the same sweeps, plane swaps and
sums as one rank per GPU, without a process group)."""
import numpy as np
import pytest
import torch

from paper_2009_12638_gb300 import Grid, inputs
from paper_2009_12638_gb300.shard import solve_local

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def grid_for(nx, ny, nz, nrhs, cx, cy, cz):
    return Grid(nx, ny, nz, nrhs).partition(len(cx) - 1, len(cy) - 1, len(cz) - 1, cx, cy, cz)


CASE = dict(nx=37, ny=29, nz=23, cx=[0, 13, 25, 37], cy=[0, 10, 20, 29], cz=[0, 11, 23])


def test_norms_match_residual_and_oracle(oracle_mod):
    c = CASE
    nrhs = 2
    g = grid_for(c["nx"], c["ny"], c["nz"], nrhs, c["cx"], c["cy"], c["cz"])
    rng = np.random.default_rng(80)
    bnd = rng.uniform(-1, 1, (nrhs, inputs.boundary_size(c["nx"], c["ny"], c["nz"])))
    f = rng.standard_normal((nrhs, c["nz"], c["ny"], c["nx"]))
    x = rng.standard_normal((nrhs, c["nz"], c["ny"], c["nx"]))
    rr, bb = g.norms(cuda(x), f=cuda(f), bnd=cuda(bnd))
    rr, bb = rr.cpu().numpy(), bb.cpu().numpy()
    np.testing.assert_allclose(np.sqrt(rr / bb), g.residual(cuda(x), f=cuda(f), bnd=cuda(bnd)), rtol=1e-14)
    for s in range(nrhs):
        bh = oracle_mod.lift(c["nx"], c["ny"], c["nz"], f[s], bnd[s])
        r = oracle_mod.residual(bh, x[s])
        assert rr[s] == pytest.approx(np.sum(r * r), rel=1e-12)
        assert bb[s] == pytest.approx(np.sum(bh * bh), rel=1e-12)


@pytest.mark.parametrize("precision,engine,shape", [("fp64", "streaming", dict(cluster=4, threads=256)),
                                                     ("mixed", "streaming", dict(cluster=4, threads=512)),
                                                     ("mixed", "resident", dict(cluster=4, threads=512))])
def test_sweep_equals_one_sweep_of_solve(precision, engine, shape):
    """ms_sweep runs the sweep kernel ms_solve runs: with the same launch shape
    the result is bit-identical to a solve stopped after one sweep, and rr is
    the squared residual of x^k."""
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = grid_for(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    b = cuda(cfg["bnd"])
    rng = np.random.default_rng(81)
    x0 = cuda(rng.standard_normal(g.shape) * 0.1)
    opts = dict(precision=precision, engine=engine, **shape)
    x1, st = g.solve(bnd=b, x0=x0, outer_tol=0.0, outer_maxit=1, **opts)
    xo = torch.empty_like(x0)
    rr, sst = g.sweep(x0, xo, bnd=b, stats=True, **opts)
    assert (sst.cluster, sst.threads) == (st.cluster, st.threads) and sst.variant == st.variant
    assert sst.inner_its == st.inner_its
    assert torch.equal(xo, x1)
    rr0, bb0 = g.norms(x0, bnd=b)
    # the sweep sums its block partials, ms_norms its own per-CTA sums: same value, other order
    np.testing.assert_allclose(rr.cpu().numpy(), rr0.cpu().numpy(), rtol=1e-12)
    assert sst.rel_residual == pytest.approx(float(np.sqrt(rr0[0].item() / bb0[0].item())), rel=1e-12)


@pytest.mark.parametrize("dims", [(37, 29, 23), (1, 5, 7), (2, 2, 9), (6, 1, 1), (3, 4, 2)])
@pytest.mark.parametrize("with_f", [False, True])
def test_sweep_bhat_norm_matches_the_full_pass(dims, with_f):
    """ms_sweep forms ||bhat|| visiting only the points next to the boundary when
    f is null (every shell point once, edges and corners included): its
    relative residual equals ms_residual's on thin and degenerate grids too."""
    nx, ny, nz = dims
    g = grid_for(nx, ny, nz, 2, [0, nx], [0, ny], [0, nz])
    rng = np.random.default_rng(83)
    bnd = cuda(rng.uniform(-1, 1, (2, inputs.boundary_size(nx, ny, nz))))
    f = cuda(rng.standard_normal((2, nz, ny, nx))) if with_f else None
    x0 = cuda(rng.standard_normal((2, nz, ny, nx)))
    rr, st = g.sweep(x0, torch.empty_like(x0), f=f, bnd=bnd, stats=True, precision="fp64")
    want = g.residual(x0, f=f, bnd=bnd)
    assert st.rel_residual == pytest.approx(want.max(), rel=1e-12)


def test_sweep_rejects_aliasing_and_async():
    g = grid_for(8, 8, 8, 1, [0, 4, 8], [0, 8], [0, 8])
    x = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        g.sweep(x, x)
    with pytest.raises(Exception):
        g.sweep(x, torch.empty_like(x), mode="async")


@pytest.mark.parametrize("ranks", [(2, 1, 1), (1, 2, 2), (3, 3, 2)])
def test_local_shards_sweep_like_the_oracle(oracle_mod, ranks):
    c = CASE
    nrhs = 2
    rng = np.random.default_rng(82)
    bnd = rng.uniform(-1, 1, (nrhs, inputs.boundary_size(c["nx"], c["ny"], c["nz"])))
    for K in (1, 3):
        x, st = solve_local(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], ranks, bnd=cuda(bnd),
                            precision="fp64", outer_tol=0.0, outer_maxit=K)
        assert st.outer_its == K
        xh = x.cpu().numpy()
        for s in range(nrhs):
            ref = oracle_mod.solve(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], bnd=bnd[s], outer_tol=0.0,
                                   outer_maxit=K)
            np.testing.assert_allclose(xh[s], ref["x"], rtol=0, atol=1e-11 * np.abs(ref["x"]).max())


def test_local_shards_converge_like_the_oracle(oracle_mod):
    cfg = inputs.make_config("laplace32_linear")
    n = cfg["nx"]
    x, st = solve_local(n, n, n, cfg["cx"], cfg["cy"], cfg["cz"], (2, 1, 2), bnd=cuda(cfg["bnd"]),
                        precision="fp64", outer_tol=1e-10)
    ref = oracle_mod.solve(n, n, n, cfg["cx"], cfg["cy"], cfg["cz"], bnd=cfg["bnd"][0], outer_tol=1e-10)
    assert st.status == 0 and abs(st.outer_its - ref["outer_its"]) <= 1
    xh = x.cpu().numpy()[0]
    assert np.abs(xh - ref["x"]).max() <= 1e-9 * np.abs(ref["x"]).max()
    # discretely harmonic data: the converged solution is the closed form within kappa * tol
    assert np.abs(xh - cfg["exact"][0]).max() <= 0.5 * (n + 1) ** 2 * 1e-10 * np.abs(cfg["exact"]).max()


def test_local_shards_mixed_match_the_single_grid_solve():
    """Mixed precision: the shards' sweeps are the single grid's up to the
    summation order at shard faces, so the same sweep count (+-1) and the
    same converged accuracy."""
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = grid_for(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    b = cuda(cfg["bnd"])
    x1, s1 = g.solve(bnd=b, precision="mixed")
    x, st = solve_local(cfg["nx"], cfg["ny"], cfg["nz"], cfg["cx"], cfg["cy"], cfg["cz"], (2, 2, 1), bnd=b,
                        precision="mixed")
    assert s1.status == 0 and st.status == 0
    assert abs(st.outer_its - s1.outer_its) <= 1
    assert st.rel_residual < 1e-8
    assert g.residual(x, bnd=b)[0] == pytest.approx(st.rel_residual, rel=1e-6)
    n = cfg["nx"]
    assert (x - x1).abs().max().item() <= 2 * 0.5 * (n + 1) ** 2 * 1e-8 * x1.abs().max().item()


# ---------------------------------------------------------------- two processes, torch.distributed
def _dist_rank(rank, world, port, ranks, out):
    import os

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2009_12638_gb300.shard import solve_distributed
        cfg = inputs.make_config("laplace32_linear")
        n = cfg["nx"]
        x, st = solve_distributed(n, n, n, cfg["cx"], cfg["cy"], cfg["cz"], ranks, bnd=cuda(cfg["bnd"]),
                                  precision="fp64", outer_tol=1e-10)
        out[rank] = (x.cpu().numpy(), st.status, st.outer_its, st.rel_residual)
    finally:
        dist.destroy_process_group()


def test_two_processes_solve_distributed_over_gloo(oracle_mod):
    """solve_distributed end to end with the GPU shards: two processes (one
    shard each, both on this GPU, exchanging through gloo and host memory --
    their kernels never wait on one another) give the oracle's solution."""
    import socket

    import torch.multiprocessing as mp
    from paper_2009_12638_gb300.shard import ShardLayout
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ranks = (1, 1, 2)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_dist_rank, args=(r, 2, port, ranks, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
        assert p.exitcode == 0
    cfg = inputs.make_config("laplace32_linear")
    n = cfg["nx"]
    lay = ShardLayout(n, n, n, cfg["cx"], cfg["cy"], cfg["cz"], ranks)
    x = np.empty((1, n, n, n))
    for r in range(2):
        (x0, x1), (y0, y1), (z0, z1) = lay.box(r)
        x[:, z0:z1, y0:y1, x0:x1] = out[r][0]
    assert out[0][1:3] == out[1][1:3] and out[0][1] == 0
    ref = oracle_mod.solve(n, n, n, cfg["cx"], cfg["cy"], cfg["cz"], bnd=cfg["bnd"][0], outer_tol=1e-10)
    assert abs(out[0][2] - ref["outer_its"]) <= 1
    assert np.abs(x[0] - ref["x"]).max() <= 1e-9 * np.abs(ref["x"]).max()
    assert out[0][3] < 1e-10
