"""The multi-GPU split of block Jacobi (paper sections 3 and 4.1: groups of
blocks per process, point-to-point boundary swaps, the global residual as a
sum of per-group shares), tested on the CPU.

The host logic (which rank owns which blocks, which planes go where, the
outer loop and stop rule of ``sharded_solve``) is the library's own; the
per-rank compute is the FP64 oracle here (a stand-in with the same three
methods as the GPU shard), so the sharded iterates must equal the unsharded
oracle's sweep for sweep.  Ranks run in one process (LocalComm) or as two
gloo processes (DistComm, the torch.distributed path the GPUs use with NCCL).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2009_12638_gb300 import inputs
from paper_2009_12638_gb300.shard import (DistComm, LocalComm, ShardLayout, face_layout, sharded_solve)


class OracleShard:
    """One rank's sub-grid computed by the FP64 CPU oracle (test stand-in for GridShard)."""

    def __init__(self, layout, rank, nrhs, inner_rtol=1e-6, inner_maxit=50):
        import oracle
        self.oracle = oracle
        self.rank = rank
        self.nrhs = nrhs
        self.dims = layout.dims(rank)
        self.cuts = layout.local_cuts(rank)
        self.device = torch.device("cpu")
        self.inner = (inner_rtol, inner_maxit)

    def face_planes(self, x):
        lx, ly, lz = self.dims
        lay = face_layout(lx, ly, lz)
        out = torch.empty((self.nrhs, lay[-1][0] + lx * ly), dtype=torch.float64)
        planes = [x[:, :, :, 0], x[:, :, :, -1], x[:, :, 0, :], x[:, :, -1, :], x[:, 0, :, :], x[:, -1, :, :]]
        for (off, shp), p in zip(lay, planes):
            out[:, off:off + shp[0] * shp[1]] = p.reshape(self.nrhs, -1)
        return out

    def sweep(self, x_in, x_out, f, bnd, opts):
        lx, ly, lz = self.dims
        for s in range(self.nrhs):
            r = self.oracle.solve(lx, ly, lz, *self.cuts, f=None if f is None else f[s].numpy(),
                                  bnd=bnd[s].numpy(), x0=x_in[s].numpy(), inner_rtol=opts.get("inner_rtol", 1e-6),
                                  inner_maxit=opts.get("inner_maxit", 50), outer_tol=0.0, outer_maxit=1)
            x_out[s] = torch.from_numpy(r["x"])
        return self.norms(x_in, f, bnd)[0]

    def norms(self, x, f, bnd):
        lx, ly, lz = self.dims
        rr = torch.empty(self.nrhs, dtype=torch.float64)
        bb = torch.empty(self.nrhs, dtype=torch.float64)
        for s in range(self.nrhs):
            bh = self.oracle.lift(lx, ly, lz, None if f is None else f[s].numpy(), bnd[s].numpy())
            r = self.oracle.residual(bh, x[s].numpy())
            rr[s] = float(np.sum(r * r))
            bb[s] = float(np.sum(bh * bh))
        return rr, bb


def assemble(layout, parts, nrhs):
    nx, ny, nz = layout.n
    x = torch.empty((nrhs, nz, ny, nx), dtype=torch.float64)
    for r, p in enumerate(parts):
        layout.local_field(r, x).copy_(p)
    return x


CASE = dict(nx=14, ny=11, nz=9, cx=[0, 4, 7, 11, 14], cy=[0, 3, 7, 11], cz=[0, 5, 9])


def problem(nrhs=2, seed=70):
    c = CASE
    bnd = inputs.boundary_uniform(c["nx"], c["ny"], c["nz"], nrhs, seed)
    f = np.random.default_rng(seed + 1).standard_normal((nrhs, c["nz"], c["ny"], c["nx"]))
    return torch.from_numpy(bnd), torch.from_numpy(f)


# ---------------------------------------------------------------- layout
@pytest.mark.parametrize("ranks", [(1, 1, 1), (2, 1, 1), (2, 3, 2), (4, 3, 2), (3, 2, 1)])
def test_layout_tiles_the_grid_with_whole_blocks(ranks):
    c = CASE
    lay = ShardLayout(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], ranks)
    owner = np.full((c["nz"], c["ny"], c["nx"]), -1)
    for r in range(lay.size):
        (x0, x1), (y0, y1), (z0, z1) = lay.box(r)
        assert (owner[z0:z1, y0:y1, x0:x1] == -1).all()
        owner[z0:z1, y0:y1, x0:x1] = r
        # the local cuts are whole global blocks, shifted to the sub-grid
        for a, (lo, hi), cut in zip(range(3), lay.box(r), (c["cx"], c["cy"], c["cz"])):
            lc = lay.local_cuts(r)[a]
            assert lc[0] == 0 and lc[-1] == hi - lo
            assert set(v + lo for v in lc) <= set(cut)
        for f in range(6):
            nb = lay.neighbour(r, f)
            if nb >= 0:
                assert lay.neighbour(nb, f ^ 1) == r
                # neighbours share the whole cross-section of the face
                a = f // 2
                assert [lay.box(r)[b] for b in range(3) if b != a] == [lay.box(nb)[b] for b in range(3) if b != a]
    assert (owner >= 0).all()


def test_layout_rejects_more_ranks_than_blocks():
    with pytest.raises(ValueError):
        ShardLayout(8, 8, 8, [0, 4, 8], [0, 8], [0, 8], (3, 1, 1))


def test_local_boundary_keeps_domain_faces_and_zeroes_internal_ones():
    c = CASE
    lay = ShardLayout(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], (2, 2, 1))
    bnd, _ = problem(1)
    glob = face_layout(c["nx"], c["ny"], c["nz"])
    for r in range(lay.size):
        lb = lay.local_boundary(r, bnd)
        (x0, x1), (y0, y1), (z0, z1) = lay.box(r)
        loc = face_layout(*lay.dims(r))
        for f in range(6):
            lo, ls = loc[f]
            got = lb[0, lo:lo + ls[0] * ls[1]].reshape(ls)
            if lay.neighbour(r, f) >= 0:
                assert not got.any()
                continue
            go, gs = glob[f]
            g = bnd[0, go:go + gs[0] * gs[1]].reshape(gs)
            want = [g[z0:z1, y0:y1]] * 2 + [g[z0:z1, x0:x1]] * 2 + [g[y0:y1, x0:x1]] * 2
            np.testing.assert_array_equal(got, want[f])


# ---------------------------------------------------------------- sweeps vs the unsharded oracle
@pytest.mark.parametrize("ranks", [(2, 1, 1), (1, 3, 1), (2, 2, 2), (4, 1, 2)])
def test_local_shards_sweep_like_the_whole_grid(oracle_mod, ranks):
    c = CASE
    nrhs = 2
    bnd, f = problem(nrhs)
    lay = ShardLayout(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], ranks)
    shards = [OracleShard(lay, r, nrhs) for r in range(lay.size)]
    for K in (1, 2, 3):
        parts, st = sharded_solve(lay, shards, LocalComm(lay), bnd=bnd, f=f, outer_tol=0.0, outer_maxit=K)
        assert st.outer_its == K and st.status == 4
        x = assemble(lay, parts, nrhs).numpy()
        for s in range(nrhs):
            ref = oracle_mod.solve(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], f=f[s].numpy(),
                                   bnd=bnd[s].numpy(), outer_tol=0.0, outer_maxit=K)
            np.testing.assert_allclose(x[s], ref["x"], rtol=0, atol=1e-11 * np.abs(ref["x"]).max())


def test_local_shards_converge_like_the_whole_grid(oracle_mod):
    c = CASE
    nrhs = 2
    bnd, f = problem(nrhs, seed=71)
    lay = ShardLayout(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], (2, 3, 1))
    shards = [OracleShard(lay, r, nrhs) for r in range(lay.size)]
    parts, st = sharded_solve(lay, shards, LocalComm(lay), bnd=bnd, f=f, outer_tol=1e-8, history=True)
    assert st.status == 0
    x = assemble(lay, parts, nrhs).numpy()
    for s in range(nrhs):
        ref = oracle_mod.solve(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], f=f[s].numpy(),
                               bnd=bnd[s].numpy(), outer_tol=1e-8, history=True)
        assert st.per_rhs_outer_its[s] == ref["outer_its"]
        np.testing.assert_allclose(x[s], ref["x"], rtol=0, atol=1e-11 * np.abs(ref["x"]).max())
        # relative residuals (of ||bhat|| = O(1)): the shard faces sum the same terms in another order
        np.testing.assert_allclose([h[s] for h in st.history[:ref["outer_its"] + 1]], ref["history"], rtol=1e-9,
                                   atol=1e-14)
        assert st.per_rhs_rel[s] == pytest.approx(ref["rel_residual"], rel=1e-9)


def test_overlap_and_async_are_rejected_across_ranks(oracle_mod):
    c = CASE
    lay = ShardLayout(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], (2, 1, 1))
    shards = [OracleShard(lay, r, 1) for r in range(lay.size)]
    bnd, _ = problem(1)
    with pytest.raises(ValueError):
        sharded_solve(lay, shards, LocalComm(lay), bnd=bnd, overlap=2)
    with pytest.raises(ValueError):
        sharded_solve(lay, shards, LocalComm(lay), bnd=bnd, mode="async")


def test_zero_data_stops_at_k0(oracle_mod):
    c = CASE
    lay = ShardLayout(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], (2, 1, 1))
    shards = [OracleShard(lay, r, 1) for r in range(lay.size)]
    parts, st = sharded_solve(lay, shards, LocalComm(lay), bnd=torch.zeros(1, inputs.boundary_size(
        c["nx"], c["ny"], c["nz"]), dtype=torch.float64), outer_tol=1e-8)
    assert st.status == 0 and st.outer_its == 0
    assert not any(p.any() for p in parts)


# ---------------------------------------------------------------- two gloo ranks (the torch.distributed path)
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ranks, K, tol, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = CASE
        nrhs = 2
        bnd, f = problem(nrhs)
        lay = ShardLayout(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], ranks)
        shard = OracleShard(lay, rank, nrhs)
        parts, st = sharded_solve(lay, [shard], DistComm(lay), bnd=bnd, f=f, outer_tol=tol, outer_maxit=K)
        out[rank] = (parts[0].numpy(), st.outer_its, st.per_rhs_outer_its, st.rel_residual)
    finally:
        dist.destroy_process_group()


def _run_ranks(ranks, K, tol):
    world = ranks[0] * ranks[1] * ranks[2]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, ranks, K, tol, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return dict(out)


@pytest.mark.parametrize("ranks", [(2, 1, 1), (1, 1, 2)])
def test_two_gloo_ranks_sweep_like_the_whole_grid(oracle_mod, ranks):
    c = CASE
    nrhs = 2
    bnd, f = problem(nrhs)
    lay = ShardLayout(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], ranks)
    out = _run_ranks(ranks, 3, 0.0)
    x = assemble(lay, [torch.from_numpy(out[r][0]) for r in range(2)], nrhs).numpy()
    assert out[0][1] == out[1][1] == 3
    for s in range(nrhs):
        ref = oracle_mod.solve(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], f=f[s].numpy(),
                               bnd=bnd[s].numpy(), outer_tol=0.0, outer_maxit=3)
        np.testing.assert_allclose(x[s], ref["x"], rtol=0, atol=1e-11 * np.abs(ref["x"]).max())


def test_two_gloo_ranks_converge_like_the_whole_grid(oracle_mod):
    c = CASE
    nrhs = 2
    bnd, f = problem(nrhs)
    lay = ShardLayout(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], (2, 1, 1))
    out = _run_ranks((2, 1, 1), 100000, 1e-8)
    x = assemble(lay, [torch.from_numpy(out[r][0]) for r in range(2)], nrhs).numpy()
    assert out[0][2] == out[1][2]  # both ranks take the same stop decisions
    for s in range(nrhs):
        ref = oracle_mod.solve(c["nx"], c["ny"], c["nz"], c["cx"], c["cy"], c["cz"], f=f[s].numpy(),
                               bnd=bnd[s].numpy(), outer_tol=1e-8)
        assert out[0][2][s] == ref["outer_its"]
        np.testing.assert_allclose(x[s], ref["x"], rtol=0, atol=1e-11 * np.abs(ref["x"]).max())
    assert out[0][3] < 1e-8
