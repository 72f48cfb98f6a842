"""Block Jacobi split over several GPUs: one rank per GPU, each holding a
contiguous sub-array of blocks.

Paper sections 3 and 4.1: every group of processes solves its blocks, swaps
boundary values point to point with the groups next to it (no master
process), and the global residual is a sum of per-group partial sums.  Here a
rank's sub-array of blocks is a grid of its own (a ``Grid`` handle of the CUDA
library); the values of the neighbouring ranks next to it are the Dirichlet
data of its internal faces.  A rank's sub-grid with that boundary data has
exactly the block rows of the global system -- the couplings A_ij x_j to
blocks on other ranks move to the right-hand side, as in the section 3
update X_i = A_ii^{-1}(B_i - sum_j A_ij X_j) -- so a sharded sweep is a sweep
of the whole grid.

One synchronous sweep k, on every rank:

1. gather the six boundary planes of its x^k in the packed face layout
   (``ms_face_gather``);
2. swap planes with the face neighbours: each plane is sent to the rank on
   that side and received straight into the receiving rank's own boundary
   array (the slot of the opposite face);
3. one sweep of its blocks (``ms_sweep``): x^{k+1}, and its share of
   ||bhat - A x^k||^2;
4. add the shares over ranks (one FP64 all-reduce of nrhs values) and apply
   the stop rule of section 2.1 to x^k, per rhs.

``DistComm`` does steps 2 and 4 with torch.distributed (NCCL between GPUs,
gloo on the CPU); ``LocalComm`` runs several shards in one process (copies
between the shards' own buffers).  The compute of steps 1 and 3 is the
shard's backend: ``GridShard`` drives the CUDA library; anything with the same
three methods (``face_planes``, ``sweep``, ``norms``) can stand in for it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

FACES = ("x-", "x+", "y-", "y+", "z-", "z+")
OPPOSITE = (1, 0, 3, 2, 5, 4)


def face_layout(nx: int, ny: int, nz: int):
    """(offset, shape) of the six faces in one rhs's packed boundary array:
    x-, x+ (nz, ny); y-, y+ (nz, nx); z-, z+ (ny, nx)."""
    shapes = [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]
    out, off = [], 0
    for s in shapes:
        out.append((off, s))
        off += s[0] * s[1]
    return out


def _split(n: int, parts: int):
    """Equal split of n items into parts, remainder to the leading parts."""
    q, r = divmod(n, parts)
    c = [0]
    for a in range(parts):
        c.append(c[-1] + q + (1 if a < r else 0))
    return c


class ShardLayout:
    """The block partition (cut arrays cx, cy, cz of an nx*ny*nz grid) split
    into a tensor grid of ranks rx*ry*rz: rank (qx, qy, qz), id
    qx + rx*(qy + ry*qz), owns a contiguous sub-array of blocks (block counts
    per axis split evenly, remainder to the leading ranks).  Host logic only."""

    def __init__(self, nx, ny, nz, cx, cy, cz, ranks):
        self.n = (int(nx), int(ny), int(nz))
        self.cuts = tuple(np.asarray(c, dtype=np.int64) for c in (cx, cy, cz))
        for n, c in zip(self.n, self.cuts):
            if c[0] != 0 or c[-1] != n or np.any(np.diff(c) < 1):
                raise ValueError("cut arrays must increase strictly from 0 to the grid size")
        self.ranks = tuple(int(r) for r in ranks)
        if len(self.ranks) != 3 or min(self.ranks) < 1:
            raise ValueError("ranks must be three positive counts (rx, ry, rz)")
        self.block_split = []
        for c, r in zip(self.cuts, self.ranks):
            nb = len(c) - 1
            if r > nb:
                raise ValueError(f"{r} ranks along an axis with only {nb} blocks")
            self.block_split.append(_split(nb, r))

    @property
    def size(self) -> int:
        return self.ranks[0] * self.ranks[1] * self.ranks[2]

    def coords(self, rank: int):
        rx, ry, _ = self.ranks
        return rank % rx, (rank // rx) % ry, rank // (rx * ry)

    def rank_of(self, q):
        rx, ry, rz = self.ranks
        if not (0 <= q[0] < rx and 0 <= q[1] < ry and 0 <= q[2] < rz):
            return -1
        return q[0] + rx * (q[1] + ry * q[2])

    def box(self, rank: int):
        """Point ranges ((x0, x1), (y0, y1), (z0, z1)) the rank owns."""
        q = self.coords(rank)
        out = []
        for a in range(3):
            b0, b1 = self.block_split[a][q[a]], self.block_split[a][q[a] + 1]
            out.append((int(self.cuts[a][b0]), int(self.cuts[a][b1])))
        return tuple(out)

    def dims(self, rank: int):
        (x0, x1), (y0, y1), (z0, z1) = self.box(rank)
        return x1 - x0, y1 - y0, z1 - z0

    def local_cuts(self, rank: int):
        """The rank's block cut arrays, relative to its own sub-grid."""
        q = self.coords(rank)
        out = []
        for a in range(3):
            b0, b1 = self.block_split[a][q[a]], self.block_split[a][q[a] + 1]
            c = self.cuts[a][b0:b1 + 1]
            out.append([int(v - c[0]) for v in c])
        return tuple(out)

    def neighbour(self, rank: int, face: int) -> int:
        """The rank across face (0..5 = x-, x+, y-, y+, z-, z+), or -1 on the domain boundary."""
        q = list(self.coords(rank))
        q[face // 2] += -1 if face % 2 == 0 else 1
        return self.rank_of(q)

    def local_field(self, rank: int, u):
        """The rank's part of a [nrhs][nz][ny][nx] field (a view; None stays None)."""
        if u is None:
            return None
        (x0, x1), (y0, y1), (z0, z1) = self.box(rank)
        return u[:, z0:z1, y0:y1, x0:x1]

    def local_boundary(self, rank: int, bnd):
        """The rank's packed boundary array [nrhs][nbnd_local]: the global Dirichlet
        data on faces that lie on the domain boundary, zeros on internal faces
        (those are filled by the plane swap every sweep).  bnd: [nrhs][nbnd] or None."""
        nx, ny, nz = self.n
        lx, ly, lz = self.dims(rank)
        (x0, x1), (y0, y1), (z0, z1) = self.box(rank)
        loc = face_layout(lx, ly, lz)
        nb_local = loc[-1][0] + loc[-1][1][0] * loc[-1][1][1]
        if bnd is None:
            return None
        nrhs = bnd.shape[0]
        out = torch.zeros((nrhs, nb_local), dtype=bnd.dtype, device=bnd.device)
        glob = face_layout(nx, ny, nz)
        # each face's (row range, column range) inside the global face of the same side
        ranges = [((z0, z1), (y0, y1))] * 2 + [((z0, z1), (x0, x1))] * 2 + [((y0, y1), (x0, x1))] * 2
        for f in range(6):
            if self.neighbour(rank, f) >= 0:
                continue
            go, gs = glob[f]
            lo, ls = loc[f]
            (r0, r1), (c0, c1) = ranges[f]
            g = bnd[:, go:go + gs[0] * gs[1]].reshape(nrhs, gs[0], gs[1])[:, r0:r1, c0:c1]
            out[:, lo:lo + ls[0] * ls[1]] = g.reshape(nrhs, -1)
        return out


# ---------------------------------------------------------------- compute backends
class GridShard:
    """A rank's sub-grid on its GPU: the CUDA library does every step
    (face planes, sweep, partial sums)."""

    def __init__(self, layout: ShardLayout, rank: int, nrhs: int, device=None):
        from . import Grid
        self.rank = rank
        lx, ly, lz = layout.dims(rank)
        lcx, lcy, lcz = layout.local_cuts(rank)
        self.grid = Grid(lx, ly, lz, nrhs, device=device)
        self.grid.partition(len(lcx) - 1, len(lcy) - 1, len(lcz) - 1, lcx, lcy, lcz)
        self.device = self.grid.device

    def face_planes(self, x):
        return self.grid.face_gather(x)

    def sweep(self, x_in, x_out, f, bnd, opts):
        return self.grid.sweep(x_in, x_out, f=f, bnd=bnd, **opts)

    def norms(self, x, f, bnd):
        return self.grid.norms(x, f=f, bnd=bnd)


# ---------------------------------------------------------------- communication
class LocalComm:
    """Several shards in one process: plane swaps are copies between the
    shards' own buffers, the sum over shards is taken in rank order."""

    def __init__(self, layout: ShardLayout):
        self.layout = layout

    def exchange(self, shards, planes, bnds):
        byrank = {s.rank: i for i, s in enumerate(shards)}
        for i, s in enumerate(shards):
            loc = face_layout(*self.layout.dims(s.rank))
            for f in range(6):
                nb = self.layout.neighbour(s.rank, f)
                if nb < 0:
                    continue
                j = byrank[nb]
                nloc = face_layout(*self.layout.dims(nb))
                so, ss = loc[f]
                no, _ = nloc[OPPOSITE[f]]
                n = ss[0] * ss[1]
                bnds[i][:, so:so + n].copy_(planes[j][:, no:no + n])

    def allreduce_sum(self, parts):
        tot = parts[0].clone()
        for p in parts[1:]:
            tot += p.to(tot.device)
        return tot


class DistComm:
    """One shard per process over torch.distributed (NCCL on GPUs, gloo on
    the CPU): every face plane goes point to point to the neighbour across
    that face (one send and one receive per neighbour pair and sweep), the
    shares of the squared norms are summed by one all-reduce."""

    def __init__(self, layout: ShardLayout, group=None, stage_on_host=None):
        """stage_on_host: move device tensors through host memory for the
        exchange and the sum (default: when the group's backend is gloo, which
        carries host tensors only -- e.g. several processes sharing a GPU)."""
        import torch.distributed as dist
        self.dist = dist
        self.layout = layout
        self.group = group
        if dist.get_world_size(group) != layout.size:
            raise ValueError(f"the layout has {layout.size} ranks, the process group {dist.get_world_size(group)}")
        if stage_on_host is None:
            stage_on_host = dist.get_backend(group) == "gloo"
        self.stage = bool(stage_on_host)

    def _wire(self, t):
        return t.cpu() if self.stage and t.is_cuda else t

    def exchange(self, shards, planes, bnds):
        dist = self.dist
        ops, recvs = [], []
        for i, s in enumerate(shards):
            loc = face_layout(*self.layout.dims(s.rank))
            for f in range(6):
                nb = self.layout.neighbour(s.rank, f)
                if nb < 0:
                    continue
                off, shp = loc[f]
                n = shp[0] * shp[1]
                send = self._wire(planes[i][:, off:off + n].contiguous())
                recv = torch.empty_like(send)
                ops.append(dist.P2POp(dist.isend, send, nb, self.group))
                ops.append(dist.P2POp(dist.irecv, recv, nb, self.group))
                recvs.append((i, off, n, recv))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        for i, off, n, recv in recvs:
            bnds[i][:, off:off + n].copy_(recv)

    def allreduce_sum(self, parts):
        tot = parts[0].clone()
        for p in parts[1:]:
            tot += p
        tot = self._wire(tot)
        self.dist.all_reduce(tot, op=self.dist.ReduceOp.SUM, group=self.group)
        return tot


# ---------------------------------------------------------------- the outer loop
@dataclass
class ShardedStats:
    status: int
    outer_its: int
    per_rhs_outer_its: list
    rel_residual: float
    per_rhs_rel: list
    sweeps: int = 0
    history: list = field(default_factory=list)


STATUS_OK = 0
STATUS_NOT_CONVERGED = 4


def sharded_solve(layout: ShardLayout, shards, comm, bnd=None, f=None, x0=None, outer_tol=1e-8, outer_maxit=100000,
                  history=False, **sweep_opts):
    """Synchronous block Jacobi over the shards of ``layout`` (this process's
    ``shards``; one per process with DistComm, all of them with LocalComm).

    bnd: the GLOBAL packed boundary array [nrhs][nbnd] (each shard takes its
    part), or None; f, x0: GLOBAL [nrhs][nz][ny][nx] fields or None.  They may
    live on any device; each shard's part is copied to its device.
    sweep_opts: ms_sweep options (precision, inner_rtol, inner_maxit, ...).
    Each rhs stops at the first x^k with ||bhat - A x^k|| / ||bhat|| <
    outer_tol (absolute if ||bhat|| = 0), tested on x^k before sweep k+1,
    k = 0 included -- the stop rule of section 2.1 on the global residual.
    Returns ([x part per shard], ShardedStats)."""
    nrhs = None
    for t in (bnd, f, x0):
        if t is not None:
            nrhs = t.shape[0]
            break
    if nrhs is None:
        raise ValueError("give at least one of bnd, f, x0")
    if int(sweep_opts.get("overlap", 0) or 0) > 0 and layout.size > 1:
        # a block box extended by o points reaches o layers into the next rank;
        # the plane swap carries one layer
        raise ValueError("overlapping blocks are not supported across ranks (the plane swap carries one layer)")
    if sweep_opts.get("mode", "sync") not in ("sync", 0):
        raise ValueError("the sharded solve runs synchronous sweeps")

    def on(dev, t):
        return None if t is None else t.to(dev, dtype=torch.float64).contiguous()

    B, F, X, BT = [], [], [], []
    for s in shards:
        lx, ly, lz = layout.dims(s.rank)
        bl = layout.local_boundary(s.rank, bnd)
        if bl is None:
            bl = torch.zeros((nrhs, face_layout(lx, ly, lz)[-1][0] + lx * ly), dtype=torch.float64)
        BT.append(on(s.device, bl))                  # domain-boundary data only (for ||bhat||)
        B.append(BT[-1].clone())                     # plus the neighbours' planes, swapped every sweep
        F.append(on(s.device, layout.local_field(s.rank, f)))
        x = layout.local_field(s.rank, x0)
        x = on(s.device, x) if x is not None else torch.zeros((nrhs, lz, ly, lx), dtype=torch.float64, device=s.device)
        # three rotating iterates: sweep k reads x^k (buffer k % 3) and writes x^{k+1}
        # while the stop test of x^{k-1} (the third buffer) is still being read
        X.append([x, torch.empty_like(x), torch.empty_like(x)])
    # ||bhat||^2 of the global system: f plus the domain-boundary data only
    bb = comm.allreduce_sum([s.norms(X[i][1].zero_(), F[i], BT[i])[1] for i, s in enumerate(shards)])
    bnorm = np.sqrt(bb.cpu().numpy())
    result = [torch.empty_like(x[0]) for x in X]
    active = np.ones(nrhs, dtype=bool)
    kfinal = np.zeros(nrhs, dtype=np.int64)
    conv = np.zeros(nrhs, dtype=bool)
    hist = []

    def launch(k):
        """Enqueue sweep k (x^k -> x^{k+1}; at k = outer_maxit the residual of x^k
        only), the sum of the shares over ranks and its copy to the host; returns
        (host sum, event that completes with the copy or None)."""
        xk = [X[i][k % 3] for i in range(len(shards))]
        planes = [s.face_planes(xk[i]) for i, s in enumerate(shards)]
        comm.exchange(shards, planes, B)
        if k < outer_maxit:
            rr = [s.sweep(xk[i], X[i][(k + 1) % 3], F[i], B[i], sweep_opts) for i, s in enumerate(shards)]
        else:  # the last allowed iterate: its residual only
            rr = [s.norms(xk[i], F[i], B[i])[0] for i, s in enumerate(shards)]
        tot = comm.allreduce_sum(rr)
        if not tot.is_cuda:
            return tot, None
        host = torch.empty(tot.shape, dtype=tot.dtype, pin_memory=True)
        host.copy_(tot, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream(tot.device))
        return host, ev

    # The stop test of x^k is read on the host only after sweep k+1 has been
    # enqueued, so the GPUs never wait for it (one sweep of work past the stop
    # is discarded).  x^k stays in its buffer until sweep k+2 is enqueued.
    k = 0
    pending = launch(0)
    while True:
        nxt = launch(k + 1) if k < outer_maxit else None
        host, ev = pending
        if ev is not None:
            ev.synchronize()
        tot = host.numpy()
        rho = np.where(bnorm > 0.0, np.sqrt(tot) / np.where(bnorm > 0.0, bnorm, 1.0), np.sqrt(tot))
        if history:
            hist.append(rho.copy())
        for r in np.nonzero(active)[0]:
            if rho[r] < outer_tol or k == outer_maxit:
                conv[r] = rho[r] < outer_tol
                active[r] = False
                kfinal[r] = k
                for i in range(len(shards)):
                    result[i][r].copy_(X[i][k % 3][r])
        if not active.any():
            break
        pending = nxt
        k += 1
    # the true residual of the returned iterates (quiescent: fresh planes, one sum)
    planes = [s.face_planes(result[i]) for i, s in enumerate(shards)]
    comm.exchange(shards, planes, B)
    tot = comm.allreduce_sum([s.norms(result[i], F[i], B[i])[0] for i, s in enumerate(shards)]).cpu().numpy()
    rel = np.where(bnorm > 0.0, np.sqrt(tot) / np.where(bnorm > 0.0, bnorm, 1.0), np.sqrt(tot))
    status = STATUS_OK if conv.all() else STATUS_NOT_CONVERGED
    st = ShardedStats(status, int(kfinal.max()), [int(v) for v in kfinal], float(rel.max()),
                      [float(v) for v in rel], sweeps=k, history=hist)
    return result, st


def solve_distributed(nx, ny, nz, cx, cy, cz, ranks, bnd=None, f=None, x0=None, group=None, device=None, **opts):
    """Convenience entry for one process per shard under torch.distributed (NCCL
    between GPUs; gloo works too, through host memory, e.g. for several
    processes sharing one GPU): this rank builds its shard of the rank grid
    ``ranks`` = (rx, ry, rz) and runs ``sharded_solve``.  Returns (this rank's
    part of x, ShardedStats)."""
    import torch.distributed as dist
    layout = ShardLayout(nx, ny, nz, cx, cy, cz, ranks)
    rank = dist.get_rank(group)
    nrhs = next(t.shape[0] for t in (bnd, f, x0) if t is not None)
    shard = GridShard(layout, rank, nrhs, device=device)
    xs, st = sharded_solve(layout, [shard], DistComm(layout, group), bnd=bnd, f=f, x0=x0, **opts)
    return xs[0], st


def solve_local(nx, ny, nz, cx, cy, cz, ranks, bnd=None, f=None, x0=None, devices=None, **opts):
    """Every shard of the rank grid in this process (``devices``: one per rank,
    default the current GPU for all): the same sweeps, swaps and sums as
    ``solve_distributed``, without a process group.  Returns (x assembled on the
    first shard's device, ShardedStats)."""
    layout = ShardLayout(nx, ny, nz, cx, cy, cz, ranks)
    nrhs = next(t.shape[0] for t in (bnd, f, x0) if t is not None)
    devs = devices or [None] * layout.size
    shards = [GridShard(layout, r, nrhs, device=devs[r]) for r in range(layout.size)]
    xs, st = sharded_solve(layout, shards, LocalComm(layout), bnd=bnd, f=f, x0=x0, **opts)
    x = torch.empty((nrhs, nz, ny, nx), dtype=torch.float64, device=xs[0].device)
    for r, part in enumerate(xs):
        layout.local_field(r, x).copy_(part)
    return x, st


__all__ = ["ShardLayout", "GridShard", "LocalComm", "DistComm", "ShardedStats", "sharded_solve", "solve_distributed",
           "solve_local", "face_layout", "FACES"]
