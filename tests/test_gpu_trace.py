"""The solve trace (opts.trace): one record per block solve, written by the
sweep kernels into a device ring and copied out in ticket order.  Checked
against what the solve reports independently: every sweep has one record per
(block, rhs) task, the records' inner iterations add up to stats.inner_its,
and the block residual shares of sweep k add up to the squared global
residual of x^k (section 3: the global residual from block partial sums),
which the residual history gives."""
import numpy as np
import pytest
import torch

from paper_2009_12638_gb300 import Grid, inputs

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def make(cfg, nrhs=1):
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], nrhs)
    return g.partition(len(cfg["cx"]) - 1, len(cfg["cy"]) - 1, len(cfg["cz"]) - 1, cfg["cx"], cfg["cy"], cfg["cz"])


def bhat_sq(g, b):
    return g.norms(torch.zeros(g.shape, dtype=torch.float64, device="cuda"), bnd=b)[1].cpu().numpy()


@pytest.mark.parametrize("opts", [dict(precision="mixed", engine="resident", persistent=False),
                                  dict(precision="mixed", engine="resident", persistent=True),
                                  dict(precision="mixed", engine="streaming"),
                                  dict(precision="fp64"),
                                  dict(precision="mixed", overlap=2)])
def test_sync_trace_matches_the_solve(opts):
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = make(cfg, 2)
    b = cuda(np.concatenate([cfg["bnd"], 0.5 * cfg["bnd"][:, ::-1]]))
    x, st = g.solve(bnd=b, history=True, trace=200000, **opts)
    assert st.status == 0
    tr = st.trace
    ntasks = 64
    assert st.trace_count == len(tr)
    assert tr["inner_its"].sum() == st.inner_its
    bb = bhat_sq(g, b)
    for s in range(2):
        K = st.per_rhs_outer_its[s]
        ts = tr[tr["rhs"] == s]
        # sweeps 0 .. K-1 solve every block once (sweep K only forms the stop residual);
        # the per-sweep launch may also have run sweep K of a rhs that stopped at K
        for k in range(K):
            tk = ts[ts["sweep"] == k]
            assert sorted(tk["block"]) == list(range(ntasks)), (s, k)
            rho = np.sqrt(tk["block_rr"].sum() / bb[s])
            assert rho == pytest.approx(st.history[s][k], rel=1e-9, abs=1e-15)
    if not opts.get("persistent"):
        # one launch per sweep: every record of sweep k is taken before any of sweep k + 1
        ks = tr["sweep"]
        assert (np.diff(ks) >= 0).all()
        for k in range(1, ks.max() + 1):
            assert tr["t_ns"][ks == k].min() >= tr["t_ns"][ks == k - 1].max()


def test_async_trace_counts_each_blocks_own_sweeps():
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = make(cfg)
    b = cuda(cfg["bnd"])
    for engine in ("resident", "streaming"):
        x, st = g.solve(bnd=b, precision="mixed", mode="async", engine=engine, trace=500000)
        assert st.status == 0
        tr = st.trace
        assert st.trace_count == len(tr) and tr["inner_its"].sum() == st.inner_its
        for blk in range(64):
            sw = tr["sweep"][tr["block"] == blk]
            # a block's visits carry its own sweep count 0, 1, 2, ... in the order taken
            np.testing.assert_array_equal(sw, np.arange(len(sw)))
        assert max(np.count_nonzero(tr["block"] == blk) for blk in range(64)) == st.outer_its


def test_trace_ring_keeps_the_last_records_in_order():
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = make(cfg)
    b = cuda(cfg["bnd"])
    cap = 100
    g.solve(bnd=b, precision="mixed", persistent=False)  # tune the launch shape first: the solves below repeat
    full_x, full = g.solve(bnd=b, precision="mixed", persistent=False, trace=400000)
    x, st = g.solve(bnd=b, precision="mixed", persistent=False, trace=cap)
    assert torch.equal(x, full_x)
    assert st.trace_count == full.trace_count > cap
    tr = st.trace
    assert len(tr) == cap
    # the ring holds the last `cap` records in ticket order: the last sweep whole
    # (64 blocks) and the end of the one before it
    kmax = full.trace["sweep"].max()
    assert (np.diff(tr["sweep"]) >= 0).all() and set(tr["sweep"]) <= {kmax - 1, kmax}
    assert sorted(tr["block"][tr["sweep"] == kmax]) == list(range(64))
    prev = tr["block"][tr["sweep"] == kmax - 1]
    assert len(prev) == cap - 64 and len(set(prev)) == len(prev)
    np.testing.assert_array_equal(np.sort(tr["inner_its"]), np.sort(full.trace["inner_its"][-cap:]))


def test_no_trace_by_default_and_rejects_negative_cap():
    cfg = inputs.make_config("laplace32_linear")
    g = make(cfg)
    x, st = g.solve(bnd=cuda(cfg["bnd"]))
    assert st.trace is None and st.trace_count == 0
    import ctypes
    from paper_2009_12638_gb300 import _lib
    lib = _lib.load()
    o = _lib.Opts()
    lib.ms_default_opts(ctypes.byref(o))
    o.trace_cap = -1
    b = cuda(cfg["bnd"])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.ms_solve(g._h, None, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), ctypes.byref(o),
                      None, stream)
    assert rc == _lib.MS_ERR_ARG and b"trace_cap" in lib.ms_last_error(g._h)
