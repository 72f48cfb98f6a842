"""Parity at the full workload sizes, in the launch configuration bench.py
times, on outputs the oracle can produce within seconds: the first outer
sweeps (every block's residual, inner CG and update), a sample of the
right-hand sides, and properties that hold at any size (the true residual
of a converged solve, the adjoint's finite-difference identity).

Tolerances: FP64 sweeps follow the oracle's arithmetic up to rounding order
(1e-11 relative); a mixed sweep is one FP32 CG solve per block, which agrees
with the FP64 one to ~1e-5 relative after 50 iterations (2e-4 allowed).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12638_gb300 import Grid, MsSolve, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(oracle.max_threads())
    yield
    oracle.set_threads(1)


def grid_for(cfg, nrhs=None):
    g = Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["nrhs"] if nrhs is None else nrhs)
    return g.partition(len(cfg["cx"]) - 1, len(cfg["cy"]) - 1, len(cfg["cz"]) - 1, cfg["cx"], cfg["cy"], cfg["cz"])


def rel_inf(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def oracle_sweeps(cfg, s, sweeps):
    return oracle.solve(cfg["nx"], cfg["ny"], cfg["nz"], cfg["cx"], cfg["cy"], cfg["cz"], bnd=cfg["bnd"][s],
                        outer_tol=0.0, outer_maxit=sweeps)


def test_laplace256_first_sweeps_mixed_bench_shape():
    cfg = inputs.make_config("laplace256_u11")
    g = grid_for(cfg)
    # the shape the autotuner picks for this workload on GB300 (resident engine, 16-CTA clusters)
    x, st = g.solve(bnd=torch.from_numpy(cfg["bnd"]).cuda(), precision="mixed", cluster=16, threads=512,
                    outer_tol=0.0, outer_maxit=2)
    assert (st.cluster, st.threads) == (16, 512) and st.outer_its == 2
    ref = oracle_sweeps(cfg, 0, 2)
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 2e-4


def test_laplace256_first_sweeps_fp64():
    cfg = inputs.make_config("laplace256_u11")
    g = grid_for(cfg)
    x, st = g.solve(bnd=torch.from_numpy(cfg["bnd"]).cuda(), precision="fp64", outer_tol=0.0, outer_maxit=2)
    ref = oracle_sweeps(cfg, 0, 2)
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 1e-11
    assert st.inner_its == ref["inner_its"]


def test_laplace256_converged_true_residual():
    cfg = inputs.make_config("laplace256_u11")
    g = grid_for(cfg)
    b = torch.from_numpy(cfg["bnd"]).cuda()
    x, st = g.solve(bnd=b, precision="mixed")
    assert st.status == 0 and st.rel_residual < 1e-8
    assert g.residual(x, bnd=b)[0] < 1e-8


def test_batched_uneven_first_sweep_sampled_rhs():
    cfg = inputs.make_config("batched_uneven")
    g = grid_for(cfg)
    x, st = g.solve(bnd=torch.from_numpy(cfg["bnd"]).cuda(), precision="mixed", outer_tol=0.0, outer_maxit=1)
    assert st.outer_its == 1
    xs = x.cpu().numpy()
    for s in (0, 15):
        ref = oracle_sweeps(cfg, s, 1)
        assert rel_inf(xs[s], ref["x"]) <= 2e-4, s


def test_batched_uneven_first_sweep_fp64_sampled_rhs():
    """The plain FP64 path on the uneven blocks (ragged x-strips: edges that are
    not multiples of 4), in the launch shape the model picks for it (the
    vectorised streaming engine on FP64 strips): one sweep of every rhs, one
    sampled rhs against the oracle."""
    cfg = inputs.make_config("batched_uneven")
    g = grid_for(cfg)
    x, st = g.solve(bnd=torch.from_numpy(cfg["bnd"]).cuda(), precision="fp64", outer_tol=0.0, outer_maxit=1)
    assert st.outer_its == 1
    ref = oracle_sweeps(cfg, 7, 1)
    assert rel_inf(x.cpu().numpy()[7], ref["x"]) <= 1e-11


def test_laplace512_first_sweep_sampled_rhs():
    cfg = inputs.make_config("laplace512_async")
    g = grid_for(cfg)
    x, st = g.solve(bnd=torch.from_numpy(cfg["bnd"]).cuda(), precision="mixed", outer_tol=0.0, outer_maxit=1)
    ref = oracle_sweeps(cfg, 3, 1)
    assert rel_inf(x[3].cpu().numpy(), ref["x"]) <= 2e-4


def test_adjoint128_central_fd():
    """The 128^3 adjoint workload: gradients of L = 0.5 ||u - u_t||^2 with
    respect to f and the Dirichlet data, from the adjoint solve, against central
    differences along 64 Gaussian probes.  L is quadratic in (f, g), so central
    differences are exact up to rounding and solve error (both solves to 1e-12).
    The 128 perturbed solves run as batched multi-rhs solves, 32 rhs each."""
    cfg = inputs.make_config("adjoint128")
    n = cfg["nx"]
    g = grid_for(cfg)
    f0 = torch.zeros((1, n, n, n), dtype=torch.float64, device="cuda")
    g0 = torch.from_numpy(cfg["bnd"]).cuda()
    target = torch.from_numpy(cfg["target"][None]).cuda()
    opts = dict(precision="mixed", outer_tol=1e-12)
    f = f0.clone().requires_grad_(True)
    gb = g0.clone().requires_grad_(True)
    u = MsSolve.apply(f, gb, g, opts)
    (0.5 * ((u - target) ** 2).sum()).backward()
    nprobe = cfg["nprobes"]
    assert nprobe == 64
    vf = inputs.gaussian_probes((1, n, n, n), nprobe, cfg["probe_seed"])
    vg = inputs.gaussian_probes((1, g.nbnd), nprobe, cfg["probe_seed"] + 1)
    theta = float(torch.linalg.vector_norm(g0))
    per = 16  # probes per batched solve (2 rhs each: +eps and -eps)
    gbatch = Grid(n, n, n, 2 * per).partition(4, 4, 4, cfg["cx"], cfg["cy"], cfg["cz"])
    errs = []
    for start in range(0, nprobe, per):
        ids = range(start, start + per)
        v_f = torch.from_numpy(np.concatenate([vf[i] for i in ids])).cuda()  # (per, n, n, n)
        v_g = torch.from_numpy(np.concatenate([vg[i] for i in ids])).cuda()  # (per, nbnd)
        eps = 1e-2 * theta / torch.sqrt((v_f ** 2).sum(dim=(1, 2, 3)) + (v_g ** 2).sum(dim=1))  # (per,)
        sign = torch.tensor([1.0, -1.0], dtype=torch.float64, device="cuda")
        se = (sign[None, :] * eps[:, None]).reshape(-1)  # rhs 2i: +eps_i, 2i+1: -eps_i
        fb = f0 + se[:, None, None, None] * v_f.repeat_interleave(2, dim=0)
        bb = g0 + se[:, None] * v_g.repeat_interleave(2, dim=0)
        uu, st = gbatch.solve(f=fb, bnd=bb, **opts)
        assert st.status == 0
        Ls = 0.5 * ((uu - target) ** 2).sum(dim=(1, 2, 3))
        fd = (Ls[0::2] - Ls[1::2]) / (2 * eps)
        ad = (f.grad * v_f).sum(dim=(1, 2, 3)) + (gb.grad * v_g).sum(dim=1)
        errs.append(((ad - fd).abs() / fd.abs()).cpu().numpy())
    errs = np.concatenate(errs)
    assert errs.size == 64
    assert errs.max() <= 1e-6, errs.max()


def test_laplace256_overlap5_and_adaptive_converge():
    """The bench's comparison paths at full size: overlapping blocks (5 points
    per face) and the inner-tolerance controller reach the true residual."""
    cfg = inputs.make_config("laplace256_u11")
    g = grid_for(cfg)
    b = torch.from_numpy(cfg["bnd"]).cuda()
    for opts in (dict(overlap=5), dict(inner_adapt=True)):
        x, st = g.solve(bnd=b, precision="mixed", **opts)
        assert st.status == 0 and st.rel_residual < 1e-8, opts
        assert g.residual(x, bnd=b)[0] < 1e-8, opts


def test_laplace256_gmres_first_sweep_fp64():
    cfg = inputs.make_config("laplace256_u11")
    g = grid_for(cfg)
    x, st = g.solve(bnd=torch.from_numpy(cfg["bnd"]).cuda(), precision="fp64", inner="gmres", outer_tol=0.0,
                    outer_maxit=1)
    ref = oracle.solve(cfg["nx"], cfg["ny"], cfg["nz"], cfg["cx"], cfg["cy"], cfg["cz"], bnd=cfg["bnd"][0],
                       outer_tol=0.0, outer_maxit=1, inner="gmres", restart=10)
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 1e-10
    assert st.inner_its == ref["inner_its"]
