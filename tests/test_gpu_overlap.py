"""Overlapping blocks (opts.overlap, section 3.2) against the oracle's
overlapped multisplitting (extended boxes, weight 1 on owned points), which is
pinned on the CPU to dense extended-box solves.  FP64 sweeps agree up to
summation order (1e-11); a mixed sweep is one FP32 CG per extended box (2e-4)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12638_gb300 import Grid, inputs

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def make(nx, ny, nz, nrhs, cx, cy, cz):
    g = Grid(nx, ny, nz, nrhs)
    g.partition(len(cx) - 1, len(cy) - 1, len(cz) - 1, cx, cy, cz)
    return g


CASES = [
    (24, 20, 16, [0, 12, 24], [0, 10, 20], [0, 8, 16]),
    (29, 17, 23, [0, 7, 19, 29], [0, 9, 17], [0, 11, 23]),   # ragged, 3 blocks along x
    (40, 8, 30, [0, 20, 40], [0, 8], [0, 10, 20, 30]),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("o", [1, 3])
def test_fp64_overlap_sweeps_match_oracle(case, o):
    nx, ny, nz, cx, cy, cz = case
    rng = np.random.default_rng(80 + o)
    bnd = rng.uniform(-1, 1, size=(2, inputs.boundary_size(nx, ny, nz)))
    f = rng.uniform(-1, 1, size=(2, nz, ny, nx))
    g = make(nx, ny, nz, 2, cx, cy, cz)
    x, st = g.solve(f=cuda(f), bnd=cuda(bnd), precision="fp64", overlap=o, outer_tol=0.0, outer_maxit=2)
    assert st.outer_its == 2
    inner = 0
    for s in range(2):
        ref = oracle.solve(nx, ny, nz, cx, cy, cz, f=f[s], bnd=bnd[s], outer_tol=0.0, outer_maxit=2, overlap=o)
        assert rel_inf(x.cpu().numpy()[s], ref["x"]) <= 1e-11, s
        inner += ref["inner_its"]
    assert st.inner_its == inner


@pytest.mark.parametrize("threads", [512, 256])
def test_mixed_overlap_sweep_matches_oracle(threads):
    """512 threads: the vectorised streaming engine; 256: the scalar one."""
    nx, ny, nz, cx, cy, cz = CASES[1]
    bnd = np.random.default_rng(85).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make(nx, ny, nz, 1, cx, cy, cz)
    x, st = g.solve(bnd=cuda(bnd), precision="mixed", overlap=2, threads=threads, outer_tol=0.0, outer_maxit=1)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], outer_tol=0.0, outer_maxit=1, overlap=2)
    assert st.engine == 1
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 2e-4


def test_fp64_overlap_converged_parity_and_fewer_sweeps():
    nx, ny, nz, cx, cy, cz = CASES[0]
    bnd = np.random.default_rng(86).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make(nx, ny, nz, 1, cx, cy, cz)
    x0, s0 = g.solve(bnd=cuda(bnd), precision="fp64")
    x2, s2 = g.solve(bnd=cuda(bnd), precision="fp64", overlap=2)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], overlap=2)
    assert s2.status == 0 and ref["status"] == 0
    assert abs(s2.outer_its - ref["outer_its"]) <= 1
    assert rel_inf(x2.cpu().numpy()[0], ref["x"]) <= 1e-9
    assert s2.outer_its < s0.outer_its
    assert g.residual(x2, bnd=cuda(bnd))[0] < 1e-8


def test_mixed_overlap_converges():
    cfg = inputs.make_config("laplace256_u11", scale=4)  # 64^3 in 4^3 blocks of 16^3
    g = make(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    b = cuda(cfg["bnd"])
    x, st = g.solve(bnd=b, precision="mixed", overlap=2)
    assert st.status == 0 and st.rel_residual < 1e-8 and st.engine == 1
    assert g.residual(x, bnd=b)[0] < 1e-8
