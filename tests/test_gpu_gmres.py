"""The GMRES inner solver (opts.inner_method = GMRES, section 3.2's Krylov
method) against the oracle's restarted GMRES, itself pinned on the CPU to
least-squares minimal residuals.  FP64 sweeps agree up to summation order in
the reductions (1e-10); a mixed sweep is one FP32 GMRES per block."""
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
    (29, 17, 23, [0, 7, 19, 29], [0, 9, 17], [0, 11, 23]),   # ragged
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("restart", [1, 4, 10])
def test_fp64_gmres_sweeps_match_oracle(case, restart):
    nx, ny, nz, cx, cy, cz = case
    rng = np.random.default_rng(90 + restart)
    bnd = rng.uniform(-1, 1, size=(2, inputs.boundary_size(nx, ny, nz)))
    g = make(nx, ny, nz, 2, cx, cy, cz)
    x, st = g.solve(bnd=cuda(bnd), precision="fp64", inner="gmres", gmres_restart=restart, inner_maxit=30,
                    outer_tol=0.0, outer_maxit=2)
    assert st.outer_its == 2 and st.engine == 1 and st.variant == -1
    inner = 0
    for s in range(2):
        ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[s], inner_maxit=30, outer_tol=0.0, outer_maxit=2,
                           inner="gmres", restart=restart)
        assert rel_inf(x.cpu().numpy()[s], ref["x"]) <= 1e-10, s
        inner += ref["inner_its"]
    nblk = (len(cx) - 1) * (len(cy) - 1) * (len(cz) - 1)
    assert abs(st.inner_its - inner) <= 2 * 2 * nblk


def test_mixed_gmres_sweep_close_to_oracle():
    nx, ny, nz, cx, cy, cz = CASES[1]
    bnd = np.random.default_rng(95).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make(nx, ny, nz, 1, cx, cy, cz)
    x, st = g.solve(bnd=cuda(bnd), precision="mixed", inner="gmres", outer_tol=0.0, outer_maxit=1)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], outer_tol=0.0, outer_maxit=1, inner="gmres", restart=10)
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 5e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gmres_converged(precision):
    nx, ny, nz, cx, cy, cz = CASES[0]
    bnd = np.random.default_rng(96).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make(nx, ny, nz, 1, cx, cy, cz)
    x, st = g.solve(bnd=cuda(bnd), precision=precision, inner="gmres")
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], inner="gmres", restart=10)
    assert st.status == 0 and ref["status"] == 0
    assert g.residual(x, bnd=cuda(bnd))[0] < 1e-8
    if precision == "fp64":
        assert abs(st.outer_its - ref["outer_its"]) <= 1
        assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 1e-9
    else:
        kappa = 0.5 * (max(nx, ny, nz) + 1) ** 2
        assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 2 * kappa * 1e-8


def test_gmres_with_overlap_matches_oracle():
    nx, ny, nz, cx, cy, cz = CASES[0]
    bnd = np.random.default_rng(97).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make(nx, ny, nz, 1, cx, cy, cz)
    x, st = g.solve(bnd=cuda(bnd), precision="fp64", inner="gmres", overlap=2, outer_tol=0.0, outer_maxit=2)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], outer_tol=0.0, outer_maxit=2, inner="gmres", restart=10,
                       overlap=2)
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 1e-10


@pytest.mark.parametrize("restart", [30, 50])
def test_fp64_long_restart_gmres_matches_oracle(restart):
    """Restarts past one projection chunk (16): PETSc's default GMRES(30) and
    the largest basis, with a tight inner tolerance so that steps j >= 16 (and,
    at 30, a restart) run; several chunks of projections per step."""
    nx, ny, nz, cx, cy, cz = CASES[1]
    bnd = np.random.default_rng(98 + restart).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make(nx, ny, nz, 1, cx, cy, cz)
    x, st = g.solve(bnd=cuda(bnd), precision="fp64", inner="gmres", gmres_restart=restart, inner_maxit=60,
                    inner_rtol=1e-10, outer_tol=0.0, outer_maxit=2)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], inner_rtol=1e-10, inner_maxit=60, outer_tol=0.0,
                       outer_maxit=2, inner="gmres", restart=restart)
    assert ref["inner_its"] > 2 * 12 * 16  # on average the blocks go past the first chunk
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 1e-9
    assert abs(st.inner_its - ref["inner_its"]) <= 2 * 12


def test_mixed_gmres30_sweep_close_to_oracle():
    nx, ny, nz, cx, cy, cz = CASES[0]
    bnd = np.random.default_rng(99).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make(nx, ny, nz, 1, cx, cy, cz)
    x, st = g.solve(bnd=cuda(bnd), precision="mixed", inner="gmres", gmres_restart=30, outer_tol=0.0,
                    outer_maxit=1)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], outer_tol=0.0, outer_maxit=1, inner="gmres", restart=30)
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 5e-4


@pytest.mark.parametrize("cuts", [
    ([0, 2, 4, 6], [0, 2, 4], [0, 2, 4]),          # 2^3 blocks: Krylov space of dimension <= 8
    ([0, 1, 2, 3], [0, 1, 2], [0, 1, 2]),          # 1^3 blocks: A_ii = 6, exact after one step
])
def test_gmres_breakdown_on_small_blocks_matches_oracle(cuts):
    """A restart larger than the block's Krylov space: the Arnoldi step that
    reaches an invariant subspace has h_{j+1,j} = 0 (the lucky breakdown), the
    cycle ends with the exact block solve, and no further step runs."""
    cx, cy, cz = cuts
    nx, ny, nz = cx[-1], cy[-1], cz[-1]
    bnd = np.random.default_rng(100 + nx).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make(nx, ny, nz, 1, cx, cy, cz)
    x, st = g.solve(bnd=cuda(bnd), precision="fp64", inner="gmres", gmres_restart=30, inner_maxit=40,
                    inner_rtol=1e-14, outer_tol=0.0, outer_maxit=3)
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], inner_rtol=1e-14, inner_maxit=40, outer_tol=0.0,
                       outer_maxit=3, inner="gmres", restart=30)
    assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 1e-10
    nblk = (len(cx) - 1) * (len(cy) - 1) * (len(cz) - 1)
    bsz = (cx[1] - cx[0]) * (cy[1] - cy[0]) * (cz[1] - cz[0])
    assert ref["inner_its"] <= 3 * nblk * bsz  # finite termination in every block solve
    assert abs(st.inner_its - ref["inner_its"]) <= 3 * nblk
