"""The resident engine's single-reduction CG rows (Chronopoulos and Gear's
rearrangement: one cluster reduction of (r.r, r.A r) per iteration).  Same
method as the two-reduction CG of sections 2.2 and 3, so the FP32 result must
meet the same bars against the FP64 oracle: one sweep within 2e-4 (FP32 CG
accuracy), the same inner iteration counts where the tolerance or the cap
stops the solve, and the same converged solution within kappa * tol."""
import numpy as np
import pytest
import torch

import oracle
from paper_2009_12638_gb300 import Grid, MsError, inputs, resident_variants

pytestmark = pytest.mark.gpu


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def make_grid(nx, ny, nz, nrhs, cx, cy, cz):
    return Grid(nx, ny, nz, nrhs).partition(len(cx) - 1, len(cy) - 1, len(cz) - 1, cx, cy, cz)


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SR_ROWS = [v for v, r in enumerate(resident_variants()) if r["one_reduction"]] if torch.cuda.is_available() else []

CASES = [
    (32, 32, 32, [0, 16, 32], [0, 16, 32], [0, 16, 32]),
    (37, 29, 23, [0, 13, 37], [0, 10, 20, 29], [0, 11, 23]),  # ragged strips and slabs
    (64, 64, 64, [0, 64], [0, 64], [0, 64]),                   # one 64^3 block
    (21, 19, 40, [0, 5, 21], [0, 1, 19], [0, 9, 40]),           # 1-wide rows
]


def solve_or_skip(g, **kw):
    try:
        return g.solve(**kw)
    except MsError:
        return None  # this layout does not fit the blocks


def test_table_has_single_reduction_rows():
    assert len(SR_ROWS) >= 3


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("inner_rtol,inner_maxit", [(1e-6, 50), (1e-2, 200), (1e-6, 1), (1e-6, 2)])
def test_one_sweep_matches_oracle(case, inner_rtol, inner_maxit):
    nx, ny, nz, cx, cy, cz = case
    bnd = np.random.default_rng(90).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[0], outer_tol=0.0, outer_maxit=1, inner_rtol=inner_rtol,
                       inner_maxit=inner_maxit)
    g = make_grid(nx, ny, nz, 1, cx, cy, cz)
    ran = 0
    for v in SR_ROWS:
        out = solve_or_skip(g, bnd=cuda(bnd), precision="mixed", variant=v, persistent=False, outer_tol=0.0,
                            outer_maxit=1, inner_rtol=inner_rtol, inner_maxit=inner_maxit)
        if out is None:
            continue
        x, st = out
        assert st.variant == v and st.outer_its == 1
        assert rel_inf(x.cpu().numpy()[0], ref["x"]) <= 2e-4, v
        # the FP32 recurrence may meet a tolerance one step apart from FP64; caps match exactly
        nblocks = (len(cx) - 1) * (len(cy) - 1) * (len(cz) - 1)
        assert abs(st.inner_its - ref["inner_its"]) <= (0 if inner_maxit <= 2 else nblocks), v
        ran += 1
    assert ran >= 1


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("persistent", [True, False])
def test_converges_like_the_two_reduction_cg(case, persistent):
    nx, ny, nz, cx, cy, cz = case
    bnd = np.random.default_rng(91).uniform(-1, 1, size=(2, inputs.boundary_size(nx, ny, nz)))
    g = make_grid(nx, ny, nz, 2, cx, cy, cz)
    x2, s2 = g.solve(bnd=cuda(bnd), precision="mixed", engine="streaming")
    ref = oracle.solve(nx, ny, nz, cx, cy, cz, bnd=bnd[1])
    kappa = 0.5 * (max(nx, ny, nz) + 1) ** 2
    ran = 0
    for v in SR_ROWS:
        out = solve_or_skip(g, bnd=cuda(bnd), precision="mixed", variant=v, persistent=persistent)
        if out is None:
            continue
        x, st = out
        assert st.status == 0 and max(st.per_rhs_rel) < 1e-8, v
        assert (g.residual(x, bnd=cuda(bnd)) < 1e-8).all()
        assert abs(st.outer_its - s2.outer_its) <= max(2, s2.outer_its // 50), v
        assert rel_inf(x.cpu().numpy()[1], ref["x"]) <= 2 * kappa * 1e-8
        ran += 1
    assert ran >= 1


def test_async_converges():
    nx, ny, nz, cx, cy, cz = CASES[0]
    bnd = np.random.default_rng(92).uniform(-1, 1, size=(1, inputs.boundary_size(nx, ny, nz)))
    g = make_grid(nx, ny, nz, 1, cx, cy, cz)
    for v in SR_ROWS:
        out = solve_or_skip(g, bnd=cuda(bnd), precision="mixed", mode="async", variant=v)
        if out is None:
            continue
        x, st = out
        assert st.status == 0 and st.rel_residual < 1e-8, v
        assert g.residual(x, bnd=cuda(bnd))[0] < 1e-8


def test_deterministic_and_persistent_equals_per_sweep():
    """Every CTA forms the scalars from the same fixed-order sums: two runs, and
    the persistent and per-sweep launches, give the same bits."""
    cfg = inputs.make_config("laplace256_u11", scale=4)
    g = make_grid(cfg["nx"], cfg["ny"], cfg["nz"], 1, cfg["cx"], cfg["cy"], cfg["cz"])
    b = cuda(cfg["bnd"])
    v = SR_ROWS[0]
    runs = []
    for persistent in (False, False, True):
        x, st = g.solve(bnd=b, precision="mixed", variant=v, cluster=4, persistent=persistent, outer_tol=0.0,
                        outer_maxit=20)
        runs.append((x.cpu().numpy(), st.inner_its))
    for x, its in runs[1:]:
        np.testing.assert_array_equal(x, runs[0][0])
        assert its == runs[0][1]
