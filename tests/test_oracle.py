"""Pins for the FP64 CPU oracle, each against something other than the oracle.

Paper: Brown, Bull and Bethune, two-stage multisplitting.  The operator is the
7-point Laplacian of section 2.1, block Jacobi is the formula of section 3,
the stop rule is ||Ax - b|| < tol (section 2.1, Listing 1).
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2009_12638_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def kron_laplacian(nx, ny, nz):
    """A = T_z (x) I (x) I + I (x) T_y (x) I + I (x) I (x) T_x with T = tridiag(-1, 2, -1):
    the textbook Kronecker-sum form of the 7-point Laplacian (x fastest)."""
    def T(n):
        return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    return (sp.kron(Iz, sp.kron(Iy, T(nx))) + sp.kron(Iz, sp.kron(T(ny), Ix)) + sp.kron(T(nz), sp.kron(Iy, Ix))).tocsr()


def padded_with_boundary(nx, ny, nz, bnd, interior=None):
    """(nz+2, ny+2, nx+2) array: boundary faces from the packed layout, interior given or 0."""
    u = np.zeros((nz + 2, ny + 2, nx + 2))
    if interior is not None:
        u[1:-1, 1:-1, 1:-1] = interior
    sl = inputs.face_slices(nx, ny, nz)
    g = [bnd[o:o + s[0] * s[1]].reshape(s) for o, s in sl]
    u[1:-1, 1:-1, 0] = g[0]
    u[1:-1, 1:-1, -1] = g[1]
    u[1:-1, 0, 1:-1] = g[2]
    u[1:-1, -1, 1:-1] = g[3]
    u[0, 1:-1, 1:-1] = g[4]
    u[-1, 1:-1, 1:-1] = g[5]
    return u


def neighbour_sum(u):
    """Sum of the six face neighbours of every interior point of a padded array."""
    return (u[1:-1, 1:-1, 2:] + u[1:-1, 1:-1, :-2] + u[1:-1, 2:, 1:-1] + u[1:-1, :-2, 1:-1]
            + u[2:, 1:-1, 1:-1] + u[:-2, 1:-1, 1:-1])


def bhat_independent(nx, ny, nz, f, bnd):
    """f plus the boundary neighbours' values, from a padded array (no oracle code)."""
    pad = padded_with_boundary(nx, ny, nz, bnd)
    b = neighbour_sum(pad)
    return b if f is None else b + f


def rng(seed=0):
    return np.random.default_rng(seed)


SHAPES = [(1, 1, 1), (2, 3, 4), (5, 4, 3), (6, 6, 6), (7, 1, 3)]


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_apply_A_equals_kronecker_sum(oracle_mod, nx, ny, nz):
    u = rng(1).standard_normal((nz, ny, nx))
    A = kron_laplacian(nx, ny, nz)
    ref = (A @ u.ravel()).reshape(nz, ny, nx)
    np.testing.assert_allclose(oracle_mod.apply_A(u), ref, rtol=0, atol=1e-13)


def test_apply_A_columns_dense(oracle_mod):
    nx, ny, nz = 3, 4, 2
    n = nx * ny * nz
    A = kron_laplacian(nx, ny, nz).toarray()
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        col = oracle_mod.apply_A(e.reshape(nz, ny, nx)).ravel()
        np.testing.assert_array_equal(col, A[:, j])


@pytest.mark.parametrize("nx,ny,nz,a,b,c", [(8, 6, 5, 1, 1, 1), (8, 6, 5, 3, 2, 4), (9, 9, 9, 9, 1, 5)])
def test_sine_eigenpairs(oracle_mod, nx, ny, nz, a, b, c):
    i = np.arange(1, nx + 1)
    j = np.arange(1, ny + 1)
    k = np.arange(1, nz + 1)
    v = (np.sin(c * np.pi * k / (nz + 1))[:, None, None] * np.sin(b * np.pi * j / (ny + 1))[None, :, None]
         * np.sin(a * np.pi * i / (nx + 1))[None, None, :])
    lam = (6 - 2 * np.cos(a * np.pi / (nx + 1)) - 2 * np.cos(b * np.pi / (ny + 1)) - 2 * np.cos(c * np.pi / (nz + 1)))
    np.testing.assert_allclose(oracle_mod.apply_A(v), lam * v, rtol=0, atol=1e-13)


def test_operator_symmetric(oracle_mod):
    r = rng(2)
    u, v = r.standard_normal((2, 5, 6, 7))
    lhs = np.vdot(oracle_mod.apply_A(u), v)
    rhs = np.vdot(u, oracle_mod.apply_A(v))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------------- lift
@pytest.mark.parametrize("fn", [inputs.harmonic_linear, inputs.harmonic_xyz])
@pytest.mark.parametrize("nx,ny,nz", [(5, 6, 7), (12, 12, 12), (3, 9, 4)])
def test_harmonic_samples_solve_lifted_system(oracle_mod, fn, nx, ny, nz):
    """u = x+2y+3z and u = xyz are affine in each coordinate separately, so every
    second difference vanishes: their samples solve A u = lift(g) exactly."""
    g = inputs.boundary_from_function(nx, ny, nz, fn)
    u = inputs.interior_from_function(nx, ny, nz, fn)
    bhat = oracle_mod.lift(nx, ny, nz, None, g)
    r = oracle_mod.residual(bhat, u)
    assert np.abs(r).max() <= 1e-13 * max(1.0, np.abs(bhat).max())


@pytest.mark.parametrize("nx,ny,nz", [(1, 1, 1), (2, 3, 4), (6, 5, 4)])
def test_lift_matches_padded_neighbour_sum(oracle_mod, nx, ny, nz):
    r = rng(3)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    f = r.standard_normal((nz, ny, nx))
    np.testing.assert_allclose(oracle_mod.lift(nx, ny, nz, f, g), bhat_independent(nx, ny, nz, f, g), atol=1e-14)
    np.testing.assert_array_equal(oracle_mod.lift(nx, ny, nz, f, None), f)


def test_golden_tiny_systems(oracle_mod):
    """Hand-solved systems (derivations in the fixture)."""
    with open(os.path.join(GOLDEN, "tiny_systems.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        nx, ny, nz = c["shape"]
        g = np.asarray(c["bnd"], dtype=np.float64)
        bhat = oracle_mod.lift(nx, ny, nz, None, g)
        np.testing.assert_allclose(bhat.ravel(), c["bhat"], atol=1e-14)
        res = oracle_mod.solve(nx, ny, nz, [0, nx], [0, ny], [0, nz], bnd=g, inner_rtol=1e-15, inner_maxit=100,
                               outer_tol=1e-14, outer_maxit=5)
        np.testing.assert_allclose(res["x"].ravel(), c["x"], rtol=1e-13)


# ---------------------------------------------------------------- inner CG
def test_block_cg_recurrence_residual_is_true_residual(oracle_mod):
    r0 = rng(4).standard_normal((5, 6, 7))
    d, r, m = oracle_mod.block_cg(r0, 1e-10, 200)
    true = r0 - oracle_mod.apply_A(d)
    assert m > 0
    assert np.abs(true - r).max() <= 1e-10 * np.abs(r0).max()
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(r0) * 1.0000001


def test_block_cg_single_point_one_step(oracle_mod):
    d, r, m = oracle_mod.block_cg(np.array([[[3.0]]]), 1e-6, 50)
    assert m == 1 and d[0, 0, 0] == 0.5 and r[0, 0, 0] == 0.0


def test_block_cg_zero_rhs_and_zero_maxit(oracle_mod):
    d, r, m = oracle_mod.block_cg(np.zeros((3, 3, 3)), 1e-6, 50)
    assert m == 0 and not d.any()
    d, r, m = oracle_mod.block_cg(np.ones((3, 3, 3)), 1e-6, 0)
    assert m == 0 and not d.any()


def test_block_cg_finite_termination(oracle_mod):
    """CG terminates within the number of distinct eigenvalues; a 2x2x2 block has
    4 distinct eigenvalues (6 - 2cos(a pi/3)... sums), so <= 4 steps reach 1e-12."""
    r0 = rng(5).standard_normal((2, 2, 2))
    d, r, m = oracle_mod.block_cg(r0, 1e-12, 100)
    assert m <= 4
    A = kron_laplacian(2, 2, 2).toarray()
    np.testing.assert_allclose(d.ravel(), np.linalg.solve(A, r0.ravel()), rtol=1e-10, atol=1e-12)


def krylov_basis(A, r0, m):
    """Orthonormal basis of K_m(A, r0) = span{r0, A r0, ..., A^(m-1) r0} by Arnoldi
    with two Gram-Schmidt passes per vector (numpy, no oracle code)."""
    Q = np.zeros((r0.size, m))
    Q[:, 0] = r0 / np.linalg.norm(r0)
    for j in range(1, m):
        w = A @ Q[:, j - 1]
        for _ in range(2):
            w = w - Q[:, :j] @ (Q[:, :j].T @ w)
        Q[:, j] = w / np.linalg.norm(w)
    return Q


def cg_minimisers(A, r0, mmax):
    """For m = 1..mmax the d_m in K_m(A, r0) minimising the A-norm of the error
    ||A^-1 r0 - d||_A, i.e. the Galerkin solution d_m = Q (Q^T A Q)^-1 Q^T r0 --
    the characterisation of the m-th CG iterate from d = 0 (section 2.2)."""
    out = []
    for m in range(1, mmax + 1):
        Q = krylov_basis(A, r0, m)
        out.append(Q @ np.linalg.solve(Q.T @ A @ Q, Q.T @ r0))
    return out


@pytest.mark.parametrize("shape", [(5, 6, 7), (8, 8, 8), (9, 3, 4)])
def test_block_cg_truncated_iterates_minimise_the_a_norm_error(oracle_mod, shape):
    """The hot path always stops CG long before finite termination (64^3 blocks,
    cap 50), so the truncated iterate itself is pinned: with inner_rtol = 0 the
    solve takes exactly m = inner_maxit steps and returns the A-norm minimiser
    over K_m(A_ii, r_0), and its r is the true residual r_0 - A_ii d."""
    bx, by, bz = shape
    A = kron_laplacian(bx, by, bz).toarray()
    r0 = rng(40 + bx).standard_normal(A.shape[0])
    ref = cg_minimisers(A, r0, 12)
    for m in range(1, 13):
        d, r, its = oracle_mod.block_cg(r0.reshape(bz, by, bx), 0.0, m)
        assert its == m
        np.testing.assert_allclose(d.ravel(), ref[m - 1], rtol=0, atol=1e-10 * np.abs(ref[m - 1]).max())
        np.testing.assert_allclose(r.ravel(), r0 - A @ d.ravel(), rtol=0, atol=1e-12 * np.abs(r0).max())


@pytest.mark.parametrize("target", [3, 7, 11])
def test_block_cg_stops_at_the_first_step_meeting_the_tolerance(oracle_mod, target):
    """With inner_rtol > 0 the returned m is the first m with
    ||r_0 - A d_m|| <= inner_rtol ||r_0||, d_m the Krylov minimiser (the CG
    residual norm need not decrease monotonically, so 'first' matters); the
    tolerance is placed just above the target step's ratio and far (relative
    1e-6) from every other step's, so rounding cannot move the stop.  A cap at
    the stop step gives the same m; a cap one below it gives the cap."""
    bx, by, bz = 6, 7, 5
    A = kron_laplacian(bx, by, bz).toarray()
    r0 = rng(50).standard_normal(A.shape[0])
    ratios = np.array([np.linalg.norm(r0 - A @ d) for d in cg_minimisers(A, r0, 14)]) / np.linalg.norm(r0)
    rtol = ratios[target - 1] * (1 + 1e-7)
    first = 1 + int(np.argmax(ratios <= rtol))
    assert np.all(np.abs(ratios / rtol - 1) > 1e-8)
    d, r, m = oracle_mod.block_cg(r0.reshape(bz, by, bx), rtol, 200)
    assert m == first
    assert np.linalg.norm(r) <= rtol * np.linalg.norm(r0)
    _, _, m_cap = oracle_mod.block_cg(r0.reshape(bz, by, bx), rtol, first)
    assert m_cap == first
    _, _, m_short = oracle_mod.block_cg(r0.reshape(bz, by, bx), rtol, first - 1)
    assert m_short == first - 1


def test_block_cg_tolerance_tie_stops(oracle_mod):
    """The stop test is ||r_m|| <= inner_rtol ||r_0|| (non-strict).  Block 2x1x1
    (A = [[6, -1], [-1, 6]]), r_0 = (1, 0): one CG step has alpha = 1/6 and
    r_1 = (1 - 6 alpha, alpha) = (0, 1/6), so ||r_1|| = ||r_0|| / 6 exactly.
    In FP64 every step is exact too: fl(1/6) * 6 rounds (a tie, to even) to 1,
    and sqrt(fl(1/6)^2) = fl(1/6).  With inner_rtol = fl(1/6) the test is a tie:
    the solve must stop after one step.  One ulp lower it must take the second
    step (which solves the 2x2 system exactly)."""
    sixth = 1.0 / 6.0
    assert sixth * 6.0 == 1.0 and np.sqrt(sixth * sixth) == sixth
    r0 = np.array([[[1.0, 0.0]]])
    d, r, m = oracle_mod.block_cg(r0, sixth, 50)
    assert m == 1
    np.testing.assert_array_equal(d.ravel(), [sixth, 0.0])
    np.testing.assert_array_equal(r.ravel(), [0.0, sixth])
    d, r, m = oracle_mod.block_cg(r0, np.nextafter(sixth, 0.0), 50)
    assert m == 2
    np.testing.assert_allclose(d.ravel(), np.linalg.solve([[6.0, -1.0], [-1.0, 6.0]], [1.0, 0.0]), rtol=1e-15)


# ---------------------------------------------------------------- outer sweeps
def test_one_sweep_with_unit_blocks_is_point_jacobi(oracle_mod):
    """1x1x1 blocks: A_ii = [6] and one CG step is exact, so one outer sweep is
    the point-Jacobi update of section 2.1: u_new = (f + sum of six neighbours)/6."""
    nx, ny, nz = 6, 5, 4
    r = rng(6)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    f = r.standard_normal((nz, ny, nx))
    x0 = r.standard_normal((nz, ny, nx))
    res = oracle_mod.solve(nx, ny, nz, np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), f=f, bnd=g, x0=x0,
                           outer_tol=0.0, outer_maxit=1)
    pad = padded_with_boundary(nx, ny, nz, g, x0)
    ref = (f + neighbour_sum(pad)) / 6.0
    assert res["outer_its"] == 1 and res["inner_its"] == nx * ny * nz
    np.testing.assert_allclose(res["x"], ref, rtol=1e-13, atol=1e-13)


def test_single_block_one_sweep_is_lu(oracle_mod):
    nx, ny, nz = 5, 4, 6
    r = rng(7)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    f = r.standard_normal((nz, ny, nx))
    res = oracle_mod.solve(nx, ny, nz, [0, nx], [0, ny], [0, nz], f=f, bnd=g, inner_rtol=1e-15, inner_maxit=1000,
                           outer_tol=0.0, outer_maxit=1)
    A = kron_laplacian(nx, ny, nz).toarray()
    x_lu = np.linalg.solve(A, bhat_independent(nx, ny, nz, f, g).ravel())
    np.testing.assert_allclose(res["x"].ravel(), x_lu, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("cuts", [((0, 4, 8), (0, 4, 8), (0, 4, 8)), ((0, 3, 7), (0, 2, 5, 6), (0, 5, 8))])
def test_exact_block_jacobi_sweeps_match_dense(oracle_mod, cuts):
    """Inner CG to 1e-15: every sweep must equal x + blockdiag(A)^{-1} (b - A x)."""
    cx, cy, cz = (np.asarray(c) for c in cuts)
    nx, ny, nz = cx[-1], cy[-1], cz[-1]
    r = rng(8)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    A = kron_laplacian(nx, ny, nz).toarray()
    b = bhat_independent(nx, ny, nz, None, g).ravel()
    ix = np.searchsorted(cx, np.arange(nx), side="right") - 1
    iy = np.searchsorted(cy, np.arange(ny), side="right") - 1
    iz = np.searchsorted(cz, np.arange(nz), side="right") - 1
    bid = ix[None, None, :] + (len(cx) - 1) * (iy[None, :, None] + (len(cy) - 1) * iz[:, None, None])
    bid = bid.ravel()
    M = np.where(bid[:, None] == bid[None, :], A, 0.0)
    x = np.zeros(A.shape[0])
    for k in range(1, 4):
        x = x + np.linalg.solve(M, b - A @ x)
        res = oracle_mod.solve(nx, ny, nz, cx, cy, cz, bnd=g, inner_rtol=1e-15, inner_maxit=2000, outer_tol=0.0,
                               outer_maxit=k)
        np.testing.assert_allclose(res["x"].ravel(), x, rtol=1e-10, atol=1e-11)


# ---------------------------------------------------------------- convergence
@pytest.mark.parametrize("fn", [inputs.harmonic_linear, inputs.harmonic_xyz])
def test_converges_to_harmonic_closed_form(oracle_mod, fn):
    n = 16
    c = inputs.equal_cuts(n, 2)
    g = inputs.boundary_from_function(n, n, n, fn)
    exact = inputs.interior_from_function(n, n, n, fn)
    res = oracle_mod.solve(n, n, n, c, c, c, bnd=g, outer_tol=1e-12)
    assert res["status"] == 0
    assert np.abs(res["x"] - exact).max() <= 1e-9 * np.abs(exact).max()


def test_linear_config_32(oracle_mod):
    cfg = inputs.make_config("laplace32_linear")
    res = oracle_mod.solve(cfg["nx"], cfg["ny"], cfg["nz"], cfg["cx"], cfg["cy"], cfg["cz"], bnd=cfg["bnd"][0],
                           history=True, **cfg["opts"])
    assert res["status"] == 0 and res["rel_residual"] < 1e-8
    assert res["history"][-1] < 1e-8 <= res["history"][-2]
    # kappa(A) ~ 0.4 (n+1)^2 bounds the error at tol 1e-8
    assert np.abs(res["x"] - cfg["exact"][0]).max() <= 440 * 1e-8 * np.abs(cfg["exact"]).max()


def test_random_dense_lu(oracle_mod):
    nx, ny, nz = 6, 5, 6
    r = rng(9)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    f = r.standard_normal((nz, ny, nx))
    A = kron_laplacian(nx, ny, nz).toarray()
    x_lu = np.linalg.solve(A, bhat_independent(nx, ny, nz, f, g).ravel())
    res = oracle_mod.solve(nx, ny, nz, [0, 3, 6], [0, 2, 5], [0, 2, 4, 6], f=f, bnd=g, outer_tol=1e-12)
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(res["x"].ravel() - x_lu) <= kappa * 1e-12 * np.linalg.norm(x_lu)


def test_more_blocks_more_outer_iterations(oracle_mod):
    """Section 3.2: splitting into more groups raises the outer iteration count."""
    n = 16
    g = inputs.boundary_uniform(n, n, n, 1, 11)[0]
    its = []
    for p in (1, 2, 4):
        c = inputs.equal_cuts(n, p)
        its.append(oracle_mod.solve(n, n, n, c, c, c, bnd=g, inner_maxit=20, outer_tol=1e-8)["outer_its"])
    assert its[0] < its[1] < its[2]


def test_more_inner_iterations_fewer_outer(oracle_mod):
    """Section 3.2: a larger inner iteration cap lowers the outer count, down to
    the count of exact block solves (8^3 blocks reach inner 1e-6 in ~15 steps)."""
    n = 16
    c = inputs.equal_cuts(n, 2)
    g = inputs.boundary_uniform(n, n, n, 1, 12)[0]
    its = [oracle_mod.solve(n, n, n, c, c, c, bnd=g, inner_maxit=m, outer_tol=1e-8)["outer_its"] for m in (2, 4, 8, 50)]
    assert its[0] > its[1] > its[2]
    assert abs(its[3] - its[2]) <= 2


# ---------------------------------------------------------------- stop rule
def test_zero_rhs_stops_at_zero(oracle_mod):
    n = 6
    c = inputs.equal_cuts(n, 2)
    res = oracle_mod.solve(n, n, n, c, c, c, bnd=np.zeros(inputs.boundary_size(n, n, n)))
    assert res["status"] == 0 and res["outer_its"] == 0 and not res["x"].any()


def test_exact_start_stops_at_zero(oracle_mod):
    n = 8
    c = inputs.equal_cuts(n, 2)
    g = inputs.boundary_from_function(n, n, n, inputs.harmonic_linear)
    x0 = inputs.interior_from_function(n, n, n, inputs.harmonic_linear)
    res = oracle_mod.solve(n, n, n, c, c, c, bnd=g, x0=x0)
    assert res["outer_its"] == 0 and res["status"] == 0


def test_outer_maxit_zero_not_converged(oracle_mod):
    n = 6
    c = inputs.equal_cuts(n, 2)
    g = inputs.boundary_uniform(n, n, n, 1, 13)[0]
    res = oracle_mod.solve(n, n, n, c, c, c, bnd=g, outer_maxit=0, history=True)
    assert res["status"] == 4 and res["outer_its"] == 0 and res["history"][0] == pytest.approx(1.0)


def test_strict_less_than(oracle_mod):
    n = 6
    c = inputs.equal_cuts(n, 2)
    g = inputs.boundary_uniform(n, n, n, 1, 14)[0]
    # x0 = 0 gives relative residual exactly 1: tol = 1 must not stop, tol just above must
    assert oracle_mod.solve(n, n, n, c, c, c, bnd=g, outer_tol=1.0, outer_maxit=0)["status"] == 4
    assert oracle_mod.solve(n, n, n, c, c, c, bnd=g, outer_tol=1.0000001, outer_maxit=0)["status"] == 0


def test_bad_cuts_rejected(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.solve(4, 4, 4, [0, 2, 2, 4], [0, 4], [0, 4])
    with pytest.raises(ValueError):
        oracle_mod.solve(4, 4, 4, [0, 3], [0, 4], [0, 4])


def test_threads_do_not_change_results(oracle_mod):
    n = 12
    c = inputs.equal_cuts(n, 3)
    g = inputs.boundary_uniform(n, n, n, 1, 15)[0]
    oracle_mod.set_threads(1)
    a = oracle_mod.solve(n, n, n, c, c, c, bnd=g, outer_maxit=5, outer_tol=0.0)
    oracle_mod.set_threads(4)
    b = oracle_mod.solve(n, n, n, c, c, c, bnd=g, outer_maxit=5, outer_tol=0.0)
    oracle_mod.set_threads(1)
    np.testing.assert_array_equal(a["x"], b["x"])


# ---------------------------------------------------------------- asynchronous model
def test_delayed_with_zero_delays_is_synchronous(oracle_mod):
    n = 10
    c = inputs.equal_cuts(n, 2)
    g = inputs.boundary_uniform(n, n, n, 1, 16)[0]
    d = np.zeros((201, 8, 6), dtype=np.int32)
    a = oracle_mod.solve(n, n, n, c, c, c, bnd=g, outer_maxit=200)
    b = oracle_mod.solve_delayed(n, n, n, c, c, c, d, 0, bnd=g, outer_maxit=200)
    assert a["outer_its"] == b["outer_its"]
    np.testing.assert_array_equal(a["x"], b["x"])


@pytest.mark.parametrize("cuts,max_delay", [(((0, 3, 6), (0, 2, 5), (0, 4, 6)), 2),
                                             (((0, 2, 5, 7), (0, 4), (0, 3, 5)), 3)])
def test_delayed_sweeps_match_dense_block_solves_with_stale_faces(oracle_mod, cuts, max_delay):
    """The asynchronous model (sections 2.1, 2.3 and 3: a block uses the latest
    values it has received, possibly several sweeps old), with exact inner
    solves, restated densely in numpy: block i's sweep k solves its dense
    diagonal block A_ii against bhat - A x~, where x~ is x^k except on the layer
    of points across each face, which comes from x^(k - d) for that face's delay
    d (capped by max_delay and by sweep 0).  Sweep for sweep the oracle must
    give the same iterates."""
    cx, cy, cz = (np.asarray(c) for c in cuts)
    nx, ny, nz = int(cx[-1]), int(cy[-1]), int(cz[-1])
    px, py, pz = len(cx) - 1, len(cy) - 1, len(cz) - 1
    nblocks = px * py * pz
    g = rng(19).standard_normal(inputs.boundary_size(nx, ny, nz))
    f = rng(20).standard_normal((nz, ny, nx))
    K = 5
    delays = rng(21).integers(0, max_delay + 2, size=(K + 1, nblocks, 6)).astype(np.int32)  # some above the cap
    A = kron_laplacian(nx, ny, nz).toarray()
    b = bhat_independent(nx, ny, nz, f, g)
    X = [np.zeros((nz, ny, nx))]
    for k in range(K):
        xn = X[k].copy()
        for blk in range(nblocks):
            bi, bj, bk = blk % px, (blk // px) % py, blk // (px * py)
            lo = (cx[bi], cy[bj], cz[bk])
            hi = (cx[bi + 1], cy[bj + 1], cz[bk + 1])
            xv = X[k].copy()
            for face in range(6):
                axis = face // 2
                d = min(int(delays[k, blk, face]), max_delay)
                ks = max(k - d, 0)
                layer = lo[axis] - 1 if face % 2 == 0 else hi[axis]
                if layer < 0 or layer >= (nx, ny, nz)[axis]:
                    continue
                sl = [slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0])]  # (z, y, x)
                sl[2 - axis] = slice(layer, layer + 1)
                xv[tuple(sl)] = X[ks][tuple(sl)]
            r = (b - (A @ xv.ravel()).reshape(nz, ny, nx))
            own = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
            mask = np.zeros((nz, ny, nx), dtype=bool)
            mask[own] = True
            m = mask.ravel()
            delta = np.linalg.solve(A[np.ix_(m, m)], r.ravel()[m])
            xn[own] += delta.reshape(hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])
        X.append(xn)
        res = oracle_mod.solve_delayed(nx, ny, nz, cx, cy, cz, np.resize(delays, (k + 2, nblocks, 6)), max_delay, f=f,
                                       bnd=g, inner_rtol=1e-15, inner_maxit=2000, outer_tol=0.0, outer_maxit=k + 1)
        np.testing.assert_allclose(res["x"], xn, rtol=0, atol=1e-10 * np.abs(xn).max())


def test_delayed_converges_to_lu(oracle_mod):
    """Bounded staleness still converges for this M-matrix (section 2.1 cites the
    asynchronous convergence theory); at least as many sweeps as synchronous."""
    n = 8
    c = inputs.equal_cuts(n, 2)
    g = inputs.boundary_uniform(n, n, n, 1, 17)[0]
    d = inputs.delay_schedule(400, 8, 3, 18)
    res = oracle_mod.solve_delayed(n, n, n, c, c, c, d, 3, bnd=g, outer_maxit=400, outer_tol=1e-10)
    sync = oracle_mod.solve(n, n, n, c, c, c, bnd=g, outer_maxit=400, outer_tol=1e-10)
    assert res["status"] == 0 and res["outer_its"] >= sync["outer_its"]
    A = kron_laplacian(n, n, n).toarray()
    x_lu = np.linalg.solve(A, bhat_independent(n, n, n, None, g).ravel())
    assert np.abs(res["x"].ravel() - x_lu).max() <= np.linalg.cond(A) * 1e-10 * np.abs(x_lu).max()


# ---------------------------------------------------------------- overlapping blocks
def _boxes(cuts, n, o):
    """Owned and extended index ranges per block along one axis."""
    c = np.asarray(cuts)
    return [(c[i], c[i + 1], max(0, c[i] - o), min(n, c[i + 1] + o)) for i in range(len(c) - 1)]


def dense_overlap_sweeps(nx, ny, nz, cx, cy, cz, o, f, g, sweeps):
    """Brute force (no oracle code): every block solves its extended-box system
    A[E,E] d = (b - A x)[E] exactly (dense LU) and x takes d on the points the
    block owns."""
    A = kron_laplacian(nx, ny, nz).toarray()
    b = bhat_independent(nx, ny, nz, f, g).ravel()
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    x = np.zeros(A.shape[0])
    out = []
    for _ in range(sweeps):
        r = b - A @ x
        xn = x.copy()
        for (wz0, wz1, ez0, ez1) in _boxes(cz, nz, o):
            for (wy0, wy1, ey0, ey1) in _boxes(cy, ny, o):
                for (wx0, wx1, ex0, ex1) in _boxes(cx, nx, o):
                    E = idx[ez0:ez1, ey0:ey1, ex0:ex1].ravel()
                    d = np.linalg.solve(A[np.ix_(E, E)], r[E]).reshape(ez1 - ez0, ey1 - ey0, ex1 - ex0)
                    W = idx[wz0:wz1, wy0:wy1, wx0:wx1].ravel()
                    xn[W] = x[W] + d[wz0 - ez0:wz1 - ez0, wy0 - ey0:wy1 - ey0, wx0 - ex0:wx1 - ex0].ravel()
        x = xn
        out.append(x.copy())
    return out


def test_overlap_zero_is_block_jacobi(oracle_mod):
    """Overlap 0 is the non-overlapping method, bit for bit."""
    nx, ny, nz = 11, 9, 7
    r = rng(20)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    f = r.standard_normal((nz, ny, nx))
    cuts = ([0, 4, 11], [0, 3, 6, 9], [0, 7])
    a = oracle_mod.solve(nx, ny, nz, *cuts, f=f, bnd=g, inner_maxit=7, outer_tol=1e-9)
    b = oracle_mod.solve(nx, ny, nz, *cuts, f=f, bnd=g, inner_maxit=7, outer_tol=1e-9, overlap=0)
    np.testing.assert_array_equal(a["x"], b["x"])
    assert (a["outer_its"], a["inner_its"]) == (b["outer_its"], b["inner_its"])


@pytest.mark.parametrize("o", [1, 2, 3])
@pytest.mark.parametrize("cuts", [((0, 3, 6), (0, 2, 5), (0, 2, 4)), ((0, 2, 4, 6), (0, 5), (0, 1, 4))])
def test_overlap_sweeps_match_dense_extended_solves(oracle_mod, o, cuts):
    cx, cy, cz = (list(c) for c in cuts)
    nx, ny, nz = cx[-1], cy[-1], cz[-1]
    r = rng(21 + o)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    f = r.standard_normal((nz, ny, nx))
    ref = dense_overlap_sweeps(nx, ny, nz, cx, cy, cz, o, f, g, 3)
    for k in range(1, 4):
        res = oracle_mod.solve(nx, ny, nz, cx, cy, cz, f=f, bnd=g, inner_rtol=1e-15, inner_maxit=2000,
                               outer_tol=0.0, outer_maxit=k, overlap=o)
        np.testing.assert_allclose(res["x"].ravel(), ref[k - 1], rtol=1e-10, atol=1e-11)


def test_overlap_covering_the_grid_solves_in_one_sweep(oracle_mod):
    """When every extended box is the whole grid, one sweep with exact inner
    solves is one exact solve per block: the LU solution."""
    nx, ny, nz = 6, 5, 4
    r = rng(25)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    A = kron_laplacian(nx, ny, nz).toarray()
    x_lu = np.linalg.solve(A, bhat_independent(nx, ny, nz, None, g).ravel())
    res = oracle_mod.solve(nx, ny, nz, [0, 3, 6], [0, 2, 5], [0, 2, 4], bnd=g, inner_rtol=1e-15, inner_maxit=2000,
                           outer_tol=0.0, outer_maxit=1, overlap=6)
    np.testing.assert_allclose(res["x"].ravel(), x_lu, rtol=1e-10, atol=1e-11)


def test_overlap_converges_to_lu(oracle_mod):
    nx, ny, nz = 8, 7, 6
    r = rng(26)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    f = r.standard_normal((nz, ny, nx))
    A = kron_laplacian(nx, ny, nz).toarray()
    x_lu = np.linalg.solve(A, bhat_independent(nx, ny, nz, f, g).ravel())
    res = oracle_mod.solve(nx, ny, nz, [0, 4, 8], [0, 3, 7], [0, 3, 6], f=f, bnd=g, outer_tol=1e-12, overlap=2)
    assert res["status"] == 0
    assert np.linalg.norm(res["x"].ravel() - x_lu) <= np.linalg.cond(A) * 1e-12 * np.linalg.norm(x_lu)


def test_small_overlap_needs_fewer_outer_sweeps(oracle_mod):
    """Section 3.2: an overlap of one to a few elements lowers the outer
    iteration count (2341 -> 1771 -> 1330 for overlaps 0, 1, 5 in the paper)."""
    n = 24
    c = inputs.equal_cuts(n, 4)
    g = rng(27).uniform(-1, 1, inputs.boundary_size(n, n, n))
    its = [oracle_mod.solve(n, n, n, c, c, c, bnd=g, outer_tol=1e-8, overlap=o)["outer_its"] for o in (0, 1, 2)]
    assert its[1] < its[0] and its[2] < its[1]


# ---------------------------------------------------------------- GMRES inner solver
def _block_matrix(bx, by, bz):
    return kron_laplacian(bx, by, bz).toarray()


@pytest.mark.parametrize("shape", [(4, 3, 3), (5, 4, 2), (3, 3, 3)])
@pytest.mark.parametrize("steps", [1, 3, 6])
def test_gmres_minimises_the_residual_over_the_krylov_space(oracle_mod, shape, steps):
    """Without restart, j GMRES steps give the d in K_j(A, r) with the smallest
    ||r - A d||: compared with a least-squares solve over an orthonormal basis
    of the Krylov space built from powers of A (numpy, no oracle code)."""
    bx, by, bz = shape
    A = _block_matrix(bx, by, bz)
    r0 = rng(30 + steps).standard_normal(bx * by * bz)
    d, r_fin, m = oracle_mod.block_gmres(r0.reshape(bz, by, bx), 0.0, steps, steps)
    assert m == steps
    K = np.empty((r0.size, steps))
    v = r0 / np.linalg.norm(r0)
    for j in range(steps):
        K[:, j] = v
        v = A @ v
        v /= np.linalg.norm(v)
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(A @ Q, r0, rcond=None)
    best = np.linalg.norm(r0 - A @ (Q @ y))
    got = np.linalg.norm(r0 - A @ d.ravel())
    assert got == pytest.approx(best, rel=1e-8, abs=1e-12)
    # r is returned as the true residual of d
    np.testing.assert_allclose(r_fin.ravel(), r0 - A @ d.ravel(), rtol=1e-12, atol=1e-12)


def test_gmres_finite_termination_equals_lu(oracle_mod):
    """With a restart at least the block size, GMRES is exact after <= n steps."""
    bx, by, bz = 3, 4, 2
    A = _block_matrix(bx, by, bz)
    r0 = rng(35).standard_normal(bx * by * bz)
    d, _, m = oracle_mod.block_gmres(r0.reshape(bz, by, bx), 1e-14, 100, 100)
    assert m <= r0.size
    np.testing.assert_allclose(d.ravel(), np.linalg.solve(A, r0), rtol=1e-9, atol=1e-11)


def test_gmres_restarts_reduce_the_residual_monotonically(oracle_mod):
    bx, by, bz = 8, 7, 6
    A = _block_matrix(bx, by, bz)
    r0 = rng(36).standard_normal(bx * by * bz)
    norms = []
    for maxit in (5, 10, 15, 20, 40):
        d, _, m = oracle_mod.block_gmres(r0.reshape(bz, by, bx), 0.0, maxit, 5)
        assert m == maxit
        norms.append(np.linalg.norm(r0 - A @ d.ravel()))
    assert all(b < a for a, b in zip(norms, norms[1:]))


def test_gmres_inner_solves_converge_to_lu(oracle_mod):
    nx, ny, nz = 8, 7, 6
    r = rng(37)
    g = r.standard_normal(inputs.boundary_size(nx, ny, nz))
    A = kron_laplacian(nx, ny, nz).toarray()
    x_lu = np.linalg.solve(A, bhat_independent(nx, ny, nz, None, g).ravel())
    res = oracle_mod.solve(nx, ny, nz, [0, 4, 8], [0, 3, 7], [0, 3, 6], bnd=g, outer_tol=1e-12, inner="gmres",
                           restart=10)
    assert res["status"] == 0
    assert np.linalg.norm(res["x"].ravel() - x_lu) <= np.linalg.cond(A) * 1e-12 * np.linalg.norm(x_lu)


def test_gmres_exact_inner_solves_are_block_jacobi(oracle_mod):
    """Inner GMRES to full accuracy is the same exact block Jacobi as inner CG."""
    nx, ny, nz = 8, 6, 6
    g = rng(38).standard_normal(inputs.boundary_size(nx, ny, nz))
    cuts = ([0, 4, 8], [0, 3, 6], [0, 3, 6])
    a = oracle_mod.solve(nx, ny, nz, *cuts, bnd=g, inner_rtol=1e-14, inner_maxit=500, outer_tol=0.0, outer_maxit=3)
    b = oracle_mod.solve(nx, ny, nz, *cuts, bnd=g, inner_rtol=1e-14, inner_maxit=500, outer_tol=0.0, outer_maxit=3,
                         inner="gmres", restart=60)
    np.testing.assert_allclose(b["x"], a["x"], rtol=1e-10, atol=1e-11)
