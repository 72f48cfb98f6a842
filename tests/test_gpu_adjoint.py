"""Adjoint of ms_solve (torch.autograd.Function MsSolve).

L = 0.5 ||u - u_t||^2 with u = A^{-1}(f + lift(g)).  A is symmetric, so
dL/df = A^{-1}(u - u_t) and dL/dg = lift^T A^{-1}(u - u_t).  Checked against
(1) a dense-solve gradient on a small grid and (2) central finite differences
on random probes: L is quadratic, so central differences are exact up to
rounding and solver truncation for any step (solves run to outer tol 1e-12).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from paper_2009_12638_gb300 import Grid, MsSolve, inputs

pytestmark = pytest.mark.gpu


def kron_laplacian(n):
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    I = sp.identity(n)
    return (sp.kron(I, sp.kron(I, T)) + sp.kron(I, sp.kron(T, I)) + sp.kron(T, sp.kron(I, I))).tocsc()


def loss_and_grads(grid, f, g, target, opts):
    f = f.clone().requires_grad_(True)
    g = g.clone().requires_grad_(True)
    u = MsSolve.apply(f, g, grid, opts)
    L = 0.5 * ((u - target) ** 2).sum()
    L.backward()
    return float(L), f.grad.detach(), g.grad.detach()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_matches_dense_gradient(precision):
    n = 10
    c = inputs.equal_cuts(n, 2)
    r = np.random.default_rng(40)
    f = r.standard_normal((1, n, n, n))
    g = r.uniform(-1, 1, size=(1, inputs.boundary_size(n, n, n)))
    target = inputs.interior_from_function(n, n, n, inputs.adjoint_target)[None]
    grid = Grid(n, n, n, 1).partition(2, 2, 2, c, c, c)
    opts = dict(precision=precision, outer_tol=1e-13)
    L, gf, gg = loss_and_grads(grid, torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(),
                               torch.from_numpy(target).cuda(), opts)
    A = kron_laplacian(n)
    nb = inputs.boundary_size(n, n, n)
    B = np.stack([oracle.lift(n, n, n, None, np.eye(1, nb, j)[0]).ravel() for j in range(nb)], axis=1)
    u = sp.linalg.spsolve(A, f[0].ravel() + B @ g[0])
    lam = sp.linalg.spsolve(A, u - target.ravel())
    np.testing.assert_allclose(gf.cpu().numpy().ravel(), lam, rtol=0, atol=1e-9 * np.abs(lam).max())
    np.testing.assert_allclose(gg.cpu().numpy().ravel(), B.T @ lam, rtol=0, atol=1e-9 * np.abs(lam).max())
    assert L == pytest.approx(0.5 * np.sum((u - target.ravel()) ** 2), rel=1e-10)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_central_fd_probes(precision):
    cfg = inputs.make_config("adjoint128", scale=4)  # 32^3, 4x4x4 blocks of 8^3
    n = cfg["nx"]
    grid = Grid(n, n, n, 1).partition(4, 4, 4, cfg["cx"], cfg["cy"], cfg["cz"])
    f0 = torch.zeros((1, n, n, n), dtype=torch.float64, device="cuda")
    g0 = torch.from_numpy(cfg["bnd"]).cuda()
    target = torch.from_numpy(cfg["target"][None]).cuda()
    opts = dict(precision=precision, outer_tol=1e-12)
    _, gf, gg = loss_and_grads(grid, f0, g0, target, opts)
    nprobe = 16
    vf = inputs.gaussian_probes((1, n, n, n), nprobe, cfg["probe_seed"])
    vg = inputs.gaussian_probes((1, grid.nbnd), nprobe, cfg["probe_seed"] + 1)
    theta = np.sqrt(float((g0 ** 2).sum()))
    worst = 0.0
    for i in range(nprobe):
        v_f = torch.from_numpy(vf[i]).cuda()
        v_g = torch.from_numpy(vg[i]).cuda()
        eps = 1e-2 * theta / np.sqrt(float((v_f ** 2).sum() + (v_g ** 2).sum()))

        def L(s):
            u, st = grid.solve(f=f0 + s * v_f, bnd=g0 + s * v_g, **opts)
            assert st.status == 0
            return 0.5 * float(((u - target) ** 2).sum())

        fd = (L(eps) - L(-eps)) / (2 * eps)
        ad = float((gf * v_f).sum() + (gg * v_g).sum())
        worst = max(worst, abs(ad - fd) / abs(fd))
    assert worst < 1e-6, worst
