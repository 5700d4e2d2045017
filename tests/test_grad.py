"""GPU adjoint kernels (nnca_gradient, autograd) against the oracle: the gradient
of L = g^T A~ x in the points and in the kernel bandwidth with the pivots held
fixed, through the C ABI.

  - against the oracle's H^2 gradient (oracle/grad.py, itself pinned by finite
    differences): FP64 on both sides, within 1e-8 of max |dL/dP| (the two sides
    sum in different orders, and the solves with the pivot blocks, condition
    about 1/eps, amplify that);
  - against central finite differences (step 1e-4, FP64, one Richardson step) of
    the assembled H^2 loss with the index sets held;
  - against the dense-oracle gradient on a 4096-point Gaussian-mixture subset of
    the 64-RHS workload's recipe: within 3e-5 (measured on the oracle: 1.1e-5,
    the H^2 approximation at eps = 1e-6), and dL/dh within 3e-6;
  - through torch.autograd: x.grad = A~ g, points.grad and bandwidth.grad equal
    the oracle's, summed over two right-hand sides.
"""
import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def gpu_grad(gpu, torch, g_h, X, G):
    n, d = g_h.n, g_h.cfg.d
    Xd = torch.as_tensor(np.ascontiguousarray(X), device="cuda")
    Gd = torch.as_tensor(np.ascontiguousarray(G), device="cuda")
    nrhs = 1 if X.ndim == 1 else X.shape[0]
    gp = torch.empty((n, d), dtype=torch.float64, device="cuda")
    gh = torch.zeros(1, dtype=torch.float64, device="cuda")
    gpu.nnca_gradient(g_h.handle, Xd, Gd, nrhs, n, gp, gh)
    return gp.cpu().numpy(), float(gh.item())


CASES = [
    ("invr2d", lambda: W.uniform_cube(2000, 2, 11), 2, 16, W.K_INV_R, (1.0, 0.0, 0.0, 0.0), 1e-6),
    ("log2d", lambda: W.uniform_cube(2000, 2, 13, -1.0, 1.0), 2, 16, W.K_LOG, (1.0, 0.0, 0.0, 0.0), 1e-8),
    ("gauss3d", lambda: W.gaussian_mixture(1200, 3, 12), 3, 16, W.K_GAUSS, (1.0, 0.2, 1.0, 0.0), 1e-6),
    ("invr3d", lambda: W.uniform_cube(2000, 3, 15), 3, 16, W.K_INV_R, (1.0, 0.0, 0.0, 0.0), 1e-6),
]


@pytest.mark.parametrize("name,make,d,nu,kernel,kparam,eps", CASES, ids=[c[0] for c in CASES])
def test_gradient_matches_oracle(gpu, orc, name, make, d, nu, kernel, kparam, eps):
    import torch
    from oracle import grad as G
    P = make()
    n = P.shape[0]
    c = dict(d=d, leaf_size=nu, aca_tol=eps, kernel=kernel, kparam=kparam)
    g_h = gpu.H2(torch.as_tensor(P, device="cuda"), gpu.Config(**c))
    o = orc.H2(P, orc.Config(**c))
    assert np.array_equal(g_h.export("PIV_ROW"), o.piv_row)
    x, g = W.vector_normal(n, 31), W.vector_normal(n, 32)
    L, dP, dh = G.h2_loss_gradient(o, x, g)
    gp, gh = gpu_grad(gpu, torch, g_h, x, g)
    assert np.max(np.abs(gp - dP)) <= 1e-8 * np.max(np.abs(dP))
    if kernel == W.K_GAUSS:
        assert abs(gh - dh) <= 1e-8 * abs(dh)
    else:
        assert gh == 0.0
    assert g_h.stats()["device_status"] & (2 | 4 | 16) == 0
    g_h.close()


def test_gradient_against_finite_differences(gpu, orc):
    import torch
    from test_oracle_grad import assembled_loss
    P = W.gaussian_mixture(500, 3, 12)
    c = dict(d=3, leaf_size=8, aca_tol=1e-6, kernel=W.K_GAUSS, kparam=(1.0, 0.2, 1.0, 0.0))
    g_h = gpu.H2(torch.as_tensor(P, device="cuda"), gpu.Config(**c))
    o = orc.H2(P, orc.Config(**c))
    x, g = W.vector_normal(500, 35), W.vector_normal(500, 36)
    gp, gh = gpu_grad(gpu, torch, g_h, x, g)
    Ps, xs, gs = o.x.copy(), x[o.perm], g[o.perm]
    inv = np.empty(500, dtype=np.int64)
    inv[o.perm] = np.arange(500)
    rng = np.random.default_rng(7)
    step = 1e-4

    def fd(i, k, s):
        Pp, Pm = Ps.copy(), Ps.copy()
        Pp[inv[i], k] += s
        Pm[inv[i], k] -= s
        return (assembled_loss(orc, o, o.cfg, Pp, xs, gs) - assembled_loss(orc, o, o.cfg, Pm, xs, gs)) / (2 * s)

    for i in rng.choice(500, 6, replace=False):
        k = int(rng.integers(3))
        est = (4 * fd(i, k, step / 2) - fd(i, k, step)) / 3
        assert abs(est - gp[i, k]) <= 1e-6 * np.max(np.abs(gp)), (i, k, est, gp[i, k])

    def loss_h(hv):
        cfg2 = orc.Config(d=3, leaf_size=8, aca_tol=1e-6, kernel=W.K_GAUSS, kparam=(1.0, hv, 1.0, 0.0))
        return assembled_loss(orc, o, cfg2, Ps, xs, gs)

    e1 = (loss_h(0.2 + step) - loss_h(0.2 - step)) / (2 * step)
    e2 = (loss_h(0.2 + step / 2) - loss_h(0.2 - step / 2)) / step
    assert abs((4 * e2 - e1) / 3 - gh) <= 1e-7 * abs(gh)
    g_h.close()


def test_gradient_against_dense_4096(gpu, orc):
    """4096 points of the 64-RHS Gaussian-mixture recipe (leaf size 64, eps 1e-6, h = 0.2)."""
    import torch
    from oracle import grad as G
    w = W.WORKLOADS["gauss_mix_256k"].scaled(4096)
    P = w.make_points()
    c = dict(d=3, leaf_size=w.leaf_size, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    g_h = gpu.H2(torch.as_tensor(P, device="cuda"), gpu.Config(**c))
    x, g = W.vector_normal(4096, 61), W.vector_normal(4096, 62)
    gp, gh = gpu_grad(gpu, torch, g_h, x, g)
    Ld, dPd, dhd = G.dense_loss_gradient(P, orc.Config(**c), x, g)
    assert np.linalg.norm(gp - dPd) / np.linalg.norm(dPd) < 3e-5
    assert abs(gh - dhd) / abs(dhd) < 3e-6
    g_h.close()


def test_autograd_points_bandwidth_and_x(gpu, orc):
    import torch
    from paper_2203_14832_gb300 import autograd as AG
    from oracle import grad as G
    P = W.gaussian_mixture(800, 3, 17)
    c = dict(d=3, leaf_size=16, aca_tol=1e-7, kernel=W.K_GAUSS, kparam=(1.0, 0.2, 1.0, 0.0))
    Pd = torch.as_tensor(P, device="cuda").requires_grad_(True)
    hb = torch.tensor(0.2, dtype=torch.float64, device="cuda", requires_grad=True)
    g_h = gpu.H2(Pd.detach(), gpu.Config(**c))
    X = torch.as_tensor(W.vector_normal(800, 41, nrhs=2), device="cuda").requires_grad_(True)
    Gv = torch.as_tensor(W.vector_normal(800, 42, nrhs=2), device="cuda")
    y = AG.h2_matvec(g_h, X, gpu.PREC_FP64, points=Pd, bandwidth=hb)
    (y * Gv).sum().backward()
    o = orc.H2(P, orc.Config(**c))
    Xn, Gn = X.detach().cpu().numpy(), Gv.cpu().numpy()
    parts = [G.h2_loss_gradient(o, Xn[r], Gn[r]) for r in range(2)]
    refP = parts[0][1] + parts[1][1]
    refh = parts[0][2] + parts[1][2]
    assert np.max(np.abs(Pd.grad.cpu().numpy() - refP)) <= 1e-8 * np.max(np.abs(refP))
    assert abs(float(hb.grad) - refh) <= 1e-8 * abs(refh)
    assert np.allclose(X.grad.cpu().numpy(), o.matvec(Gn), rtol=0, atol=1e-11 * np.abs(o.matvec(Gn)).max())
    g_h.close()
