"""Pins for the oracle's gradient of L = g^T A~ x with the pivots held fixed
(oracle/grad.py): the loss it carries equals the oracle's H^2 product; central
finite differences (step 1e-4, FP64, one Richardson step) of an independently
assembled loss, the H^2 matrix written out from bases recomputed at the moved
points (Eqs. 11 and 14 with the index sets held), match it; and it approaches
the gradient of the dense L = g^T A x as the ACA tolerance falls.
"""
import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W

STEP = 1e-4


def assembled_loss(orc, h, cfg, Ps, xs, gs):
    """g^T A~ x for the points Ps (sorted order) and kernel cfg with every index
    set of h held: bases X_B = A_{t~ sigma}(Ps) A_{tau sigma}(Ps)^{-1} (identity for
    pass-through cells), column bases U_B nested as blockdiag(U_c) X_B, far blocks
    U_X S_XY U_Y^T, near blocks exact, all written out as one dense matrix."""
    Afull = orc.kernel_block(cfg, Ps, Ps)
    np.fill_diagonal(Afull, cfg.kparam[2])

    def A(rows, cols):
        return Afull[np.ix_(np.asarray(rows, dtype=np.int64), np.asarray(cols, dtype=np.int64))]

    U = {}
    for l in range(h.kappa, h.lmin - 1, -1):
        for c in h.level_cells(l):
            cand, tau, sig = h.candidates(c), h.pivots(c), h.colpivots(c)
            m, r = len(cand), len(tau)
            if h.passthru[c]:
                Xc = np.eye(m)
            elif r == 0:
                Xc = np.zeros((m, 0))
            else:
                Xc = np.linalg.solve(A(tau, sig).T, A(cand, sig).T).T
            if l == h.kappa:
                U[c] = Xc
            else:
                blocks, r0 = [], 0
                for cc in range(h.cch_beg[c], h.cch_end[c]):
                    rc = U[cc].shape[1]
                    blocks.append(U[cc] @ Xc[r0:r0 + rc])
                    r0 += rc
                U[c] = np.vstack(blocks) if blocks else np.zeros((0, r))
    n = h.n
    M = np.zeros((n, n))
    for c in range(h.ncell):
        tX = slice(h.cbeg[c], h.cend[c])
        for Y in h.il(c):
            M[tX, h.cbeg[Y]:h.cend[Y]] += U[c] @ A(h.pivots(c), h.pivots(Y)) @ U[Y].T
        if h.level_of(c) == h.kappa:
            for Y in h.nb(c):
                M[tX, h.cbeg[Y]:h.cend[Y]] += Afull[tX, h.cbeg[Y]:h.cend[Y]]
    return float(gs @ M @ xs)


CASES = [
    # name, points, d, leaf size, kernel, kparam, ACA tolerance
    ("invr2d", lambda: W.uniform_cube(500, 2, 11), 2, 8, W.K_INV_R, (1.0, 0.0, 0.0, 0.0), 1e-6),
    ("log2d", lambda: W.uniform_cube(500, 2, 13, -1.0, 1.0), 2, 8, W.K_LOG, (1.0, 0.0, 0.0, 0.0), 1e-8),
    ("gauss3d", lambda: W.gaussian_mixture(500, 3, 12), 3, 8, W.K_GAUSS, (1.0, 0.2, 1.0, 0.0), 1e-6),
    ("invr3d", lambda: W.uniform_cube(500, 3, 15), 3, 8, W.K_INV_R, (1.0, 0.0, 0.0, 0.0), 1e-6),
]


def build(orc, P, d, nu, kernel, kparam, eps):
    cfg = orc.Config(d=d, leaf_size=nu, aca_tol=eps, kernel=kernel, kparam=kparam)
    return orc.H2(P, cfg), cfg


@pytest.mark.parametrize("name,make,d,nu,kernel,kparam,eps", CASES, ids=[c[0] for c in CASES])
def test_gradient_against_finite_differences(orc, name, make, d, nu, kernel, kparam, eps):
    from oracle import grad as G
    P = make()
    n = P.shape[0]
    h, cfg = build(orc, P, d, nu, kernel, kparam, eps)
    assert h.lmin < h.kappa and int(h.il_off[-1]) > 0
    x = W.vector_normal(n, 21)
    g = W.vector_normal(n, 22)
    L, dP, dh = G.h2_loss_gradient(h, x, g)
    # the loss is the oracle's product
    assert abs(L - g @ h.matvec(x)) <= 1e-12 * abs(L)
    Ps, xs, gs = h.x.copy(), x[h.perm], g[h.perm]
    assert abs(assembled_loss(orc, h, cfg, Ps, xs, gs) - L) <= 1e-12 * abs(L)
    inv = np.empty(n, dtype=np.int64)
    inv[h.perm] = np.arange(n)
    rng = np.random.default_rng(5)
    scale = np.max(np.abs(dP))

    def fd(i_sorted, k, step):
        Pp, Pm = Ps.copy(), Ps.copy()
        Pp[i_sorted, k] += step
        Pm[i_sorted, k] -= step
        return (assembled_loss(orc, h, cfg, Pp, xs, gs) - assembled_loss(orc, h, cfg, Pm, xs, gs)) / (2 * step)

    for i in rng.choice(n, 8, replace=False):
        k = int(rng.integers(d))
        d1, d2 = fd(inv[i], k, STEP), fd(inv[i], k, STEP / 2)
        est = (4 * d2 - d1) / 3
        assert abs(est - dP[i, k]) <= 1e-6 * scale, (i, k, est, dP[i, k])
    if kernel == W.K_GAUSS:
        def loss_h(hv):
            c2 = orc.Config(d=d, leaf_size=nu, aca_tol=eps, kernel=kernel, kparam=(kparam[0], hv, kparam[2], 0.0))
            return assembled_loss(orc, h, c2, Ps, xs, gs)

        e1 = (loss_h(kparam[1] + STEP) - loss_h(kparam[1] - STEP)) / (2 * STEP)
        e2 = (loss_h(kparam[1] + STEP / 2) - loss_h(kparam[1] - STEP / 2)) / STEP
        assert abs((4 * e2 - e1) / 3 - dh) <= 1e-7 * abs(dh)


def test_gradient_approaches_dense(orc):
    """The H^2 gradient (pivots fixed) converges to the gradient of the dense
    loss as the ACA tolerance falls (Sec. 5.1-5.2 for the product itself)."""
    from oracle import grad as G
    P = W.gaussian_mixture(900, 3, 14)
    kp = (1.0, 0.2, 1.0, 0.0)
    x = W.vector_normal(900, 23)
    g = W.vector_normal(900, 24)
    cfg = orc.Config(d=3, leaf_size=16, aca_tol=1e-6, kernel=W.K_GAUSS, kparam=kp)
    Ld, dPd, dhd = G.dense_loss_gradient(P, cfg, x, g)
    errs, errh = [], []
    for eps in (1e-3, 1e-5, 1e-7, 1e-9):
        h, _ = build(orc, P, 3, 16, W.K_GAUSS, kp, eps)
        L, dP, dh = G.h2_loss_gradient(h, x, g)
        errs.append(np.linalg.norm(dP - dPd) / np.linalg.norm(dPd))
        errh.append(abs(dh - dhd) / abs(dhd))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6 and errh[-1] < 1e-6, (errs, errh)


def test_dense_gradient_closed_form(orc):
    """The dense gradient of two points: dL/dp_0 = f'(r) (p_0 - p_1)/r (g_0 x_1 + x_0 g_1)."""
    from oracle import grad as G
    P = np.array([[0.1, 0.2, 0.3], [0.4, -0.2, 0.7]])
    x, g = np.array([0.5, -1.5]), np.array([2.0, 0.25])
    for kernel, kp in ((W.K_INV_R, (2.0, 0, 0, 0)), (W.K_GAUSS, (1.5, 0.3, 1.5, 0))):
        cfg = orc.Config(d=3, kernel=kernel, kparam=kp)
        L, dP, dh = G.dense_loss_gradient(P, cfg, x, g)
        dvec = P[0] - P[1]
        r = np.linalg.norm(dvec)
        if kernel == W.K_INV_R:
            fp, K01, kh = -kp[0] / r ** 2, kp[0] / r, 0.0
        else:
            K01 = kp[0] * np.exp(-r * r / (2 * kp[1] ** 2))
            fp, kh = -r / kp[1] ** 2 * K01, r * r / kp[1] ** 3 * K01
        wgt = g[0] * x[1] + x[0] * g[1]
        assert np.allclose(dP[0], fp * dvec / r * wgt, rtol=1e-14)
        assert np.allclose(dP[1], -fp * dvec / r * wgt, rtol=1e-14)
        assert abs(L - (g @ np.array([[kp[2], K01], [K01, kp[2]]]) @ x)) < 1e-13
        assert abs(dh - kh * wgt) < 1e-13
