"""Gradient of L = g^T A~ x with respect to the points and the kernel bandwidth,
with the pivots held fixed (oracle; TEST INFRASTRUCTURE ONLY: the tests use it to
check the CUDA adjoint kernels, the product never imports it).

A~ is the H^2 matrix of a built oracle handle (symmetric shortcut of Sec. 5,
P = Q): near blocks A_XY = K(p_X, p_Y) for leaves Y in N(X) (Sec. 3 step 3),
and far blocks U_X S_XY U_Y^T for Y in IL(X) (Sec. 3 step 2), with
S_XY = K(p_{t^{X,i}}, p_{t^{Y,i}}) and the nested bases of Sec. 2.3.1: per cell
the operator X_B = A_{t~ sigma} (A_{tau sigma})^{-1} (Eqs. 11 and 14), U_B = X_B
for a leaf and U_B = blockdiag(U_c) X_B for a non-leaf. "Pivots held fixed" means
every index set (tree, lists, tau, sigma, t~) stays as built and only the entries
K(p_i, p_j) move with the points.

Reverse mode, in the order of the product (Sec. 4):
  1. the upward pass w_B(v) = U_B^T v_B for v = x and v = g, and the downward
     pass u_B(v) = sum_{Y in IL(B)} S_BY w_Y(v) + (the parent's translation of
     the parent's u): u_B(g) is dL/dw_B(x), u_B(x) is dL/dw_B(g);
  2. near blocks: dL/dp_k += sum_j grad_a K(p_k, p_j) (g_k x_j + x_k g_j);
  3. interaction blocks: for a pivot a of cell B at point k,
     dL/dp_k += sum_{Y in IL(B)} sum_b grad_a K(p_k, p_{tau_Y b})
                (w_B(g)_a w_Y(x)_b + w_B(x)_a w_Y(g)_b);
  4. bases: with G_B = dL/dX_B = z_B(x) u_B(g)^T + z_B(g) u_B(x)^T, z_B(v) the
     vector X_B multiplies upward (v on the leaf's points, or the children's
     multipoles stacked in candidate order), and dX = (dA_{t~ sigma} - X dA_{tau sigma})
     A_{tau sigma}^{-1}: H = G A_{tau sigma}^{-T}, the entries A_{t~ sigma} take the
     adjoint H and the entries A_{tau sigma} take -X^T H; each entry K(p_i, p_j)
     passes its adjoint times grad_a K to p_i and times grad_b K = -grad_a K to p_j.
The same sums with dK/dh in place of grad K give dL/dh. Diagonal entries are a
constant (the configured value) and carry no derivative; two distinct points at
r = 0 carry none either.
"""
from __future__ import annotations

import numpy as np

from .oracle import K_GAUSS, K_INV_R, K_LOG, K_MATERN


def radial_kernel_derivatives(cfg, X: np.ndarray, Y: np.ndarray):
    """K(X_i, Y_j), grad_a K (n_x x n_y x d) and dK/dh for K = s f(r), r = |X_i - Y_j|.

    f(r) = log r, 1/r, exp(-r^2 / (2 h^2)) or exp(-r / h); f'(r) and df/dh by
    differentiation of those definitions; 0 where r = 0."""
    s, h = float(cfg.kparam[0]), float(cfg.kparam[1])
    D = X[:, None, :] - Y[None, :, :]
    r2 = np.einsum("ijk,ijk->ij", D, D)
    r = np.sqrt(r2)
    nz = r > 0
    rs = np.where(nz, r, 1.0)
    if cfg.kernel == K_LOG:
        f = np.log(rs)
        fp = 1.0 / rs
        fh = np.zeros_like(r)
    elif cfg.kernel == K_INV_R:
        f = 1.0 / rs
        fp = -1.0 / (rs * rs)
        fh = np.zeros_like(r)
    elif cfg.kernel == K_GAUSS:
        f = np.exp(-r2 / (2.0 * h * h))
        fp = -r / (h * h) * f
        fh = r2 / (h ** 3) * f
        nz = np.ones_like(nz)          # smooth at r = 0: K(0) = s, gradient 0
    elif cfg.kernel == K_MATERN:
        f = np.exp(-r / h)
        fp = -f / h
        fh = r / (h * h) * f
        nz = np.ones_like(nz)
    else:
        raise ValueError("gradients are defined for the log, 1/r, Gaussian and Matern kernels")
    K = np.where(nz, s * f, 0.0)
    # grad_a f(|a - b|) = f'(r) (a - b) / r
    gK = np.where((r > 0)[..., None], (s * fp / rs)[..., None] * D, 0.0)
    hK = np.where(nz, s * fh, 0.0)
    return K, gK, hK


def _entries(h, rows, cols):
    """K, grad_a K and dK/dh over sorted positions rows x cols, diagonal by index."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    K, gK, hK = radial_kernel_derivatives(h.cfg, h.x[rows], h.x[cols])
    diag = rows[:, None] == cols[None, :]
    K[diag] = h.cfg.kparam[2]
    gK[diag] = 0.0
    hK[diag] = 0.0
    return K, gK, hK


def _child_slices(h, c):
    """Row ranges of cell c's operator that belong to each child (candidate order)."""
    out, r0 = [], 0
    for cc in range(int(h.cch_beg[c]), int(h.cch_end[c])):
        rc = int(h.piv_off[cc + 1] - h.piv_off[cc])
        out.append((cc, r0, r0 + rc))
        r0 += rc
    return out


def h2_loss_gradient(h, x: np.ndarray, g: np.ndarray):
    """(L, dL/dP in the caller's point order (n x d), dL/dh) for L = g^T A~ x."""
    n, d = h.n, h.d
    xs = np.asarray(x, dtype=np.float64)[h.perm]
    gs = np.asarray(g, dtype=np.float64)[h.perm]
    kappa, lmin = h.kappa, h.lmin
    leaf = lambda c: h.level_of(c) == kappa
    # 1. upward and downward passes for x and g
    w = {0: {}, 1: {}}
    for l in range(kappa, lmin - 1, -1):
        for c in h.level_cells(l):
            X = h.operator(c)
            for t, v in ((0, xs), (1, gs)):
                if l == kappa:
                    z = v[h.cbeg[c]:h.cend[c]]
                else:
                    z = np.concatenate([w[t][cc] for cc, _, _ in _child_slices(h, c)]) if X.shape[0] else np.zeros(0)
                w[t][c] = X.T @ z
    u = {0: {}, 1: {}}
    L = 0.0
    for l in range(lmin, kappa + 1):
        for c in h.level_cells(l):
            r = int(h.piv_off[c + 1] - h.piv_off[c])
            for t in (0, 1):
                acc = np.zeros(r)
                for Y in h.il(c):
                    S = _entries(h, h.pivots(c), h.pivots(Y))[0]
                    acc += S @ w[t][Y]
                u[t][c] = acc
            if l > lmin:
                P = int(h.cpar[c])
                for cc, a0, a1 in _child_slices(h, P):
                    if cc == c:
                        XP = h.operator(P)
                        for t in (0, 1):
                            u[t][c] = u[t][c] + XP[a0:a1] @ u[t][P]
    grad = np.zeros((n, d))
    dh = 0.0
    # near field (and the loss)
    for c in h.level_cells(kappa):
        rows = np.arange(h.cbeg[c], h.cend[c])
        cols = np.concatenate([np.arange(h.cbeg[Y], h.cend[Y]) for Y in h.nb(c)])
        K, gK, hK = _entries(h, rows, cols)
        L += gs[rows] @ K @ xs[cols]
        wgt = gs[rows][:, None] * xs[cols][None, :] + xs[rows][:, None] * gs[cols][None, :]
        grad[rows] += np.einsum("ij,ijk->ik", wgt, gK)
        dh += float(gs[rows] @ hK @ xs[cols])
    # interaction lists
    for l in range(lmin, kappa + 1):
        for c in h.level_cells(l):
            tc = h.pivots(c)
            for Y in h.il(c):
                K, gK, hK = _entries(h, tc, h.pivots(Y))
                L += w[1][c] @ K @ w[0][Y]
                wgt = np.outer(w[1][c], w[0][Y]) + np.outer(w[0][c], w[1][Y])
                np.add.at(grad, tc, np.einsum("ab,abk->ak", wgt, gK))
                dh += float(w[1][c] @ hK @ w[0][Y])
    # bases
    for l in range(kappa, lmin - 1, -1):
        for c in h.level_cells(l):
            if h.passthru[c]:
                continue
            X = h.operator(c)
            m, r = X.shape
            if r == 0:
                continue
            if l == kappa:
                z = [xs[h.cbeg[c]:h.cend[c]], gs[h.cbeg[c]:h.cend[c]]]
            else:
                z = [np.concatenate([w[t][cc] for cc, _, _ in _child_slices(h, c)]) for t in (0, 1)]
            G = np.outer(z[0], u[1][c]) + np.outer(z[1], u[0][c])
            tau, sig, cand = h.pivots(c), h.colpivots(c), h.candidates(c)
            M = _entries(h, tau, sig)[0]
            H = np.linalg.solve(M, G.T).T           # H = G M^{-T}
            Mbar = -(X.T @ H)
            for rows, adj in ((cand, H), (tau, Mbar)):
                _, gK, hK = _entries(h, rows, sig)
                contrib = adj[..., None] * gK
                np.add.at(grad, rows, contrib.sum(axis=1))
                np.add.at(grad, sig, -contrib.sum(axis=0))
                dh += float(np.sum(adj * hK))
    out = np.zeros((n, d))
    out[h.perm] = grad
    return float(L), out, dh


def dense_loss_gradient(P: np.ndarray, cfg, x: np.ndarray, g: np.ndarray, rows_per_block: int = 256):
    """(L, dL/dP, dL/dh) of the dense L = g^T A x, A(i, j) = K(p_i, p_j), A(i, i) fixed,
    by blocks of rows (the same sums, bounded memory)."""
    P = np.asarray(P, dtype=np.float64)
    n = P.shape[0]
    L, dh = 0.0, 0.0
    grad = np.zeros_like(P)
    for i0 in range(0, n, rows_per_block):
        i1 = min(n, i0 + rows_per_block)
        K, gK, hK = radial_kernel_derivatives(cfg, P[i0:i1], P)
        idx = np.arange(i0, i1)
        K[idx - i0, idx] = cfg.kparam[2]
        gK[idx - i0, idx] = 0.0
        hK[idx - i0, idx] = 0.0
        L += float(g[i0:i1] @ K @ x)
        wgt = g[i0:i1, None] * x[None, :] + x[i0:i1, None] * g[None, :]
        grad[i0:i1] = np.einsum("ij,ijk->ik", wgt, gK)
        dh += float(g[i0:i1] @ hK @ x)
    return L, grad, dh
