"""The NNCA representation of A(P, Q) for distinct point sets (oracle; TEST
INFRASTRUCTURE ONLY: the tests use it as the reference form of Sec. 2.3 for P != Q;
the product never imports it).

Sec. 2.3 gives every cell B four pivot sets: the incoming row and column pivots
t^{B,i} (points of P in B) and s^{B,i} (points of Q in the far field of B), and the
outgoing row and column pivots t^{B,o} (points of P in the far field) and s^{B,o}
(points of Q in B). With them (Eq. 12 and its nested form)

    A(t^X, s^Y) ~ U_X S_{X,Y} V_Y^T,   U_X = A(t^X, s^{X,i}) A(t^{X,i}, s^{X,i})^{-1},
    S_{X,Y} = A(t^{X,i}, s^{Y,o}),     V_Y^T = A(t^{Y,o}, s^{Y,o})^{-1} A(t^{Y,o}, s^Y)

for Y in IL(X). The pivots come bottom-up from two ACAs per cell (Sec. 2.3.2) on the
candidate sets of Eqs. 15-18:
  leaf B:     t~^{B,i} = t^B (P in B),           s~^{B,i} = Q in the cells of IL(B),
              t~^{B,o} = P in the cells of IL(B), s~^{B,o} = s^B (Q in B);
  non-leaf B: t~^{B,i} = children's t^{C,i},     s~^{B,i} = s^{B'',o} of the children
              B'' of the cells B' in IL(B),       t~^{B,o} = t^{B'',i} of those children,
              s~^{B,o} = children's s^{C,o}.
The ACA on A(t~^{B,i}, s~^{B,i}) gives t^{B,i} (rows) and s^{B,i} (columns); the ACA
on A(t~^{B,o}, s~^{B,o}) gives t^{B,o} (rows) and s^{B,o} (columns). The bases over
the candidates: U_B = A(t~^{B,i}, s^{B,i}) A(t^{B,i}, s^{B,i})^{-1} (for a non-leaf the
stacked translations to its children) and V_B^T = A(t^{B,o}, s^{B,o})^{-1}
A(t^{B,o}, s~^{B,o}). The product (Sec. 4): upward w_B = V_B^T z_B (z_B: x on s^B, or
the children's w stacked), transverse u_X += S_{X,Y} w_Y over Y in IL(X), downward
u_C += (rows of U_P for C) u_P, and at a leaf y(t^B) = U_B u_B + the near blocks
A(t^B, s^{B'}) x(s^{B'}) over B' in N(B).

Readings, as in the symmetric oracle: the tree and lists are those of the union [P; Q]
(one cube holding both sets, Sec. 2.1); candidate sets in Morton order of the cells, each
cell's pivots in selection order, leaf sets in sorted point order; levels above the
first with an interaction list take no pivots; pass-through (a cell whose far-field
candidates cannot determine its basis keeps all its candidates with an identity basis):
incoming when s~^{B,i} is empty or the ACA uses up every column of it while rows
remain, outgoing when t~^{B,o} is empty or the ACA uses up every row of it while
columns remain. Entries K(p_i, q_j) with no diagonal rule (distinct sets).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


class H2PQ:
    """The representation of A(P, Q) (P: n x d targets, Q: m x d sources)."""

    def __init__(self, P: np.ndarray, Q: np.ndarray, cfg: O.Config):
        P = np.ascontiguousarray(P, dtype=np.float64)
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        self.cfg, self.n, self.m = cfg, P.shape[0], Q.shape[0]
        t = O.H2(np.vstack([P, Q]), cfg, structure_only=True)
        self.t = t
        self.X = t.x                                     # union points in sorted order
        is_p = t.perm < self.n
        # per cell: sorted positions of its P points and of its Q points
        self.tB = [np.arange(t.cbeg[c], t.cend[c])[is_p[t.cbeg[c]:t.cend[c]]] for c in range(t.ncell)]
        self.sB = [np.arange(t.cbeg[c], t.cend[c])[~is_p[t.cbeg[c]:t.cend[c]]] for c in range(t.ncell)]
        nc = t.ncell
        empty = np.zeros(0, dtype=np.int64)
        self.ti, self.si = [empty] * nc, [empty] * nc      # incoming row / column pivots
        self.to, self.so = [empty] * nc, [empty] * nc      # outgoing row / column pivots
        self.tci, self.sco = [empty] * nc, [empty] * nc    # candidate rows (incoming), columns (outgoing)
        self.U = [np.zeros((0, 0))] * nc                   # |t~^{B,i}| x |t^{B,i}|
        self.V = [np.zeros((0, 0))] * nc                   # |s~^{B,o}| x |s^{B,o}|  (V_B; V_B^T is applied)
        eps = cfg.aca_tol
        first = self._first_il_level()
        for l in range(t.kappa, first - 1, -1):
            for c in t.level_cells(l):
                leaf = l == t.kappa
                il = t.il(c)
                ch = range(int(t.cch_beg[c]), int(t.cch_end[c]))
                if leaf:
                    tci = self.tB[c]
                    sci = np.concatenate([self.sB[y] for y in il] + [empty])
                    tco = np.concatenate([self.tB[y] for y in il] + [empty])
                    sco = self.sB[c]
                else:
                    tci = np.concatenate([self.ti[k] for k in ch] + [empty])
                    sci = np.concatenate([self.so[k] for y in il for k in self._children(y)] + [empty])
                    tco = np.concatenate([self.ti[k] for y in il for k in self._children(y)] + [empty])
                    sco = np.concatenate([self.so[k] for k in ch] + [empty])
                self.tci[c], self.sco[c] = tci, sco
                self._incoming(c, tci, sci, eps)
                self._outgoing(c, tco, sco, eps)

    # --- build -----------------------------------------------------------
    def _children(self, c):
        return range(int(self.t.cch_beg[c]), int(self.t.cch_end[c]))

    def _first_il_level(self) -> int:
        t = self.t
        for l in range(t.lmin, t.kappa + 1):
            if any(len(t.il(c)) for c in t.level_cells(l)):
                return l
        return t.kappa + 1

    def _K(self, rows, cols) -> np.ndarray:
        return O.kernel_block(self.cfg, self.X[rows], self.X[cols])

    def _incoming(self, c, tci, sci, eps):
        if len(tci) == 0:
            return
        if len(sci) == 0:
            self.ti[c], self.U[c] = tci, np.eye(len(tci))
            return
        pr, pc, _, _ = O.aca_dense(self._K(tci, sci), eps)
        if len(pc) == len(sci) < len(tci):
            self.ti[c], self.U[c] = tci, np.eye(len(tci))
            return
        tau, sig = tci[pr], sci[pc]
        X = O.solve_right(self._K(tau, sig), self._K(tci, sig)) if len(pr) else np.zeros((len(tci), 0))
        X[pr, :] = np.eye(len(pr))                       # the pivot rows are the identity by definition
        self.ti[c], self.si[c], self.U[c] = tau, sig, X

    def _outgoing(self, c, tco, sco, eps):
        if len(sco) == 0:
            return
        if len(tco) == 0:
            self.so[c], self.V[c] = sco, np.eye(len(sco))
            return
        pr, pc, _, _ = O.aca_dense(self._K(tco, sco), eps)
        if len(pr) == len(tco) < len(sco):
            self.so[c], self.V[c] = sco, np.eye(len(sco))
            return
        tau, sig = tco[pr], sco[pc]
        # V^T = A(tau, sig)^{-1} A(tau, s~): V = A(tau, s~)^T A(tau, sig)^{-T}, solved as V M^T = B^T
        V = O.solve_right(self._K(tau, sig).T.copy(), self._K(tau, sco).T.copy()) if len(pr) else np.zeros((len(sco), 0))
        V[pc, :] = np.eye(len(pc))
        self.to[c], self.so[c], self.V[c] = tau, sig, V

    # --- product ---------------------------------------------------------
    def matvec(self, x: np.ndarray) -> np.ndarray:
        """y = A~(P, Q) x, x on Q (m,), y on P (n,), both in the caller's order."""
        t = self.t
        x = np.asarray(x, dtype=np.float64)
        xs = np.zeros(t.n)
        q = t.perm >= self.n
        xs[q] = x[t.perm[q] - self.n]
        first = self._first_il_level()
        w = {}
        for l in range(t.kappa, first - 1, -1):
            for c in t.level_cells(l):
                if len(self.sco[c]) == 0:
                    w[c] = np.zeros(0)
                    continue
                z = xs[self.sco[c]] if l == t.kappa else np.concatenate([w[k] for k in self._children(c)])
                w[c] = self.V[c].T @ z
        u = {}
        ys = np.zeros(t.n)
        for l in range(first, t.kappa + 1):
            for c in t.level_cells(l):
                acc = np.zeros(len(self.ti[c]))
                for y in t.il(c):
                    if len(self.so[y]) and len(acc):
                        acc += self._K(self.ti[c], self.so[y]) @ w[y]
                if l > first:
                    p = int(t.cpar[c])
                    off = 0
                    for k in self._children(p):
                        r = len(self.ti[k])
                        if k == c and r:
                            acc += self.U[p][off:off + r] @ u[p]
                        off += r
                u[c] = acc
                if l == t.kappa and len(self.tB[c]):
                    yt = self.U[c] @ acc if len(acc) else np.zeros(len(self.tB[c]))
                    for b in t.nb(c):
                        if len(self.sB[b]):
                            yt = yt + self._K(self.tB[c], self.sB[b]) @ xs[self.sB[b]]
                    ys[self.tB[c]] = yt
        out = np.zeros(self.n)
        pmask = t.perm < self.n
        out[t.perm[pmask]] = ys[pmask]
        return out

    def ranks(self):
        """(incoming pivots, outgoing pivots) summed over the cells."""
        return int(sum(len(a) for a in self.ti)), int(sum(len(a) for a in self.so))
