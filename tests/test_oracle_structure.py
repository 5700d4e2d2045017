"""Pins for the oracle's tree (Sec. 2.1) and lists (Sec. 2.2, Eq. 2, Table 1, Fig. 1).

Each check uses something other than the oracle's own formulas: geometric
containment and bisection for the tree, real-valued distances and diameters
for the admissibility test, the picture of Fig. 1, symmetry, and the
partition of the matrix into near blocks and admissible blocks.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cell_box(h, c):
    """Geometric box of cell c: corner + [coords, coords+1] * side / 2^l."""
    l = h.level_of(c)
    key = int(h.ckey[c])
    co = [0] * h.d
    for b in range(l):
        for k in range(h.d):
            co[k] |= ((key >> (b * h.d + k)) & 1) << b
    s = h.side / 2 ** l
    lo = h.corner + np.array(co) * s
    return lo, lo + s, np.array(co)


@pytest.mark.parametrize("n,d,nu,seed", [(3000, 2, 16, 1), (5000, 3, 32, 2), (777, 1, 8, 3), (2000, 4, 64, 4)])
def test_tree_geometry(orc, n, d, nu, seed):
    P = W.uniform_cube(n, d, seed, -1.0, 1.0)
    h = orc.H2(P, orc.Config(d=d, leaf_size=nu), structure_only=True)
    # perm is a permutation and x is P in that order
    assert sorted(h.perm.tolist()) == list(range(n))
    assert np.array_equal(h.x, P[h.perm])
    # the cube contains every point
    assert np.all(P >= h.corner - 1e-15) and np.all(P <= h.corner + h.side + 1e-15)
    # leaf level: every leaf holds <= nu points, the level above has a fuller cell
    leaves = h.level_cells(h.kappa)
    assert max(h.cend[c] - h.cbeg[c] for c in leaves) <= nu
    if h.kappa > 0:
        assert max(h.cend[c] - h.cbeg[c] for c in h.level_cells(h.kappa - 1)) > nu
    # every point lies in the box of its cell at every level (closed box, rounding slack)
    tol = 1e-12 * h.side
    for l in range(h.kappa + 1):
        for c in h.level_cells(l):
            lo, hi, _ = cell_box(h, c)
            pts = h.x[h.cbeg[c]: h.cend[c]]
            assert np.all(pts >= lo - tol) and np.all(pts <= hi + tol)
    # nesting: children partition the parent's point range, parent key = child key >> d
    for l in range(h.kappa):
        for c in h.level_cells(l):
            ch = range(h.cch_beg[c], h.cch_end[c])
            assert h.cbeg[ch[0]] == h.cbeg[c] and h.cend[ch[-1]] == h.cend[c]
            for a, b in zip(ch[:-1], ch[1:]):
                assert h.cend[a] == h.cbeg[b]
            for cc in ch:
                assert h.cpar[cc] == c and int(h.ckey[cc]) >> d == int(h.ckey[c])
    # cells are non-empty and level ranges tile the points
    for l in range(h.kappa + 1):
        cs = h.level_cells(l)
        assert h.cbeg[cs[0]] == 0 and h.cend[cs[-1]] == n
        assert all(h.cend[c] > h.cbeg[c] for c in cs)


def test_tree_bisection_brute_force(orc):
    """Cells by explicit recursive bisection of the cube agree with the tree."""
    n, d = 400, 2
    P = W.uniform_cube(n, d, 11, -1.0, 1.0)
    h = orc.H2(P, orc.Config(d=d, leaf_size=6), structure_only=True)
    for l in range(h.kappa + 1):
        for c in h.level_cells(l):
            _, _, co = cell_box(h, c)
            for p in h.x[h.cbeg[c]: h.cend[c]]:
                lo = h.corner.copy()
                s = h.side
                idx = np.zeros(d, dtype=int)
                for _ in range(l):
                    s = s / 2
                    up = p >= lo + s
                    lo = lo + s * up
                    idx = 2 * idx + up
                assert np.array_equal(idx, co)


def test_sorted_order_stable_and_permutation_invariant(orc):
    n, d = 2000, 3
    P = W.uniform_cube(n, d, 5)
    # duplicate a few points: equal keys keep original index order
    P[10] = P[3]
    P[1500] = P[3]
    h = orc.H2(P, orc.Config(d=3, leaf_size=16), structure_only=True)
    keys = h.keys.astype(object)
    for i in range(n - 1):
        assert keys[i] < keys[i + 1] or (keys[i] == keys[i + 1] and h.perm[i] < h.perm[i + 1])


@pytest.mark.parametrize("d,eta2", [(2, (2, 1)), (3, (2, 1)), (3, (3, 1)), (2, (1, 1))])
def test_lists_against_geometry(orc, d, eta2):
    n = 1500 if d == 2 else 2500
    P = W.uniform_cube(n, d, 7 + d, -1.0, 1.0)
    h = orc.H2(P, orc.Config(d=d, leaf_size=8, eta2_num=eta2[0], eta2_den=eta2[1]), structure_only=True)
    e2 = eta2[0] / eta2[1]
    for l in range(h.kappa + 1):
        cells = np.array(list(h.level_cells(l)))
        boxes = [cell_box(h, c) for c in cells]
        lo = np.array([b[0] for b in boxes])
        hi = np.array([b[1] for b in boxes])
        diam = np.linalg.norm(hi - lo, axis=1)
        for t, X in enumerate(cells):
            # max(diam X, diam Y) <= eta dist(X, Y) from the real boxes (Eq. 2)
            gap = np.maximum(0.0, np.maximum(lo - hi[t], lo[t] - hi))
            dist = np.sqrt(np.sum(gap * gap, axis=1))
            adm = np.maximum(diam, diam[t]) <= math.sqrt(e2) * dist * (1 + 1e-12)
            nb = set(cells[~adm].tolist())
            assert set(h.nb(X).tolist()) == nb
            if l == 0:
                assert len(h.il(X)) == 0
                continue
            P_ = h.cpar[X]
            cand = [Y for Z in h.nb(P_) for Y in range(h.cch_beg[Z], h.cch_end[Z])]
            il = {Y for Y in cand if Y not in nb}
            assert set(h.il(X).tolist()) == il
            assert list(h.il(X)) == sorted(h.il(X)) and list(h.nb(X)) == sorted(h.nb(X))


def full_grid(d, level, jitter_seed=0):
    """One point at the centre of every cell of a full level: all cells exist."""
    m = 2 ** level
    g = (np.array(list(itertools.product(range(m), repeat=d)), dtype=float) + 0.5) / m
    return g


@pytest.mark.parametrize("d,eta2,nb_int,il_int", [(2, (2, 1), 9, 27), (3, (2, 1), 81, 567), (3, (3, 1), 27, 189)])
def test_interior_counts(orc, d, eta2, nb_int, il_int):
    level = 3 if d == 2 else 4
    P = full_grid(d, level)
    h = orc.H2(P, orc.Config(d=d, leaf_size=1, eta2_num=eta2[0], eta2_den=eta2[1]), structure_only=True)
    assert h.kappa == level
    cnb = [len(h.nb(c)) for c in h.level_cells(level)]
    cil = [len(h.il(c)) for c in h.level_cells(level)]
    assert max(cnb) == nb_int and max(cil) == il_int


def test_figure1_golden(orc):
    g = json.load(open(os.path.join(GOLDEN, "fig1_lists_2d.json")))
    P = full_grid(2, 3)
    h = orc.H2(P, orc.Config(d=2, leaf_size=1, eta2_num=2, eta2_den=1), structure_only=True)

    def find(l, co):
        for c in h.level_cells(l):
            if list(cell_box(h, c)[2]) == list(co):
                return c
        raise KeyError(co)

    def coords(cs):
        return {tuple(cell_box(h, c)[2]) for c in cs}

    X1 = find(1, g["levels"]["1"]["X"])
    assert len(h.nb(X1)) == 4 and len(h.il(X1)) == 0
    X2 = find(2, g["levels"]["2"]["X"])
    (a0, a1), (b0, b1) = g["levels"]["2"]["neighbours_box"]
    box = {(i, j) for i in range(a0, a1 + 1) for j in range(b0, b1 + 1)}
    assert coords(h.nb(X2)) == box
    assert coords(h.il(X2)) == {(i, j) for i in range(4) for j in range(4)} - box
    assert len(h.il(X2)) == g["levels"]["2"]["il_count"]
    X3 = find(3, g["levels"]["3"]["X"])
    (a0, a1), (b0, b1) = g["levels"]["3"]["neighbours_box"]
    nbox = {(i, j) for i in range(a0, a1 + 1) for j in range(b0, b1 + 1)}
    (c0, c1), (e0, e1) = g["levels"]["3"]["il_box"]
    ibox = {(i, j) for i in range(c0, c1 + 1) for j in range(e0, e1 + 1)} - nbox
    assert coords(h.nb(X3)) == nbox and coords(h.il(X3)) == ibox
    assert len(h.il(X3)) == g["levels"]["3"]["il_count"]


@pytest.mark.parametrize("d,n,nu", [(2, 2000, 12), (3, 2500, 16)])
def test_lists_symmetric_and_partition(orc, d, n, nu):
    """Y in IL(X) iff X in IL(Y); every leaf pair is covered exactly once,
    by N at the leaf level or by IL at exactly one ancestor level. Also what the
    symmetric FP32 M2L relies on when it serves each pair {X, Y} from one side:
    no cell has a sibling in its IL, and the parent of every Y in IL(X) is in
    N(parent(X)) (Table 1)."""
    P = W.gaussian_mixture(n, d, 21, k=4, sigma=0.15)
    h = orc.H2(P, orc.Config(d=d, leaf_size=nu), structure_only=True)
    for c in range(h.ncell):
        for Y in h.il(c):
            assert c in set(h.il(Y).tolist())
            assert h.cpar[Y] != h.cpar[c]
            assert h.cpar[Y] in set(h.nb(h.cpar[c]).tolist())
        for Y in h.nb(c):
            assert c in set(h.nb(Y).tolist())
    leaves = list(h.level_cells(h.kappa))
    anc = {}
    for c in leaves:
        chain = [c]
        while h.cpar[chain[-1]] >= 0:
            chain.append(h.cpar[chain[-1]])
        anc[c] = chain  # chain[k] is the ancestor k levels up
    ils = [set(h.il(c).tolist()) for c in range(h.ncell)]
    nbs = [set(h.nb(c).tolist()) for c in range(h.ncell)]
    for X in leaves:
        for Y in leaves:
            cover = int(Y in nbs[X])
            for k in range(h.kappa + 1):
                cover += int(anc[Y][k] in ils[anc[X][k]])
            assert cover == 1, (X, Y)
