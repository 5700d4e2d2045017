"""Pins for the oracle's ACA (Sec. 2.2.1, Eqs. 3-4), its canonical reductions,
the pivot-submatrix solve (Sec. 2.3.1) and the bases built from them.

The pins: a hand trace (tests/golden), matrices of exact rank r, matrices with
known singular values, exact rational sums, and the identities X A_{tau sigma}
= A_{t~ sigma} and X[tau] = I that define the bases.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_aca_hand_trace(orc):
    g = json.load(open(os.path.join(GOLDEN, "aca_3x3_trace.json")))
    A = np.array(g["A"], dtype=float)
    for eps_s, rank in g["rank_for_eps"].items():
        pr, pc, U, V = orc.aca_dense(A, float(eps_s))
        assert len(pr) == rank
        assert pr.tolist() == g["pivot_rows"][:rank]
        assert pc.tolist() == g["pivot_cols"][:rank]
    pr, pc, U, V = orc.aca_dense(A, 0.01)
    # the full-rank cross approximation reproduces A
    assert np.allclose(U @ V.T, A, rtol=0, atol=1e-14)
    # the first cross is row 0 scaled by its pivot, and column 2
    assert np.allclose(V[:, 0], [1 / 3, 2 / 3, 1.0]) and np.allclose(U[:, 0], [3, 6, 10])
    assert np.allclose(U[:, 1], [0, 2, 11 / 3]) and np.allclose(V[:, 1], [1, 4 / 11, 0])


@pytest.mark.parametrize("m,n,r,seed", [(40, 300, 1, 0), (40, 300, 5, 1), (64, 2000, 12, 2), (7, 9, 7, 3), (300, 50, 20, 4)])
def test_aca_exact_rank(orc, m, n, r, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
    pr, pc, U, V = orc.aca_dense(A, 1e-10)
    assert len(pr) == r
    assert len(set(pr.tolist())) == r and len(set(pc.tolist())) == r
    err = np.linalg.norm(U @ V.T - A) / np.linalg.norm(A)
    assert err <= 1e-13
    # cross approximation form (Eq. 3): A_{:,sigma} A_{tau,sigma}^{-1} A_{tau,:}
    X = A[:, pc] @ np.linalg.inv(A[np.ix_(pr, pc)]) @ A[pr, :]
    assert np.linalg.norm(X - A) / np.linalg.norm(A) <= 1e-10


def test_aca_rank_one_block_recovered_exactly(orc):
    rng = np.random.default_rng(7)
    f = 1.0 + rng.random(50)
    g = 1.0 + rng.random(400)
    A = np.outer(f, g)
    pr, pc, U, V = orc.aca_dense(A, 1e-8)
    assert len(pr) == 1
    assert pr[0] == 0 and pc[0] == int(np.argmax(g))
    assert np.max(np.abs(U @ V.T - A)) <= 1e-14 * np.max(np.abs(A))


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6, 1e-8])
def test_aca_known_singular_decay(orc, eps):
    """sigma_k = 10^-k: the stopping rule (Eq. 4) ends near the first sigma_k below
    eps |A|_F and the approximation error is of order eps |A|_F."""
    rng = np.random.default_rng(3)
    m, n, K = 60, 500, 14
    Q1, _ = np.linalg.qr(rng.standard_normal((m, K)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, K)))
    s = 10.0 ** -np.arange(K)
    A = (Q1 * s) @ Q2.T
    pr, pc, U, V = orc.aca_dense(A, eps)
    k = len(pr)
    k_expected = int(np.sum(s > eps * np.linalg.norm(s)))
    assert abs(k - k_expected) <= 2
    err = np.linalg.norm(U @ V.T - A) / np.linalg.norm(A)
    assert err <= 30 * eps


def test_aca_zero_rows_skipped(orc):
    A = np.zeros((5, 6))
    A[3, :] = np.arange(1, 7)
    pr, pc, U, V = orc.aca_dense(A, 1e-12)
    assert pr.tolist() == [3] and pc.tolist() == [5]
    pr, pc, U, V = orc.aca_dense(np.zeros((4, 4)), 1e-12)
    assert len(pr) == 0


def test_cdot_exact_and_order(orc):
    rng = np.random.default_rng(9)
    # integer-valued products: every partial sum is exact, so the result is the exact sum
    a = rng.integers(-1000, 1000, 5000).astype(float)
    b = rng.integers(-1000, 1000, 5000).astype(float)
    assert orc.cdot(a, b) == float(np.sum(a.astype(np.int64) * b.astype(np.int64)))
    # real values: within the error bound of a 256-way split and pairwise fold
    a = rng.standard_normal(10001)
    b = rng.standard_normal(10001)
    exact = float(sum(Fraction(x) * Fraction(y) for x, y in zip(a, b)))
    bound = (10001 / 256 + 8 + 2) * 2 ** -53 * float(np.sum(np.abs(a * b)))
    assert abs(orc.cdot(a, b) - exact) <= bound
    assert orc.cdot(a[:0], b[:0]) == 0.0
    # the fold first adds partial t + 128 to partial t: 2^60 + 1 rounds to 2^60 and the
    # 1 is lost, while a left-to-right sum (2^60 - 2^60) + 1 would keep it
    x = np.zeros(256)
    y = np.ones(256)
    x[0], x[1], x[128] = 2.0 ** 60, -(2.0 ** 60), 1.0
    assert orc.cdot(x, y) == 0.0
    assert math.fsum(x * y) == 1.0


@pytest.mark.parametrize("r,m,seed", [(1, 3, 0), (5, 20, 1), (40, 120, 2), (90, 30, 3)])
def test_solve_right(orc, r, m, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((r, r)) + 3 * np.eye(r)
    B = rng.standard_normal((m, r))
    X = orc.solve_right(M, B)
    assert np.linalg.norm(X @ M - B) <= 1e-13 * np.linalg.norm(B) * np.linalg.cond(M)
    Xn = np.linalg.solve(M.T, B.T).T
    assert np.allclose(X, Xn, rtol=0, atol=1e-12 * np.linalg.cond(M) * np.max(np.abs(Xn)))


def test_solve_right_permutation_exact(orc):
    """A permutation matrix needs only row swaps: the solve is exact."""
    r = 6
    Pm = np.eye(r)[[3, 0, 5, 1, 4, 2]]
    B = np.arange(12 * r, dtype=float).reshape(12, r)
    assert np.array_equal(orc.solve_right(Pm, B), B @ Pm.T)


@pytest.mark.parametrize("wl,n", [("log2d_4096", 2500), ("invr3d_1m", 6000), ("gauss_mix_256k", 5000)])
def test_bases_identities(orc, wl, n):
    """Every cell's basis X = A_{t~ sigma} A_{tau sigma}^{-1} (Sec. 2.3.1, Eq. 11 and 14):
    X at the pivot rows is the identity, X A_{tau sigma} = A_{t~ sigma}, the pivots are
    candidates, and the column pivots lie in the interaction-list region."""
    w = W.WORKLOADS[wl].scaled(n)
    P = w.make_points()
    cfg = orc.Config(d=w.d, leaf_size=32, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    h = orc.H2(P, cfg)

    def K(rows, cols):
        return orc.entry_block(h, list(rows), list(cols))

    rng = np.random.default_rng(0)
    checked = 0
    for l in range(h.lmin, h.kappa + 1):
        cells = list(h.level_cells(l))
        for c in rng.choice(cells, size=min(6, len(cells)), replace=False):
            cand = h.candidates(c)
            tau, sigma = h.pivots(c), h.colpivots(c)
            X = h.operator(c)
            assert set(tau.tolist()) <= set(cand.tolist())
            if l == h.kappa:
                assert cand.tolist() == list(range(h.cbeg[c], h.cend[c]))
            else:
                kids = [h.pivots(cc) for cc in range(h.cch_beg[c], h.cch_end[c])]
                assert cand.tolist() == np.concatenate(kids).tolist()
            if h.passthru[c]:
                assert np.array_equal(X, np.eye(len(cand)))
                continue
            region = set()
            for Y in h.il(c):
                region |= set(range(h.cbeg[Y], h.cend[Y]))
            assert set(sigma.tolist()) <= region
            pos = [cand.tolist().index(t) for t in tau]
            assert np.array_equal(X[pos], np.eye(len(tau)))
            Ats = K(tau, sigma)
            Acs = K(cand, sigma)
            res = np.linalg.norm(X @ Ats - Acs) / np.linalg.norm(Acs)
            assert res <= 1e-12 * max(1.0, np.linalg.cond(Ats) * 1e-4)
            checked += 1
    assert checked > 0


def test_aca_repeated_row_not_taken(orc):
    """A row equal to another (two points at one location) is represented by that row
    exactly: its residual after the other is taken is round-off, and the ACA skips it
    like a zero row (the smallest unused row is taken next). The copy is never a pivot, the
    pivot block stays regular, and the crosses approximate the matrix, copy included, as
    well as those of the matrix without it."""
    rng = np.random.default_rng(3)
    X = rng.uniform(0.0, 1.0, (12, 3))
    Y = rng.uniform(3.0, 4.0, (40, 3))
    c = orc.Config(d=3, kernel=orc.K_INV_R, kparam=(1.0, 0.0, 0.0, 0.0))
    A = orc.kernel_block(c, X, Y)
    B = np.vstack([A, A[4:5]])                      # row 12 repeats row 4
    for eps in (1e-6, 1e-12):
        pa, qa, Ua, Va = orc.aca_dense(A, eps)
        pb, qb, Ub, Vb = orc.aca_dense(B, eps)
        assert 12 not in pb
        M = B[np.ix_(pb, qb)]
        assert np.linalg.cond(M) < 1e12
        ea = np.linalg.norm(A - Ua @ Va.T) / np.linalg.norm(A)
        eb = np.linalg.norm(B - Ub @ Vb.T) / np.linalg.norm(B)
        assert eb <= 10 * eps and ea <= 10 * eps


def test_repeated_points_against_dense(orc):
    """A cloud with repeated points (distinct indices, one location) keeps the product
    within 10 eps of the dense product; with the repeated rows taken as pivots the pivot
    blocks were singular and the product was off by orders of magnitude more."""
    rng = np.random.default_rng(11)
    P = rng.uniform(0.0, 1.0, (2700, 3))
    P = np.vstack([P, P[:7], rng.uniform(0.4, 1.4, (600, 3))])
    x = rng.standard_normal(P.shape[0])
    c = orc.Config(d=3, leaf_size=32, aca_tol=1e-8, kernel=orc.K_INV_R, kparam=(1.0, 0.0, 0.0, 0.0))
    h = orc.H2(P, c)
    y, yd = h.matvec(x), orc.dense_matvec(P, x, c)
    assert np.linalg.norm(y - yd) <= 10 * 1e-8 * np.linalg.norm(yd)
