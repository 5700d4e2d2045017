"""Pins for the oracle's H^2 product (Sec. 4) and dense product (Eq. 19).

Special cases with a known answer (one leaf, separable and polynomial kernels
of exact low rank), the symmetry of A~ under the symmetric shortcut, the
stored and on-the-fly forms, the decay of the error with the ACA tolerance
(Sec. 5.1-5.2), and an independent assembly of the H^2 matrix from its nested
bases (Eqs. 5, 12-14) that the passes of Sec. 4 must reproduce.
"""
import math

import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W


def cfg_for(orc, w, **kw):
    c = dict(d=w.d, leaf_size=w.leaf_size, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    c.update(kw)
    return orc.Config(**c)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_kernel_closed_forms(orc):
    z = np.zeros(2)
    e1 = np.array([1.0, 0.0])
    C = orc.Config
    assert orc.kernel(C(d=2, kernel=orc.K_LOG, kparam=(1.0, 0, 0, 0)), z, e1) == 0.0
    assert abs(orc.kernel(C(d=2, kernel=orc.K_LOG, kparam=(2.0, 0, 0, 0)), z, math.e * e1) - 2.0) < 1e-15
    assert orc.kernel(C(d=2, kernel=orc.K_INV_R, kparam=(3.0, 0, 0, 0)), z, np.array([0.0, 4.0])) == 0.75
    g = C(d=2, kernel=orc.K_GAUSS, kparam=(1.0, 0.2, 1.0, 0))
    assert abs(orc.kernel(g, z, 0.2 * e1) - math.exp(-0.5)) < 1e-16
    assert orc.kernel(g, z, z) == 1.0
    m = C(d=2, kernel=orc.K_MATERN, kparam=(1.0, 0.5, 1.0, 0))
    assert abs(orc.kernel(m, z, e1) - math.exp(-2.0)) < 1e-16
    a = 1e-4
    for k in (orc.K_PAPER_I, orc.K_PAPER_II):
        c = C(d=2, kernel=k, kparam=(1.0, a, 0, 0))
        # both branches of the Sec. 5.1 kernels equal 1 at r = a, continuously
        lo = orc.kernel(c, z, a * (1 - 1e-12) * e1)
        hi = orc.kernel(c, z, a * e1)
        assert abs(lo - 1.0) < 1e-9 and abs(hi - 1.0) < 1e-12
    # the singular kernels take 0 at r = 0 for distinct coincident points
    assert orc.kernel(C(d=2, kernel=orc.K_INV_R, kparam=(1.0, 0, 0, 0)), z, z) == 0.0


def test_dense_matches_numpy_matrix(orc):
    w = W.WORKLOADS["log2d_4096"].scaled(700)
    P = w.make_points()
    x = w.make_vector()
    cfg = cfg_for(orc, w)
    D = np.sqrt(((P[:, None, :] - P[None, :, :]) ** 2).sum(-1))
    with np.errstate(divide="ignore"):
        A = np.log(D)
    np.fill_diagonal(A, 0.0)
    y = orc.dense_matvec(P, x, cfg)
    assert rel(y, A @ x) < 1e-13
    rows = np.array([0, 5, 699, 5])
    assert np.array_equal(orc.dense_rows(P, rows, x, cfg), y[rows])


@pytest.mark.parametrize("wl", ["log2d_4096", "invr3d_1m", "sphere_512k"])
def test_single_leaf_is_dense(orc, wl):
    """N <= nu: one leaf, no admissible block, the H^2 product is the dense product."""
    w = W.WORKLOADS[wl].scaled(60)
    P = w.make_points()
    x = w.make_vector()
    cfg = cfg_for(orc, w)
    h = orc.H2(P, cfg)
    assert h.kappa == 0 and h.ncell == 1
    assert rel(h.matvec(x), orc.dense_matvec(P, x, cfg)) < 1e-15


@pytest.mark.parametrize("kernel,d,n,tol", [("sep", 2, 3000, 1e-13), ("sep", 3, 4000, 1e-13),
                                            ("poly2", 2, 3000, 1e-12), ("poly2", 3, 4000, 1e-12)])
def test_exact_low_rank_kernels(orc, kernel, d, n, tol):
    """Separable K = f(x) f(y) (rank 1) and (1 + x.y)^2 (rank <= (d+1)(d+2)/2): every
    admissible block has exact low rank, so the H^2 product equals the dense one to
    round-off and every cell's rank is bounded by the kernel's rank."""
    P = W.uniform_cube(n, d, 31, -1.0, 1.0)
    x = W.vector_normal(n, 32)
    k = orc.K_SEPARABLE if kernel == "sep" else orc.K_POLY2
    cfg = orc.Config(d=d, leaf_size=16, aca_tol=1e-10, kernel=k, kparam=(1.0, 0, 0, 0))
    h = orc.H2(P, cfg)
    assert h.lmin <= h.kappa
    rmax = 1 if kernel == "sep" else (d + 1) * (d + 2) // 2
    for l in range(h.lmin, h.kappa + 1):
        for c in h.level_cells(l):
            if not h.passthru[c]:
                assert h.piv_off[c + 1] - h.piv_off[c] <= rmax
    assert rel(h.matvec(x), orc.dense_matvec(P, x, cfg)) < tol


def test_symmetry_and_linearity(orc):
    w = W.WORKLOADS["invr3d_1m"].scaled(5000)
    P = w.make_points()
    cfg = cfg_for(orc, w, leaf_size=32)
    h = orc.H2(P, cfg)
    x = W.vector_normal(5000, 1)
    z = W.vector_normal(5000, 2)
    ax, az = h.matvec(x), h.matvec(z)
    # S_{X,Y} = S_{Y,X}^T and V = U under the symmetric shortcut: A~ is symmetric
    assert abs(x @ az - z @ ax) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(az)
    both = h.matvec(np.stack([x, z]))
    assert np.array_equal(both[0], ax) and np.array_equal(both[1], az)
    assert rel(h.matvec(2.0 * x - 3.0 * z), 2.0 * ax - 3.0 * az) < 1e-14


def test_stored_equals_on_the_fly(orc):
    w = W.WORKLOADS["gauss_mix_256k"].scaled(4000)
    P = w.make_points()
    cfg = cfg_for(orc, w, leaf_size=32)
    h = orc.H2(P, cfg)
    x = W.vector_normal(4000, 3)
    assert np.array_equal(h.matvec(x, form=0), h.matvec(x, form=1))


@pytest.mark.parametrize("wl,n,nu", [("invr3d_1m", 6000, 32), ("log2d_4096", 4096, 32), ("gauss_mix_256k", 4000, 32)])
def test_symmetric_transverse_pass(orc, wl, n, nu):
    """The transverse pass taken over each admissible pair of cells once (S applied to one
    side, its transpose to the other; what the FP32 product's symmetric M2L computes) gives
    the product of the per-cell pass within FP64 rounding, and both stay within the ACA
    bound of the dense product (interaction lists are non-empty, so a pair the symmetric
    pass missed would show as a far-field error far above 1e-13)."""
    w = W.WORKLOADS[wl].scaled(n)
    P = w.make_points()
    h = orc.H2(P, cfg_for(orc, w, leaf_size=nu))
    assert int(h.il_off[-1]) > 0
    x = W.vector_normal(n, 5)
    y0, y2 = h.matvec(x, form=0), h.matvec(x, form=2)
    assert rel(y2, y0) < 1e-13
    yd = orc.dense_matvec(P, x, cfg_for(orc, w, leaf_size=nu))
    assert rel(y2, yd) < 10 * w.aca_tol + 1e-12


def test_input_permutation(orc):
    """Points with distinct keys sort the same way whatever their input order, so
    the product of the permuted problem is the permuted product, bit for bit."""
    w = W.WORKLOADS["invr3d_1m"].scaled(3000)
    P = w.make_points()
    x = W.vector_normal(3000, 4)
    cfg = cfg_for(orc, w, leaf_size=24)
    pi = np.random.default_rng(5).permutation(3000)
    y = orc.H2(P, cfg).matvec(x)
    yp = orc.H2(P[pi], cfg).matvec(x[pi])
    assert np.array_equal(yp, y[pi])


def test_tolerance_decay_and_bound(orc):
    """Sec. 5.1-5.2: the error of the H^2 product falls as the ACA tolerance falls.
    The log r workload at eps = 1e-8 stays within 10 eps of the dense product."""
    w = W.WORKLOADS["log2d_4096"]
    P = w.make_points()
    x = w.make_vector()
    yd = orc.dense_matvec(P, x, cfg_for(orc, w))
    errs = []
    for eps in [1e-2, 1e-4, 1e-6, 1e-8, 1e-10]:
        h = orc.H2(P, cfg_for(orc, w, aca_tol=eps))
        errs.append(rel(h.matvec(x), yd))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[3] <= 10 * 1e-8, errs


def assembled_matrix(orc, h, cfg):
    """The H^2 matrix written out from its parts (Sec. 3, Eqs. 5 and 12-14).

    Column basis of every cell B over its points t^B, by the nested form:
    U_B(leaf) = operator, U_B(non-leaf) = blockdiag(U_{B_c}) [C_{B_1 B}; ...].
    Symmetric shortcut: V_B = U_B. Block (X, Y) with Y in IL(X) is
    U_X S_{X,Y} U_Y^T with S_{X,Y} = A(t^{X,i}, t^{Y,i}); near blocks are exact."""
    n = h.n
    U = {}
    for l in range(h.kappa, h.lmin - 1, -1):
        for c in h.level_cells(l):
            op = h.operator(c)
            if l == h.kappa:
                U[c] = op
            else:
                rows, r0 = [], 0
                for cc in range(h.cch_beg[c], h.cch_end[c]):
                    rc = U[cc].shape[1]
                    rows.append(U[cc] @ op[r0:r0 + rc])
                    r0 += rc
                U[c] = np.vstack(rows) if rows else np.zeros((0, op.shape[1]))

    def K(rows, cols):
        return orc.entry_block(h, list(rows), list(cols))

    M = np.zeros((n, n))
    for c in range(h.ncell):
        tX = slice(h.cbeg[c], h.cend[c])
        for Y in h.il(c):
            S = K(h.pivots(c), h.pivots(Y))
            M[tX, h.cbeg[Y]:h.cend[Y]] += U[c] @ S @ U[Y].T
        if h.level_of(c) == h.kappa:
            for Y in h.nb(c):
                M[tX, h.cbeg[Y]:h.cend[Y]] += K(range(h.cbeg[c], h.cend[c]), range(h.cbeg[Y], h.cend[Y]))
    return M


@pytest.mark.parametrize("wl,n,nu", [("log2d_4096", 900, 16), ("invr3d_1m", 1200, 16)])
def test_passes_match_assembled_matrix(orc, wl, n, nu):
    w = W.WORKLOADS[wl].scaled(n)
    P = w.make_points()
    cfg = cfg_for(orc, w, leaf_size=nu)
    h = orc.H2(P, cfg)
    assert h.lmin < h.kappa
    M = assembled_matrix(orc, h, cfg)
    # M is the H^2 approximation of A in tree order: every entry is covered once
    A = orc.entry_block(h, range(n), range(n))
    assert rel(M, A) < 100 * w.aca_tol
    assert np.allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
    x = W.vector_normal(n, 8)
    ys = h.matvec(x)[h.perm]          # product in tree order
    assert rel(ys, M @ x[h.perm]) < 1e-13


# --- pass-through cells -------------------------------------------------------
# A cell whose far-field candidate columns cannot determine its basis (no
# candidates at all, or an ACA that used up every candidate column without
# meeting its stopping rule while candidate rows remain) passes all its
# candidate rows up with the identity basis, so that its points still reach
# the far field of its ancestors. These clouds contain such cells; the pins are
# the dense product, for a full vector and for a vector supported only on the
# points of pass-through cells, whose far field would vanish if those points
# were dropped.

def background_and_cluster(n_background, n_cluster, delta, seed):
    """Sparse uniform points in [0,1]^3 plus one tight Gaussian cluster: the uniform
    tree goes deep for the cluster, and the background points' cells form chains of
    cells with tiny or empty interaction-list regions."""
    rng = np.random.default_rng(seed)
    centre = np.array([0.3, 0.6, 0.45])
    return np.vstack([rng.uniform(0.0, 1.0, (n_background, 3)),
                      centre + delta * rng.standard_normal((n_cluster, 3))])


def far_field_columns(h, c):
    """|s~| of cell c: points of the IL cells (leaf) or their children's pivots."""
    if h.level_of(c) == h.kappa:
        return int(sum(h.cend[Y] - h.cbeg[Y] for Y in h.il(c)))
    return int(sum(h.piv_off[z + 1] - h.piv_off[z] for Y in h.il(c) for z in range(h.cch_beg[Y], h.cch_end[Y])))


def near_only(h, x_sorted):
    """The leaf-level near field alone (Sec. 3 step 3), in sorted order."""
    y = np.zeros(h.n)
    for c in h.level_cells(h.kappa):
        cols = np.concatenate([np.arange(h.cbeg[Y], h.cend[Y]) for Y in h.nb(c)])
        rows = np.arange(h.cbeg[c], h.cend[c])
        y[rows] = orc_entry(h, rows, cols) @ x_sorted[cols]
    return y


def orc_entry(h, rows, cols):
    from oracle import oracle as O
    return O.entry_block(h, rows, cols)


PASSTHRU_CASES = [
    # name, points, leaf size, kernel, kparam
    ("gauss_mix_8000", lambda: W.WORKLOADS["gauss_mix_256k"].scaled(8000).make_points(), 16, W.K_GAUSS,
     (1.0, 0.2, 1.0, 0.0)),
    ("cluster_540", lambda: background_and_cluster(500, 40, 1e-4, 2), 8, W.K_INV_R, (1.0, 0.0, 0.0, 0.0)),
    ("coincident_250", lambda: np.repeat(W.uniform_cube(50, 3, 3), 5, axis=0), 3, W.K_INV_R, (1.0, 0.0, 0.0, 0.0)),
]


@pytest.mark.parametrize("name,make,nu,kernel,kparam", PASSTHRU_CASES, ids=[c[0] for c in PASSTHRU_CASES])
def test_passthrough_against_dense(orc, name, make, nu, kernel, kparam):
    P = make()
    n = P.shape[0]
    eps = 1e-8
    cfg = orc.Config(d=3, leaf_size=nu, aca_tol=eps, kernel=kernel, kparam=kparam)
    h = orc.H2(P, cfg)
    pt = np.nonzero(h.passthru)[0]
    assert len(pt) > 0
    for c in pt:
        # all candidates passed up, with the identity basis and no column pivots
        m = int(h.cand_off[c + 1] - h.cand_off[c])
        assert h.piv_off[c + 1] - h.piv_off[c] == m
        assert np.array_equal(h.pivots(c), h.candidates(c))
        assert np.array_equal(h.operator(c), np.eye(m))
        assert np.all(h.colpivots(c) == -1)
    if name != "gauss_mix_8000":
        # pass-through above the leaves, and cells whose ACA used up its columns
        assert any(h.level_of(c) < h.kappa for c in pt)
        assert any(far_field_columns(h, c) > 0 for c in pt)
    x = W.vector_normal(n, 5)
    assert rel(h.matvec(x), orc.dense_matvec(P, x, cfg)) <= 10 * eps
    # a vector on the points of pass-through cells only
    on = np.zeros(n, dtype=bool)
    for c in pt:
        on[h.perm[h.cbeg[c]:h.cend[c]]] = True
    xs = np.where(on, x, 0.0)
    yd = orc.dense_matvec(P, xs, cfg)
    assert rel(h.matvec(xs), yd) <= 10 * eps
    # the far field carries much of that product: dropping those points from it
    # would miss the dense product by far more than the bound above
    yn = np.empty(n)
    yn[h.perm] = near_only(h, xs[h.perm])
    assert rel(yn, yd) > 1e-2


def test_passthrough_assembled_matrix(orc):
    """On a cloud with pass-through chains the passes reproduce the H^2 matrix written
    out from its nested bases (identity blocks for pass-through cells), and that matrix
    is within the ACA bound of A."""
    P = background_and_cluster(300, 30, 1e-4, 4)
    cfg = orc.Config(d=3, leaf_size=8, aca_tol=1e-8, kernel=W.K_INV_R, kparam=(1.0, 0, 0, 0))
    h = orc.H2(P, cfg)
    assert h.passthru.sum() > 0 and h.lmin < h.kappa
    M = assembled_matrix(orc, h, cfg)
    A = orc.entry_block(h, range(h.n), range(h.n))
    assert rel(M, A) < 100 * cfg.aca_tol
    x = W.vector_normal(h.n, 8)
    assert rel(h.matvec(x)[h.perm], M @ x[h.perm]) < 1e-13


def test_dense_pq_definition(orc):
    """A(P, Q) x with distinct point sets: values fixed by hand (1/r and a Gaussian), the
    coincident pair p_0 = q_0 giving 0 for the singular kernel and K(0) for the smooth one."""
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    Q = np.array([[0.0, 0.0, 0.0], [0.0, 2.0, 0.0], [3.0, 0.0, 0.0]])
    x = np.array([1.0, 2.0, 3.0])
    c = orc.Config(d=3, kernel=orc.K_INV_R, kparam=(1.0, 0.0, 7.0, 0.0))
    y = orc.dense_matvec_pq(P, Q, x, c)
    assert abs(y[0] - (0.0 + 2.0 / 2.0 + 3.0 / 3.0)) < 1e-15
    assert abs(y[1] - (1.0 + 2.0 / np.sqrt(5.0) + 3.0 / 2.0)) < 1e-15
    g = orc.Config(d=3, kernel=orc.K_GAUSS, kparam=(1.0, 1.5, 7.0, 0.0))
    yg = orc.dense_matvec_pq(P, Q, x, g)
    e = lambda r2: np.exp(-r2 / (2 * 1.5 ** 2))
    assert abs(yg[0] - (1.0 + 2 * e(4.0) + 3 * e(9.0))) < 1e-15
    assert abs(yg[1] - (e(1.0) + 2 * e(5.0) + 3 * e(4.0))) < 1e-15
    # rows and several right-hand sides agree with the full product
    X = np.vstack([x, -x])
    Y = orc.dense_matvec_pq(P, Q, X, c, rows=np.array([1]))
    assert abs(Y[0, 0] - y[1]) < 1e-15 and abs(Y[1, 0] + y[1]) < 1e-15


def test_pq_through_union(orc):
    """A(P, Q) x as the P rows of the symmetric H^2 product of the union [P; Q] applied
    to [0; x]: within the ACA tolerance of the dense P x Q product, and exactly the
    union's own H^2 product (the embedding adds no error of its own)."""
    rng = np.random.default_rng(11)
    P = rng.uniform(0.0, 1.0, (1500, 3))
    Q = np.vstack([rng.uniform(0.4, 1.4, (1200, 3)), P[:7]])     # overlapping box, 7 shared points
    x = rng.standard_normal(Q.shape[0])
    for kern, kp, eps in ((orc.K_INV_R, (1.0, 0.0, 0.0, 0.0), 1e-8), (orc.K_GAUSS, (1.0, 0.3, 1.0, 0.0), 1e-8)):
        c = orc.Config(d=3, leaf_size=32, aca_tol=eps, kernel=kern, kparam=kp)
        U = np.vstack([P, Q])
        h = orc.H2(U, c)
        yu = h.matvec(np.concatenate([np.zeros(P.shape[0]), x]))
        yd = orc.dense_matvec_pq(P, Q, x, c)
        assert np.linalg.norm(yu[:P.shape[0]] - yd) <= 10 * eps * np.linalg.norm(yd)
        # the union's dense product on the same embedded vector, restricted to P: the
        # P x Q block of the union matrix (the diagonal rule never applies there)
        ydu = orc.dense_matvec(U, np.concatenate([np.zeros(P.shape[0]), x]), c)[:P.shape[0]]
        assert np.linalg.norm(ydu - yd) <= 1e-14 * np.linalg.norm(yd)
