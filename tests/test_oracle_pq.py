"""The oracle's form of Sec. 2.3 for distinct point sets (oracle/pq.py: incoming and
outgoing pivots and bases from two ACAs per cell, Eqs. 12 and 15-18) against what the
mathematics fixes: the dense P x Q product within the ACA tolerance, the error falling
with the tolerance, kernels of low exact rank reproduced to round-off, and the defining
identities of the bases."""
import numpy as np
import pytest


def clouds(n, m, shared, seed):
    rng = np.random.default_rng(seed)
    P = rng.uniform(0.0, 1.0, (n, 3))
    Q = np.vstack([rng.uniform(0.4, 1.4, (m - shared, 3)), P[:shared]])
    return P, Q, rng.standard_normal(m)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,m,shared", [(1500, 1207, 7), (900, 1600, 0)])
@pytest.mark.parametrize("kernel", ["invr", "gauss"])
def test_pq_form_against_dense(orc, n, m, shared, kernel):
    from oracle.pq import H2PQ
    P, Q, x = clouds(n, m, shared, 40 + n)
    k, kp = (orc.K_INV_R, (1.0, 0.0, 0.0, 0.0)) if kernel == "invr" else (orc.K_GAUSS, (1.0, 0.3, 1.0, 0.0))
    errs = []
    for eps in (1e-4, 1e-6, 1e-8):
        c = orc.Config(d=3, leaf_size=32, aca_tol=eps, kernel=k, kparam=kp)
        y = H2PQ(P, Q, c).matvec(x)
        e = rel(y, orc.dense_matvec_pq(P, Q, x, c))
        assert e <= 10 * eps
        errs.append(e)
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("kernel,bound", [("sep", 1e-13), ("poly2", 1e-12)])
def test_pq_form_low_rank_kernels(orc, kernel, bound):
    from oracle.pq import H2PQ
    P, Q, x = clouds(1200, 1000, 5, 7)
    c = orc.Config(d=3, leaf_size=32, aca_tol=1e-10, kernel=orc.K_SEPARABLE if kernel == "sep" else orc.K_POLY2,
                   kparam=(1.0, 0.0, 0.0, 0.0))
    h = H2PQ(P, Q, c)
    assert rel(h.matvec(x), orc.dense_matvec_pq(P, Q, x, c)) <= bound
    if kernel == "sep":
        # a rank-1 kernel: at most one incoming and one outgoing pivot per cell
        assert all(len(h.si[c]) <= 1 for c in range(h.t.ncell))
        assert all(len(h.to[c]) <= 1 for c in range(h.t.ncell))


def test_pq_bases_identities(orc):
    """U_B = A(t~, sigma) A(tau, sigma)^{-1}: the identity on the pivot rows and
    U_B A(tau, sigma) = A(t~, sigma); V_B^T = A(tau_o, sigma_o)^{-1} A(tau_o, s~): the identity
    on the pivot columns and A(tau_o, sigma_o) V_B^T = A(tau_o, s~)."""
    from oracle.pq import H2PQ
    P, Q, _ = clouds(1500, 1207, 7, 3)
    c = orc.Config(d=3, leaf_size=32, aca_tol=1e-8, kernel=orc.K_INV_R, kparam=(1.0, 0.0, 0.0, 0.0))
    h = H2PQ(P, Q, c)
    checked = 0
    for cell in range(h.t.ncell):
        if len(h.si[cell]):
            U, tci, tau, sig = h.U[cell], h.tci[cell], h.ti[cell], h.si[cell]
            pos = [int(np.where(tci == r)[0][0]) for r in tau]
            assert np.array_equal(U[pos], np.eye(len(tau)))
            M = h._K(tau, sig)
            B = h._K(tci, sig)
            assert np.linalg.norm(U @ M - B) <= 1e-9 * np.linalg.norm(B)
            checked += 1
        if len(h.to[cell]):
            V, sco, tau, sig = h.V[cell], h.sco[cell], h.to[cell], h.so[cell]
            pos = [int(np.where(sco == s)[0][0]) for s in sig]
            assert np.array_equal(V[pos], np.eye(len(sig)))
            M = h._K(tau, sig)
            B = h._K(tau, sco)
            assert np.linalg.norm(M @ V.T - B) <= 1e-9 * np.linalg.norm(B)
            checked += 1
    assert checked > 50
