"""A(P, Q) with distinct point sets (P != Q) through the C ABI: the handle is built on
the union [P; Q] and a product returns the P rows of the union matrix applied to [0; x].
Checked against the oracle's H^2 of the same union (the same pivots and bases: FP64 to
1e-12) and against the dense P x Q product (within the ACA tolerance), with points shared
by P and Q, several right-hand sides, both sizes orders and the host-buffer product."""
import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def clouds(n, m, shared, seed):
    rng = np.random.default_rng(seed)
    P = rng.uniform(0.0, 1.0, (n, 3))
    Q = np.vstack([rng.uniform(0.4, 1.4, (m - shared, 3)), P[:shared]])
    return P, Q


CASES = [
    # name, n, m, shared, kernel, kparam, eps
    ("invr_more_targets", 9000, 6000, 25, W.K_INV_R, (1.0, 0.0, 0.0, 0.0), 1e-8),
    ("invr_more_sources", 5000, 8000, 0, W.K_INV_R, (1.0, 0.0, 0.0, 0.0), 1e-8),
    ("gauss", 7000, 7000, 40, W.K_GAUSS, (1.0, 0.3, 1.0, 0.0), 1e-8),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pq_products(gpu, orc, case):
    import torch
    name, n, m, shared, kern, kp, eps = case
    P, Q = clouds(n, m, shared, 900 + n)
    kw = dict(d=3, leaf_size=48, aca_tol=eps, kernel=kern, kparam=kp)
    g = gpu.H2(P, gpu.Config(**kw), Q=Q)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, m))
    xd = torch.as_tensor(X, device="cuda")
    y64 = g.matvec(xd, gpu.PREC_FP64).cpu().numpy()
    y32 = g.matvec(xd, gpu.PREC_FP32).cpu().numpy()
    assert y64.shape == (3, n)
    # the oracle's H^2 of the union, product of [0; x], rows of P
    o = orc.H2(np.vstack([P, Q]), orc.Config(**kw))
    yo = o.matvec(np.hstack([np.zeros((3, n)), X]))[:, :n]
    assert rel(y64, yo) <= 1e-12
    assert rel(y32, yo) <= 1e-6
    # the dense P x Q product on sampled rows
    rows = rng.choice(n, 600, replace=False)
    yd = orc.dense_matvec_pq(P, Q, X, orc.Config(**kw), rows=rows)
    assert rel(y64[:, rows], yd) <= 10 * eps
    # one right-hand side and the host-buffer product
    y1 = g.matvec(xd[1], gpu.PREC_FP64).cpu().numpy()
    assert np.array_equal(y1, y64[1])
    yh = g.matvec_host(X, gpu.PREC_FP64)
    assert np.array_equal(yh, y64)
    assert g.stats()["device_status"] & (2 | 16) == 0
    g.close()


def test_pq_unsupported_calls(gpu):
    """P != Q handles serve nnca_matvec and nnca_matvec_host only; the other calls refuse."""
    import torch
    P, Q = clouds(3000, 2000, 0, 3)
    g = gpu.H2(P, gpu.Config(d=3, leaf_size=48, aca_tol=1e-6, kernel=W.K_INV_R, kparam=(1.0, 0.0, 0.0, 0.0)), Q=Q)
    x = torch.zeros(3000, dtype=torch.float64, device="cuda")
    y = torch.zeros(3000, dtype=torch.float64, device="cuda")
    with pytest.raises(gpu.NncaError):
        gpu.nnca_matvec_noalloc(g.handle, x, y, 3000, gpu.PREC_FP64)
    with pytest.raises(gpu.NncaError):
        gpu.nnca_matvec_batch([g.handle], [x], [y], 1, [3000], gpu.PREC_FP64)
    grad = torch.zeros((5000, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu.NncaError):
        gpu.nnca_gradient(g.handle, x, x, 1, 3000, grad)
    g.close()


def test_duplicate_points_against_dense(gpu, orc):
    """Points repeated in the cloud (distinct indices at one location): a pivot row that
    repeats another's residual only to round-off is not taken (it would make the pivot
    block singular); FP64 within the tolerance of the dense product, pivots bit-exact."""
    import torch
    rng = np.random.default_rng(21)
    base = rng.uniform(0.0, 1.0, (4000, 3))
    P = np.vstack([base, base[:30], base[100:105]])
    kw = dict(d=3, leaf_size=32, aca_tol=1e-8, kernel=W.K_INV_R, kparam=(1.0, 0.0, 0.0, 0.0))
    g = gpu.H2(P, gpu.Config(**kw))
    o = orc.H2(P, orc.Config(**kw))
    assert np.array_equal(g.export("PIV_ROW"), o.piv_row)
    x = rng.standard_normal(P.shape[0])
    y64 = g.matvec(torch.as_tensor(x, device="cuda"), gpu.PREC_FP64).cpu().numpy()
    yd = orc.dense_matvec(P, x, orc.Config(**kw))
    assert rel(y64, yd) <= 10 * 1e-8
    g.close()
