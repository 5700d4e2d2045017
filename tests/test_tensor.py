"""Tensor-core forms of the product (M2L of up to 64 right-hand sides at once as
dense contractions on tcgen05.mma) against the FP64 oracle, through the C ABI.

3xTF32 (split operands, main products flushed into compensated sums): every
right-hand side within 1e-6 of the oracle's H^2 product, the accuracy the
mixed-precision form is measured at, and within 1e-6 of the SIMT FP32 form.
TF32 and BF16 operands (11 and 8 significant bits) cannot reach that; their
bounds are stated from the operand rounding: a relative error of about 2^-11
(TF32) or 2^-8 (BF16) per kernel value and weight, amplified by cancellation in
the far-field sums (measured on these workloads: TF32 up to 1.6e-3, BF16 up to
1.3e-2 in a column).
"""
import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    ("gauss_mix_256k", 12000, {"leaf_size": 32}),
    ("invr3d_1m", 12000, {"leaf_size": 32}),
    ("sphere_512k", 12000, {}),
]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("wl,n,kw", CASES)
def test_tensor_forms_many_rhs(gpu, orc, wl, n, kw):
    """70 right-hand sides: one pass of 64 and one of 6 (rows of the MMA left empty)."""
    import torch
    w = W.WORKLOADS[wl].scaled(n)
    P = w.make_points()
    c = dict(d=w.d, leaf_size=w.leaf_size, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    c.update(kw)
    g = gpu.H2(torch.as_tensor(P, device="cuda"), gpu.Config(**c))
    o = orc.H2(P, orc.Config(**c))
    X = W.vector_normal(n, 51, nrhs=70)
    Yo = o.matvec(X)
    Xd = torch.as_tensor(X, device="cuda")
    Y3 = g.matvec(Xd, gpu.PREC_TF32X3).cpu().numpy()
    Y32 = g.matvec(Xd, gpu.PREC_FP32).cpu().numpy()
    for r in range(70):
        assert rel(Y3[r], Yo[r]) < 1e-6, r
        assert rel(Y3[r], Y32[r]) < 1e-6, r
    # deterministic: every order is fixed
    assert np.array_equal(g.matvec(Xd, gpu.PREC_TF32X3).cpu().numpy(), Y3)
    Yt = g.matvec(Xd, gpu.PREC_TF32).cpu().numpy()
    Yb = g.matvec(Xd, gpu.PREC_BF16).cpu().numpy()
    et = [rel(Yt[r], Yo[r]) for r in range(70)]
    eb = [rel(Yb[r], Yo[r]) for r in range(70)]
    assert max(et) < 5e-3 and max(eb) < 5e-2
    # the rounding of the operands sets the error: BF16 above TF32 above 3xTF32
    assert np.median(eb) > np.median(et) > 10 * max(rel(Y3[r], Yo[r]) for r in range(70))
    assert g.stats()["device_status"] & (2 | 16) == 0
    g.close()


def test_tensor_form_one_rhs_and_float_io(gpu, orc):
    """One right-hand side (63 empty rows) and float input/output buffers."""
    import torch
    w = W.WORKLOADS["invr3d_1m"].scaled(9000)
    P = w.make_points()
    c = dict(d=3, leaf_size=32, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    g = gpu.H2(torch.as_tensor(P, device="cuda"), gpu.Config(**c))
    o = orc.H2(P, orc.Config(**c))
    x = W.vector_normal(9000, 52)
    yo = o.matvec(x)
    y = g.matvec(torch.as_tensor(x, device="cuda"), gpu.PREC_TF32X3).cpu().numpy()
    assert rel(y, yo) < 1e-6
    X = W.vector_normal(9000, 53, nrhs=5).astype(np.float32)
    Y = g.matvec(torch.as_tensor(X, device="cuda"), gpu.PREC_TF32X3).cpu().numpy()
    for r in range(5):
        assert rel(Y[r].astype(np.float64), o.matvec(X[r].astype(np.float64))) < 1e-6
    g.close()
