"""Failure handling of the FP32 product's bounded waits, without a GPU fault.

The FP32 M2L and near-field kernels wait on shared-memory barriers of their own
thread block for their own bulk (TMA) copies. Every wait has a clock budget;
one that runs out records DEV_WAIT_TIMEOUT (bit 16 of device_status), lets the
block's copies in flight land and returns, so the context stays usable. The
testing hook nnca_set_wait_test shortens the budget and raises every staging
round's expected byte count above what its copies deliver, so every wait runs
out while every copy lands: nothing faults and nothing hangs.
"""
import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV_WAIT_TIMEOUT = 16


def test_bounded_waits_run_out_and_report(gpu):
    import torch
    w = W.WORKLOADS["invr3d_1m"].scaled(20000)
    P = torch.as_tensor(w.make_points(), device="cuda")
    cfg = gpu.Config(d=3, leaf_size=64, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    x = torch.as_tensor(w.make_vector(), device="cuda")
    X4 = torch.as_tensor(W.vector_normal(w.n, 3, nrhs=4), device="cuda")
    h = gpu.H2(P, cfg)
    X16 = torch.as_tensor(W.vector_normal(w.n, 4, nrhs=16), device="cuda")
    ref1 = h.matvec(x, gpu.PREC_FP32).cpu().numpy()
    ref4 = h.matvec(X4, gpu.PREC_FP32).cpu().numpy()
    ref16 = h.matvec(X16, gpu.PREC_TF32X3).cpu().numpy()
    assert h.stats()["device_status"] & (2 | DEV_WAIT_TIMEOUT) == 0
    gpu.nnca_set_wait_test(20000, 16)
    try:
        # one right-hand side (symmetric M2L, grouped near field), a pass of four
        # (M2L and near field of four right-hand sides): every wait runs out
        h.matvec(x, gpu.PREC_FP32)
        h.matvec(X4, gpu.PREC_FP32)
        # the tensor-core M2L: its staging, evaluation and MMA roles all give up,
        # the block waits for its copies and MMAs and frees its tensor memory
        h.matvec(X16, gpu.PREC_TF32X3)
        torch.cuda.synchronize()
        assert h.stats()["device_status"] & DEV_WAIT_TIMEOUT
        # the synchronising host-buffer product reports the failed check
        with pytest.raises(gpu.NncaError):
            h.matvec_host(w.make_vector(), gpu.PREC_FP32)
    finally:
        gpu.nnca_set_wait_test(0, 0)
    h.close()
    # the context is intact: a new handle reproduces the products bit for bit
    g = gpu.H2(P, cfg)
    assert np.array_equal(g.matvec(x, gpu.PREC_FP32).cpu().numpy(), ref1)
    assert np.array_equal(g.matvec(X4, gpu.PREC_FP32).cpu().numpy(), ref4)
    assert np.array_equal(g.matvec(X16, gpu.PREC_TF32X3).cpu().numpy(), ref16)
    assert g.stats()["device_status"] & (2 | DEV_WAIT_TIMEOUT) == 0
    g.close()
