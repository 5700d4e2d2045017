"""Batched independent problems (nnca_matvec_batch), the leaf-size tuner and the
CUDA-graph capture of the batched product."""
import ctypes

import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W


def test_batch_arguments_checked_on_host():
    """NULL arrays and a bad count are rejected before any device work."""
    from paper_2203_14832_gb300 import _build
    lib = ctypes.CDLL(_build.build())
    lib.nnca_matvec_batch.restype = ctypes.c_int
    st = lib.nnca_matvec_batch(None, 2, None, None, None, ctypes.c_int64(1), 0, 0, None)
    assert st == 1
    H = (ctypes.c_void_p * 1)(None)
    X = (ctypes.c_void_p * 1)(None)
    LD = (ctypes.c_int64 * 1)(10)
    assert lib.nnca_matvec_batch(H, 0, X, X, LD, ctypes.c_int64(1), 0, 0, None) == 1
    assert lib.nnca_matvec_batch(H, 1, X, X, LD, ctypes.c_int64(1), 0, 0, None) == 1
    lib.nnca_last_error.restype = ctypes.c_char_p
    assert b"NULL handle" in lib.nnca_last_error(None)


def test_batch_recipe():
    ws = W.batch_workloads()
    assert len(ws) == 32
    assert all((1 << 14) <= w.n <= (1 << 19) for w in ws)
    assert sum(w.kernel == W.K_INV_R for w in ws) == 16 and sum(w.kernel == W.K_GAUSS for w in ws) == 16
    assert all(w.nrhs == 8 for w in ws)
    # seeded: the same sizes every time
    assert [w.n for w in ws] == [w.n for w in W.batch_workloads()]


def small_batch(gpu, count=4, nrhs=3):
    import torch
    probs = []
    for k, w in enumerate(W.batch_workloads(count=count, n_lo=3000, n_hi=12000, nrhs=nrhs)):
        P = torch.as_tensor(w.make_points(), device="cuda")
        cfg = gpu.Config(d=3, leaf_size=32, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
        x = torch.as_tensor(np.ascontiguousarray(w.make_vector()), device="cuda")
        probs.append((w, P, cfg, x))
    return probs


@pytest.mark.gpu
def test_batch_equals_single_products(gpu, orc):
    import torch
    from paper_2203_14832_gb300 import batch
    probs = small_batch(gpu)
    for prec in (gpu.PREC_FP32, gpu.PREC_FP64):
        b = batch.Batch([batch.Problem(P, cfg, x) for (_, P, cfg, x) in probs], precision=prec)
        ys = [y.clone() for y in b.matvec()]
        torch.cuda.synchronize()
        for (w, P, cfg, x), h, y in zip(probs, b.handles, ys):
            # same kernels in the same order: bit for bit
            assert torch.equal(h.matvec(x, prec), y)
        if prec == gpu.PREC_FP64:
            w, P, cfg, x = probs[0]
            o = orc.H2(w.make_points(), orc.Config(d=3, leaf_size=32, aca_tol=w.aca_tol, kernel=w.kernel,
                                                   kparam=w.kparam))
            yo = o.matvec(w.make_vector())
            assert np.linalg.norm(ys[0].cpu().numpy() - yo) / np.linalg.norm(yo) < 1e-12
        for h in b.handles:
            assert h.stats()["device_status"] & (2 | 16) == 0
        b.close()


@pytest.mark.gpu
def test_cross_problem_batch(gpu):
    """Nine right-hand sides (two passes of four and one of one): the passes of four run
    synchronised across the problems, the M2L of each pass as one launch per kernel family
    over the cross-problem item list (1/r and Gaussian problems). Bit for bit the single
    products, through a captured graph too, with the M2L tile tuned differently per problem."""
    import torch
    from paper_2203_14832_gb300 import batch
    probs = small_batch(gpu, count=6, nrhs=9)
    tiled = []
    for k, (w, P, cfg, x) in enumerate(probs):
        c = gpu.Config(d=3, leaf_size=32, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam,
                       m2l_item_targets=(0, 64, 128)[k % 3])
        tiled.append((w, P, c, x))
    b = batch.Batch([batch.Problem(P, cfg, x) for (_, P, cfg, x) in tiled], precision=gpu.PREC_FP32)
    ys = [y.clone() for y in b.matvec()]
    torch.cuda.synchronize()
    for (w, P, cfg, x), h, y in zip(tiled, b.handles, ys):
        assert torch.equal(h.matvec(x, gpu.PREC_FP32), y)
        y64 = h.matvec(x, gpu.PREC_FP64)
        assert float(torch.linalg.norm(y - y64) / torch.linalg.norm(y64)) < 1e-6
        assert h.stats()["device_status"] & (2 | 16) == 0
    g = b.capture()
    for y in b.y:
        y.zero_()
    g.replay()
    torch.cuda.synchronize()
    for y, r in zip(b.y, ys):
        assert torch.equal(y, r)
    b.close()


@pytest.mark.gpu
def test_batch_graph_replay(gpu):
    import torch
    from paper_2203_14832_gb300 import batch
    probs = small_batch(gpu)
    b = batch.Batch([batch.Problem(P, cfg, x) for (_, P, cfg, x) in probs], precision=gpu.PREC_FP32)
    ref = [y.clone() for y in b.matvec()]
    g = b.capture()
    for y in b.y:
        y.zero_()
    g.replay()
    torch.cuda.synchronize()
    for y, r in zip(b.y, ref):
        assert torch.equal(y, r)
    # new inputs in the same buffers flow through the captured graph
    for x in b.x:
        x.mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    for y, r in zip(b.y, ref):
        assert torch.allclose(y, 2.0 * r, rtol=1e-5, atol=1e-5 * float(r.abs().max()))
    b.close()


@pytest.mark.gpu
def test_leaf_size_tuner(gpu):
    import torch
    from paper_2203_14832_gb300 import batch
    w, P, cfg, x = small_batch(gpu, count=1)[0]
    h, times = batch.tune_leaf_size(P, cfg, x, candidates=(16, 32, 64), reps=2, tiles=(0, 64))
    first = {nu: times[f"{nu}/0"] for nu in (16, 32, 64)}
    nu = min(first, key=first.get)
    assert set(times) == {"16/0", "32/0", "64/0", f"{nu}/64"} and all(t > 0 for t in times.values())
    assert h.cfg.leaf_size == nu
    assert h.cfg.m2l_item_targets == (64 if times[f"{nu}/64"] < times[f"{nu}/0"] else 0)
    y = h.matvec(x, gpu.PREC_FP64)
    h2 = gpu.H2(P, gpu.Config(d=3, leaf_size=64, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam))
    y2 = h2.matvec(x, gpu.PREC_FP64)
    # a different leaf size is a different approximation of the same matrix
    assert float(torch.linalg.norm(y - y2) / torch.linalg.norm(y2)) < 50 * w.aca_tol
    h.close()
    h2.close()


@pytest.mark.gpu
def test_autograd_in_x(gpu, orc):
    """dL/dx of L = <w, A x> is A^T w = A w (symmetric); against the oracle's dense product."""
    import torch
    from paper_2203_14832_gb300.autograd import h2_matvec
    w = W.WORKLOADS["invr3d_1m"].scaled(6000)
    P = w.make_points()
    cfg = gpu.Config(d=3, leaf_size=32, aca_tol=1e-8, kernel=w.kernel, kparam=w.kparam)
    h = gpu.H2(torch.as_tensor(P, device="cuda"), cfg)
    x = torch.as_tensor(w.make_vector(), device="cuda").requires_grad_(True)
    wt = torch.as_tensor(W.vector_normal(w.n, 77), device="cuda")
    y = h2_matvec(h, x)
    (wt * y).sum().backward()
    ocfg = orc.Config(d=3, leaf_size=32, aca_tol=1e-8, kernel=w.kernel, kparam=w.kparam)
    gd = orc.dense_matvec(P, wt.cpu().numpy(), ocfg)
    g = x.grad.cpu().numpy()
    assert np.linalg.norm(g - gd) / np.linalg.norm(gd) < 1e-6
    # the gradient is the same handle's product on w, bit for bit
    assert torch.equal(x.grad, h.matvec(wt))
    h.close()
