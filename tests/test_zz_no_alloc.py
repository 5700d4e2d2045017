"""nnca_matvec_noalloc: the product without device allocation, against nnca_matvec.

Callers that cannot allocate device memory when they run the product (a fixed
budget already given to their own allocator, or loops that cannot take
cudaMalloc's implicit synchronisation) use the entry point whose workspace is
a fixed device array of the library. This file runs last (pytest collects it
after the other test files), so a failure here comes after every other test.
The entry point is called first on a fresh handle, whose own workspace does not
exist yet, with the device's free memory read before and after: it must not
change (a first handle has run both products before, so that loading the
library's kernels and its fixed array does not count). Two calls in a row must both reproduce the ordinary product: the shared
array keeps the previous call's contents, so the second call checks that
whatever must start at zero is cleared.
"""
import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_14832_gb300 import _build, nnca
    _build.build()
    w = W.WORKLOADS["invr3d_1m"].scaled(20000)
    P = torch.as_tensor(w.make_points(), device="cuda")
    cfg = nnca.Config(d=3, leaf_size=64, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    return torch, nnca, w, P, cfg


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_noalloc_matches_matvec(precision, tol):
    torch, nnca, w, P, cfg = _setup(precision)
    x = torch.as_tensor(w.make_vector(), device="cuda")
    z = torch.as_tensor(W.vector_normal(w.n, 99), device="cuda")
    ys = [torch.full_like(x, float("nan")), torch.full_like(z, float("nan"))]
    # load every kernel and the fixed array once (lazy module loading allocates
    # device memory on a kernel's first launch), on a handle of its own
    h0 = nnca.H2(P, cfg)
    nnca.nnca_matvec_noalloc(h0.handle, x, ys[0], w.n, precision)
    h0.matvec(x, precision)
    torch.cuda.synchronize()
    h0.close()
    h = nnca.H2(P, cfg)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # first products of a fresh handle, through the entry point that allocates nothing
    for xin, y in zip([x, z], ys):          # two calls in a row
        nnca.nnca_matvec_noalloc(h.handle, xin, y, w.n, precision)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    got = [y.cpu().numpy() for y in ys]
    # the ordinary product (which allocates the handle's workspace now)
    for xin, g in zip([x, z], got):
        ref = h.matvec(xin, precision).cpu().numpy()
        assert np.linalg.norm(g - ref) <= tol * np.linalg.norm(ref)
    # and the fixed array serves again after the handle's own workspace exists
    y = torch.full_like(x, float("nan"))
    nnca.nnca_matvec_noalloc(h.handle, x, y, w.n, precision)
    torch.cuda.synchronize()
    ref = h.matvec(x, precision).cpu().numpy()
    assert np.linalg.norm(y.cpu().numpy() - ref) <= tol * np.linalg.norm(ref)
    h.close()


def test_noalloc_rejects_host_buffers():
    """Host memory where device buffers are required is rejected before any device work."""
    import ctypes
    torch, nnca, w, P, cfg = _setup(0)
    h = nnca.H2(P, cfg)
    xh = np.zeros(w.n)
    yh = np.zeros(w.n)
    st = nnca.lib().nnca_matvec_noalloc(h.handle, xh.ctypes.data, yh.ctypes.data, w.n, nnca.F64, nnca.PREC_FP64,
                                        None)
    assert st == nnca.NNCA_ERR_INVALID_ARG
    assert b"device memory" in nnca.lib().nnca_last_error(h.handle)
    h.close()
