"""nnca_matvec_noalloc: the product without device allocation, against nnca_matvec.

Callers that cannot allocate device memory when they run the product (a fixed
budget already given to their own allocator, or loops that cannot take
cudaMalloc's implicit synchronisation) use the entry point whose workspace is
a fixed device array of the library. This file runs last (pytest collects it
after the other test files), so a failure here comes after every other test.
Two calls in a row must both reproduce the ordinary product: the shared array
keeps the previous call's contents, so the second call checks that whatever
must start at zero is cleared.
"""
import numpy as np
import pytest

from paper_2203_14832_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_noalloc_matches_matvec(precision, tol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_14832_gb300 import _build, nnca
    _build.build()
    w = W.WORKLOADS["invr3d_1m"].scaled(20000)
    h = nnca.H2(torch.as_tensor(w.make_points(), device="cuda"),
                nnca.Config(d=3, leaf_size=64, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam))
    x = torch.as_tensor(w.make_vector(), device="cuda")
    z = torch.as_tensor(W.vector_normal(w.n, 99), device="cuda")
    ref_x = h.matvec(x, precision).cpu().numpy()
    ref_z = h.matvec(z, precision).cpu().numpy()
    for xin, ref in [(x, ref_x), (z, ref_z)]:          # two calls in a row
        y = torch.full_like(xin, float("nan"))
        nnca.nnca_matvec_noalloc(h.handle, xin, y, w.n, precision)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    # the handle's own workspace still serves the ordinary product afterwards
    assert np.array_equal(h.matvec(x, precision).cpu().numpy(), ref_x)
    h.close()
