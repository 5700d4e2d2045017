"""Thin Python binding of the C ABI in ``include/nnca.h`` (argument marshalling only).

The functions keep the C names: ``nnca_build``, ``nnca_matvec``,
``nnca_matvec_host``, ``nnca_destroy``, ``nnca_get_stats``, ``nnca_export``,
``nnca_last_error``. Every step of the build and of the product runs in the
CUDA library ``libnnca.so``; this module only passes pointers, sizes and
streams. PyTorch provides device memory and streams.

If the library is missing the import of this module still succeeds, but every
call raises ``RuntimeError``: there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnnca.so")

NNCA_OK, NNCA_ERR_INVALID_ARG, NNCA_ERR_OOM, NNCA_ERR_CUDA, NNCA_ERR_UNSUPPORTED, NNCA_ERR_TIMEOUT, \
    NNCA_ERR_INTERNAL = range(7)
K_LOG, K_INV_R, K_GAUSS, K_MATERN, K_PAPER_I, K_PAPER_II, K_SEPARABLE, K_POLY2 = range(8)
LAYOUT_AOS, LAYOUT_SOA = 0, 1
M2L_AUTO, M2L_FULL = 0, 1
F64, F32 = 0, 1
PREC_FP64, PREC_FP32, PREC_TF32X3, PREC_TF32, PREC_BF16 = 0, 1, 2, 3, 4
EXPORTS = ["PERM", "KEYS", "LEVEL_BASE", "CKEY", "CBEG", "CEND", "CPAR", "CCH_BEG", "CCH_END", "NB_OFF", "NB_IDX",
           "IL_OFF", "IL_IDX", "PIV_OFF", "PIV_ROW", "PIV_COL", "PASSTHRU", "CAND_OFF", "OP_OFF", "OP"]
SYMBOLS = ["nnca_build", "nnca_matvec", "nnca_matvec_host", "nnca_matvec_noalloc", "nnca_matvec_batch",
           "nnca_destroy", "nnca_get_stats", "nnca_export", "nnca_set_profiling", "nnca_set_wait_test",
           "nnca_gradient",
           "nnca_last_error", "nnca_status_string"]


class NncaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"nnca status {status}: {msg}")
        self.status = status


class _Config(C.Structure):
    _fields_ = [("d", C.c_int), ("leaf_size", C.c_int), ("eta2_num", C.c_int), ("eta2_den", C.c_int),
                ("aca_tol", C.c_double), ("kernel", C.c_int), ("kparam", C.c_double * 4), ("symmetric", C.c_int),
                ("m2l_form", C.c_int), ("m2l_item_targets", C.c_int), ("reserved", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("d", C.c_int), ("lmax", C.c_int), ("kappa", C.c_int), ("lmin", C.c_int), ("n", C.c_int64),
                ("ncell", C.c_int64), ("ncell_level", C.c_int64 * 64), ("n_il", C.c_int64), ("n_nb", C.c_int64),
                ("n_pivots", C.c_int64), ("max_rank", C.c_int64), ("n_passthru", C.c_int64),
                ("p2p_pairs", C.c_int64), ("m2l_pairs", C.c_int64), ("op_entries", C.c_int64),
                ("device_bytes", C.c_int64), ("build_ms", C.c_double * 8), ("aca_retries", C.c_int64),
                ("pass_ms", C.c_double * 8), ("pass_calls", C.c_int64), ("launches_per_product", C.c_int64),
                ("device_status", C.c_int64), ("m2l_evals", C.c_int64)]


_lib = None


def lib() -> C.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.nnca_build.restype = C.c_int
        L.nnca_build.argtypes = [C.POINTER(_Config), vp, C.c_int64, vp, C.c_int64, C.c_int, vp, C.POINTER(vp)]
        L.nnca_matvec.restype = C.c_int
        L.nnca_matvec.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, C.c_int, C.c_int, vp]
        L.nnca_matvec_host.restype = C.c_int
        L.nnca_matvec_host.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, C.c_int, C.c_int, vp]
        L.nnca_destroy.restype = None
        L.nnca_destroy.argtypes = [vp]
        L.nnca_get_stats.restype = C.c_int
        L.nnca_get_stats.argtypes = [vp, C.POINTER(_Stats)]
        L.nnca_export.restype = C.c_int
        L.nnca_export.argtypes = [vp, C.c_int, vp, C.c_int64, C.POINTER(C.c_int64)]
        L.nnca_matvec_noalloc.restype = C.c_int
        L.nnca_matvec_noalloc.argtypes = [vp, vp, vp, C.c_int64, C.c_int, C.c_int, vp]
        L.nnca_matvec_batch.restype = C.c_int
        L.nnca_matvec_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int64),
                                        C.c_int64, C.c_int, C.c_int, vp]
        L.nnca_gradient.restype = C.c_int
        L.nnca_gradient.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, vp, vp, vp]
        L.nnca_set_wait_test.restype = C.c_int
        L.nnca_set_wait_test.argtypes = [C.c_int64, C.c_uint]
        L.nnca_set_profiling.restype = C.c_int
        L.nnca_set_profiling.argtypes = [vp, C.c_int]
        L.nnca_last_error.restype = C.c_char_p
        L.nnca_last_error.argtypes = [vp]
        L.nnca_status_string.restype = C.c_char_p
        L.nnca_status_string.argtypes = [C.c_int]
        _lib = L
    return _lib


@dataclass
class Config:
    """nnca_config: d, leaf size nu, eta^2 = num/den, ACA tolerance, kernel and its parameters."""
    d: int = 3
    leaf_size: int = 64
    eta2_num: int = 2
    eta2_den: int = 1
    aca_tol: float = 1e-6
    kernel: int = K_INV_R
    kparam: tuple = (1.0, 0.0, 0.0, 0.0)
    m2l_form: int = M2L_AUTO
    m2l_item_targets: int = 0

    def c(self) -> _Config:
        k = (C.c_double * 4)(*[float(v) for v in (list(self.kparam) + [0.0] * 4)[:4]])
        return _Config(self.d, self.leaf_size, self.eta2_num, self.eta2_den, float(self.aca_tol), self.kernel, k, 1,
                       self.m2l_form, self.m2l_item_targets, 0)


def _check(status: int, handle=None):
    if status != NNCA_OK:
        msg = lib().nnca_last_error(handle).decode(errors="replace")
        raise NncaError(status, msg)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def nnca_last_error(handle=None) -> str:
    return lib().nnca_last_error(handle).decode(errors="replace")


def nnca_build(cfg: Config, P, stream=None, layout: int = LAYOUT_AOS, Q=None):
    """Build the H^2 representation of the points P (a CUDA float64 tensor, n x d for the
    AoS layout), or of A(P, Q) when Q (the same kind of tensor) is given. Returns the
    opaque handle (a ctypes void pointer)."""
    import torch
    assert isinstance(P, torch.Tensor) and P.is_cuda and P.dtype == torch.float64 and P.is_contiguous()
    n = P.shape[0] if layout == LAYOUT_AOS else P.shape[1]
    qp, nq = None, 0
    if Q is not None:
        assert isinstance(Q, torch.Tensor) and Q.is_cuda and Q.dtype == torch.float64 and Q.is_contiguous()
        qp, nq = Q.data_ptr(), (Q.shape[0] if layout == LAYOUT_AOS else Q.shape[1])
    c = cfg.c()
    out = C.c_void_p()
    st = lib().nnca_build(C.byref(c), P.data_ptr(), n, qp, nq, layout, _stream_ptr(stream), C.byref(out))
    _check(st, None)
    return out


def nnca_matvec(handle, x, y, nrhs: int, ld: int, precision: int = PREC_FP64, stream=None):
    """y = A~ x on CUDA tensors (float64 or float32, right-hand side r at [r*ld, r*ld + n))."""
    import torch
    dtype = F64 if x.dtype == torch.float64 else F32
    assert x.dtype == y.dtype and x.is_cuda and y.is_cuda
    _check(lib().nnca_matvec(handle, x.data_ptr(), y.data_ptr(), nrhs, ld, dtype, precision, _stream_ptr(stream)),
           handle)


def nnca_matvec_batch(handles, xs, ys, nrhs: int, lds, precision: int = PREC_FP64, stream=None):
    """y_k = A_k x_k for independent handles at once (CUDA tensors of one dtype)."""
    import torch
    k = len(handles)
    assert k == len(xs) == len(ys) == len(lds) and k > 0
    dtype = F64 if xs[0].dtype == torch.float64 else F32
    for x, y in zip(xs, ys):
        assert x.dtype == y.dtype == xs[0].dtype and x.is_cuda and y.is_cuda
    H = (C.c_void_p * k)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    X = (C.c_void_p * k)(*[x.data_ptr() for x in xs])
    Y = (C.c_void_p * k)(*[y.data_ptr() for y in ys])
    LD = (C.c_int64 * k)(*[int(v) for v in lds])
    _check(lib().nnca_matvec_batch(H, k, X, Y, LD, nrhs, dtype, precision, _stream_ptr(stream)), None)


def nnca_matvec_noalloc(handle, x, y, ld: int, precision: int = PREC_FP64, stream=None):
    """y = A~ x for one right-hand side with no device allocation (workspace in a
    fixed device array of the library; see include/nnca.h for the limit)."""
    import torch
    dtype = F64 if x.dtype == torch.float64 else F32
    assert x.dtype == y.dtype and x.is_cuda and y.is_cuda
    _check(lib().nnca_matvec_noalloc(handle, x.data_ptr(), y.data_ptr(), ld, dtype, precision, _stream_ptr(stream)),
           handle)


def nnca_matvec_host(handle, x: np.ndarray, y: np.ndarray, nrhs: int, ld: int, precision: int = PREC_FP64,
                     stream=None):
    """Same product on host (numpy) buffers; copies are inside the call."""
    dtype = F64 if x.dtype == np.float64 else F32
    assert x.dtype == y.dtype and x.flags.c_contiguous and y.flags.c_contiguous
    _check(lib().nnca_matvec_host(handle, x.ctypes.data, y.ctypes.data, nrhs, ld, dtype, precision,
                                  _stream_ptr(stream)), handle)


def nnca_gradient(handle, x, g, nrhs: int, ld: int, grad_p, grad_h=None, stream=None) -> None:
    """dL/dP (into grad_p, n x d) and dL/dh (into grad_h, one element) of
    L = sum_r g_r^T A~ x_r with the pivots fixed; all FP64 device tensors."""
    import torch
    assert x.dtype == g.dtype == grad_p.dtype == torch.float64 and x.is_cuda and g.is_cuda and grad_p.is_cuda
    _check(lib().nnca_gradient(handle, x.data_ptr(), g.data_ptr(), nrhs, ld, grad_p.data_ptr(),
                               grad_h.data_ptr() if grad_h is not None else None, _stream_ptr(stream)), handle)


def nnca_set_wait_test(wait_limit_clocks: int, extra_tx_bytes: int) -> None:
    """Testing hook of the FP32 kernels' bounded waits (include/nnca.h); (0, 0)
    restores normal operation."""
    _check(lib().nnca_set_wait_test(int(wait_limit_clocks), int(extra_tx_bytes)), None)


def nnca_destroy(handle) -> None:
    if handle:
        lib().nnca_destroy(handle)


def nnca_get_stats(handle) -> dict:
    s = _Stats()
    _check(lib().nnca_get_stats(handle, C.byref(s)), handle)
    out = {}
    for name, _ in _Stats._fields_:
        v = getattr(s, name)
        out[name] = list(v) if hasattr(v, "__len__") else v
    out["ncell_level"] = out["ncell_level"][: out["kappa"] + 1]
    return out


def nnca_set_profiling(handle, on: bool) -> None:
    _check(lib().nnca_set_profiling(handle, 1 if on else 0), handle)


def nnca_export(handle, what: str) -> np.ndarray:
    code = EXPORTS.index(what)
    nbytes = C.c_int64(0)
    _check(lib().nnca_export(handle, code, None, 0, C.byref(nbytes)), handle)
    dt = {"KEYS": np.uint64, "CKEY": np.uint64, "OP": np.float64}.get(what, np.int64)
    buf = np.zeros(nbytes.value // 8, dtype=dt)
    if buf.size:
        _check(lib().nnca_export(handle, code, buf.ctypes.data, nbytes.value, C.byref(nbytes)), handle)
    return buf


class H2:
    """Convenience owner of a handle: build on construction, destroy on close/del.
    With Q, the handle represents A(P, Q): products take x on Q (m entries) and
    return y on P (n entries)."""

    def __init__(self, P, cfg: Config, stream=None, Q=None):
        import torch
        if not isinstance(P, torch.Tensor):
            P = torch.as_tensor(np.ascontiguousarray(P, dtype=np.float64), device="cuda")
        if Q is not None and not isinstance(Q, torch.Tensor):
            Q = torch.as_tensor(np.ascontiguousarray(Q, dtype=np.float64), device="cuda")
        self.P = P.contiguous()
        self.Q = Q.contiguous() if Q is not None else None
        self.cfg = cfg
        self.n = self.P.shape[0]
        self.m = self.Q.shape[0] if self.Q is not None else self.n
        self.handle = nnca_build(cfg, self.P, stream, Q=self.Q)

    def matvec(self, x, precision: int = PREC_FP64, out=None, stream=None):
        """x: CUDA tensor (m,) or (nrhs, m); returns y, (n,) or (nrhs, n), of x's dtype."""
        import torch
        x = x.contiguous()
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        assert x.shape[-1] == self.m
        shape = (self.n,) if x.dim() == 1 else (nrhs, self.n)
        if self.m == self.n:
            y = out if out is not None else torch.empty_like(x)
            nnca_matvec(self.handle, x, y, nrhs, self.n, precision, stream)
            return y
        ld = max(self.n, self.m)
        xp = torch.zeros((nrhs, ld), dtype=x.dtype, device=x.device)
        xp[:, :self.m] = x.reshape(nrhs, self.m)
        yp = torch.empty((nrhs, ld), dtype=x.dtype, device=x.device)
        nnca_matvec(self.handle, xp, yp, nrhs, ld, precision, stream)
        y = yp[:, :self.n].reshape(shape)
        if out is not None:
            out.copy_(y)
            return out
        return y.contiguous()

    def matvec_host(self, x: np.ndarray, precision: int = PREC_FP64, stream=None) -> np.ndarray:
        x = np.ascontiguousarray(x)
        nrhs = 1 if x.ndim == 1 else x.shape[0]
        assert x.shape[-1] == self.m
        ld = max(self.n, self.m)
        xp = np.zeros((nrhs, ld), dtype=x.dtype)
        xp[:, :self.m] = x.reshape(nrhs, self.m)
        yp = np.empty((nrhs, ld), dtype=x.dtype)
        nnca_matvec_host(self.handle, xp, yp, nrhs, ld, precision, stream)
        y = yp[:, :self.n]
        return np.ascontiguousarray(y[0] if x.ndim == 1 else y)

    def stats(self) -> dict:
        return nnca_get_stats(self.handle)

    def export(self, what: str) -> np.ndarray:
        return nnca_export(self.handle, what)

    def set_profiling(self, on: bool) -> None:
        nnca_set_profiling(self.handle, on)

    def close(self):
        if getattr(self, "handle", None):
            nnca_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
