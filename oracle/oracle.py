"""Python access to the FP64 CPU oracle (``liboracle.so``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it to check and time against the CUDA path.
The product never imports this module. The oracle shares no code with the
CUDA library; see ``oracle.h`` for what each C file computes and which passage
of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = ["orc_kernel.c", "orc_tree.c", "orc_lists.c", "orc_aca.c", "orc_build.c", "orc_matvec.c"]

K_LOG, K_INV_R, K_GAUSS, K_MATERN, K_PAPER_I, K_PAPER_II, K_SEPARABLE, K_POLY2 = range(8)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, no contraction of multiply-adds)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, "oracle.h"), os.path.join(HERE, "orc_internal.h")]
    if not force and os.path.exists(LIB_PATH):
        t = os.path.getmtime(LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in deps):
            return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Config(C.Structure):
    _fields_ = [("d", C.c_int), ("leaf_size", C.c_int), ("eta2_num", C.c_int), ("eta2_den", C.c_int),
                ("aca_tol", C.c_double), ("kernel", C.c_int), ("kparam", C.c_double * 4)]


_P = C.POINTER
_L = _P(C.c_long)
_D = _P(C.c_double)


class _H2(C.Structure):
    _fields_ = [("d", C.c_int), ("lmax", C.c_int), ("kappa", C.c_int), ("lmin", C.c_int),
                ("n", C.c_long), ("corner", C.c_double * 4), ("side", C.c_double),
                ("perm", _L), ("key", _P(C.c_uint64)), ("x", _D),
                ("ncell", C.c_long), ("level_base", C.c_long * 66),
                ("ckey", _P(C.c_uint64)), ("cbeg", _L), ("cend", _L), ("cpar", _L),
                ("cch_beg", _L), ("cch_end", _L),
                ("nb_off", _L), ("nb_idx", _L), ("il_off", _L), ("il_idx", _L),
                ("piv_off", _L), ("piv_row", _L), ("piv_col", _L), ("passthru", _P(C.c_int)),
                ("cand_off", _L), ("cand", _L), ("op_off", _L), ("op", _D),
                ("s_off", _L), ("s_blk", _D), ("near_off", _L), ("near_blk", _D),
                ("cfg", _Config)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        L.orc_build.restype = _P(_H2)
        L.orc_build.argtypes = [_P(_Config), _D, C.c_long, C.c_int]
        L.orc_build_structure.restype = _P(_H2)
        L.orc_build_structure.argtypes = [_P(_Config), _D, C.c_long, C.c_int]
        L.orc_free.argtypes = [_P(_H2)]
        L.orc_leaf_pivots.restype = C.c_long
        L.orc_leaf_pivots.argtypes = [_P(_H2), C.c_long, _L, _L, C.c_long]
        L.orc_assemble.argtypes = [_P(_H2)]
        L.orc_h2_matvec.argtypes = [_P(_H2), _D, _D, C.c_long, C.c_long, C.c_int, C.c_int]
        L.orc_dense_matvec.argtypes = [_P(_Config), _D, C.c_long, _D, _D, C.c_long, C.c_long, C.c_int]
        L.orc_dense_rows.argtypes = [_P(_Config), _D, C.c_long, _L, C.c_long, _D, _D, C.c_long, C.c_long,
                                     C.c_int]
        L.orc_aca_dense.restype = C.c_long
        L.orc_aca_dense.argtypes = [_D, C.c_long, C.c_long, C.c_long, C.c_double, _L, _L, _D, _D]
        L.orc_solve_right.restype = C.c_int
        L.orc_solve_right.argtypes = [_D, C.c_long, _D, C.c_long, _D]
        L.orc_cdot.restype = C.c_double
        L.orc_cdot.argtypes = [_D, _D, C.c_long]
        L.orc_kernel_block.argtypes = [_P(_Config), _D, C.c_long, _D, C.c_long, _D]
        L.orc_kernel.restype = C.c_double
        L.orc_kernel.argtypes = [_P(_Config), _D, _D]
        _lib = L
    return _lib


@dataclass
class Config:
    """Oracle parameters (Sec. 2.1 nu, Sec. 2.2 eta, Eq. 4 epsilon, the kernel)."""
    d: int = 3
    leaf_size: int = 64
    eta2_num: int = 2
    eta2_den: int = 1
    aca_tol: float = 1e-6
    kernel: int = K_INV_R
    kparam: tuple = (1.0, 0.0, 0.0, 0.0)

    def c(self) -> _Config:
        k = (C.c_double * 4)(*[float(v) for v in (list(self.kparam) + [0.0] * 4)[:4]])
        return _Config(self.d, self.leaf_size, self.eta2_num, self.eta2_den, float(self.aca_tol),
                        self.kernel, k)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _lp(a: np.ndarray):
    return a.ctypes.data_as(_L)


def _arr(ptr, n, dtype):
    if n <= 0 or not ptr:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


class H2:
    """An oracle H^2 representation built from points P (n x d)."""

    def __init__(self, P: np.ndarray, cfg: Config, structure_only: bool = False, nthreads: int = 0):
        P = np.ascontiguousarray(P, dtype=np.float64)
        assert P.ndim == 2 and P.shape[1] == cfg.d
        self.cfg = cfg
        self._c = cfg.c()
        fn = lib().orc_build_structure if structure_only else lib().orc_build
        self._h = fn(C.byref(self._c), _dp(P), P.shape[0], nthreads)
        if not self._h:
            raise ValueError("oracle rejected the input")
        h = self._h.contents
        self.n, self.d, self.kappa, self.lmin, self.lmax = h.n, h.d, h.kappa, h.lmin, h.lmax
        self.corner = np.array(h.corner[: self.d])
        self.side = h.side
        nc = h.ncell
        self.ncell = nc
        self.level_base = np.array(h.level_base[: self.kappa + 2], dtype=np.int64)
        self.perm = _arr(h.perm, self.n, np.int64)
        self.keys = _arr(h.key, self.n, np.uint64)
        self.x = _arr(h.x, self.n * self.d, np.float64).reshape(self.n, self.d)
        self.ckey = _arr(h.ckey, nc, np.uint64)
        self.cbeg = _arr(h.cbeg, nc, np.int64)
        self.cend = _arr(h.cend, nc, np.int64)
        self.cpar = _arr(h.cpar, nc, np.int64)
        self.cch_beg = _arr(h.cch_beg, nc, np.int64)
        self.cch_end = _arr(h.cch_end, nc, np.int64)
        self.nb_off = _arr(h.nb_off, nc + 1, np.int64)
        self.nb_idx = _arr(h.nb_idx, int(self.nb_off[-1]) if nc else 0, np.int64)
        self.il_off = _arr(h.il_off, nc + 1, np.int64)
        self.il_idx = _arr(h.il_idx, int(self.il_off[-1]) if nc else 0, np.int64)
        if not structure_only:
            self.piv_off = _arr(h.piv_off, nc + 1, np.int64)
            npiv = int(self.piv_off[-1]) if nc else 0
            self.piv_row = _arr(h.piv_row, npiv, np.int64)
            self.piv_col = _arr(h.piv_col, npiv, np.int64)
            self.passthru = _arr(h.passthru, nc, np.int32)
            self.cand_off = _arr(h.cand_off, nc + 1, np.int64)
            self.cand = _arr(h.cand, int(self.cand_off[-1]) if nc else 0, np.int64)
            self.op_off = _arr(h.op_off, nc + 1, np.int64)
            self.op = _arr(h.op, int(self.op_off[-1]) if nc else 0, np.float64)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_free(self._h)
            self._h = None

    # --- views ---------------------------------------------------------
    def level_cells(self, l: int) -> range:
        return range(int(self.level_base[l]), int(self.level_base[l + 1]))

    def level_of(self, c: int) -> int:
        return int(np.searchsorted(self.level_base, c, side="right") - 1)

    def nb(self, c: int) -> np.ndarray:
        return self.nb_idx[self.nb_off[c]: self.nb_off[c + 1]]

    def il(self, c: int) -> np.ndarray:
        return self.il_idx[self.il_off[c]: self.il_off[c + 1]]

    def pivots(self, c: int) -> np.ndarray:
        return self.piv_row[self.piv_off[c]: self.piv_off[c + 1]]

    def colpivots(self, c: int) -> np.ndarray:
        return self.piv_col[self.piv_off[c]: self.piv_off[c + 1]]

    def candidates(self, c: int) -> np.ndarray:
        return self.cand[self.cand_off[c]: self.cand_off[c + 1]]

    def operator(self, c: int) -> np.ndarray:
        m = int(self.cand_off[c + 1] - self.cand_off[c])
        r = int(self.piv_off[c + 1] - self.piv_off[c])
        return self.op[self.op_off[c]: self.op_off[c + 1]].reshape(m, r)

    def leaf_pivots(self, c: int):
        """(t^{B,i}, s^{B,i}) of leaf c computed from the tree and lists alone."""
        cap = int(self.cend[c] - self.cbeg[c]) + 1
        pr = np.zeros(cap, dtype=np.int64)
        pc = np.zeros(cap, dtype=np.int64)
        r = lib().orc_leaf_pivots(self._h, int(c), _lp(pr), _lp(pc), cap)
        if r < 0:
            raise ValueError("not a leaf")
        return pr[:r].copy(), pc[:r].copy()

    # --- products ------------------------------------------------------
    def assemble(self):
        lib().orc_assemble(self._h)

    def matvec(self, x: np.ndarray, form: int = 0, nthreads: int = 0) -> np.ndarray:
        """y = A~ x for x of shape (n,) or (nrhs, n); form 0 on the fly, 1 stored, 2 on the fly
        with each admissible pair of cells evaluated once (S and its transpose)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        one = x.ndim == 1
        xx = x.reshape(1, -1) if one else x
        y = np.zeros_like(xx)
        if form == 1:
            self.assemble()
        rc = lib().orc_h2_matvec(self._h, _dp(xx), _dp(y), xx.shape[0], self.n, form, nthreads)
        if rc != 0:
            raise RuntimeError("oracle matvec failed")
        return y[0] if one else y


def dense_matvec(P: np.ndarray, x: np.ndarray, cfg: Config, nthreads: int = 0) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    one = x.ndim == 1
    xx = x.reshape(1, -1) if one else x
    y = np.zeros_like(xx)
    c = cfg.c()
    lib().orc_dense_matvec(C.byref(c), _dp(P), P.shape[0], _dp(xx), _dp(y), xx.shape[0], P.shape[0], nthreads)
    return y[0] if one else y


def dense_rows(P: np.ndarray, rows: np.ndarray, x: np.ndarray, cfg: Config, nthreads: int = 0) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    one = x.ndim == 1
    xx = x.reshape(1, -1) if one else x
    y = np.zeros((xx.shape[0], rows.shape[0]))
    c = cfg.c()
    lib().orc_dense_rows(C.byref(c), _dp(P), P.shape[0], _lp(rows), rows.shape[0], _dp(xx), _dp(y),
                         xx.shape[0], P.shape[0], nthreads)
    return y[0] if one else y


def aca_dense(A: np.ndarray, eps: float):
    """Partially pivoted ACA of an explicit matrix: (row pivots, col pivots, U, V)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    kmax = min(m, n)
    pr = np.zeros(max(kmax, 1), dtype=np.int64)
    pc = np.zeros(max(kmax, 1), dtype=np.int64)
    U = np.zeros((max(kmax, 1), m))
    V = np.zeros((max(kmax, 1), n))
    k = lib().orc_aca_dense(_dp(A), m, n, n, float(eps), _lp(pr), _lp(pc), _dp(U), _dp(V))
    return pr[:k].copy(), pc[:k].copy(), U[:k].T.copy(), V[:k].T.copy()


def solve_right(M: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X with X M = B (LU with partial pivoting of M^T)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    X = np.zeros_like(B)
    rc = lib().orc_solve_right(_dp(M), M.shape[0], _dp(B), B.shape[0], _dp(X))
    if rc != 0:
        raise ZeroDivisionError("exactly singular pivot block")
    return X


def cdot(a: np.ndarray, b: np.ndarray) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return lib().orc_cdot(_dp(a), _dp(b), a.shape[0])


def kernel(cfg: Config, x: np.ndarray, y: np.ndarray) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    c = cfg.c()
    return lib().orc_kernel(C.byref(c), _dp(x), _dp(y))


def kernel_block(cfg: Config, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """K(X_i, Y_j) for all pairs (no diagonal rule)."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, cfg.d)
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(-1, cfg.d)
    out = np.zeros((X.shape[0], Y.shape[0]))
    c = cfg.c()
    lib().orc_kernel_block(C.byref(c), _dp(X), X.shape[0], _dp(Y), Y.shape[0], _dp(out))
    return out


def dense_matvec_pq(P: np.ndarray, Q: np.ndarray, x: np.ndarray, cfg: Config, rows=None,
                    block: int = 512) -> np.ndarray:
    """y = A x with A(i, j) = K(p_i, q_j), P and Q distinct point sets (Sec. 1, Eq. 1; no
    diagonal rule: coincident p_i = q_j give the kernel's value at r = 0, 0 for the singular
    kernels), on the rows `rows` of P (all if None), by blocks of rows."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    one = x.ndim == 1
    xx = x.reshape(1, -1) if one else x
    idx = np.arange(P.shape[0]) if rows is None else np.asarray(rows, dtype=np.int64)
    y = np.zeros((xx.shape[0], idx.shape[0]))
    for i0 in range(0, idx.shape[0], block):
        blk = kernel_block(cfg, P[idx[i0:i0 + block]], Q)
        y[:, i0:i0 + block] = xx @ blk.T
    return y[0] if one else y


def entry_block(h: "H2", rows, cols) -> np.ndarray:
    """A(rows, cols) of a built tree (sorted positions), with the diagonal rule."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    A = kernel_block(h.cfg, h.x[rows], h.x[cols])
    A[rows[:, None] == cols[None, :]] = h.cfg.kparam[2]
    return A
