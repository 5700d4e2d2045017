"""Batched independent H^2 problems: leaf-size tuning, the batched product, and
its capture into a CUDA graph.

Everything here is marshalling around the C ABI: the products run in
``nnca_matvec_batch`` (independent problems on worker streams forked from and
joined back to the caller's stream), and the tuner only builds handles and
times their products with CUDA events.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import nnca

LEAF_CANDIDATES = (32, 64, 96, 128)


def time_product(h: "nnca.H2", x, y, precision: int, reps: int = 5) -> float:
    """Mean device time (ms) of `reps` products after one warm-up, by CUDA events."""
    import torch
    h.matvec(x, precision, out=y)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        h.matvec(x, precision, out=y)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_leaf_size(P, cfg: "nnca.Config", x, precision: int = nnca.PREC_FP32,
                   candidates=LEAF_CANDIDATES, reps: int = 5):
    """Build the problem with every candidate leaf size, time its product on x, and
    keep the fastest. Returns (handle of the best leaf size, {leaf size: ms})."""
    import torch
    best, times = None, {}
    y = torch.empty_like(x)
    for nu in candidates:
        c = nnca.Config(d=cfg.d, leaf_size=nu, eta2_num=cfg.eta2_num, eta2_den=cfg.eta2_den, aca_tol=cfg.aca_tol,
                        kernel=cfg.kernel, kparam=cfg.kparam)
        h = nnca.H2(P, c)
        times[nu] = time_product(h, x, y, precision, reps)
        if best is None or times[nu] < times[best[0]]:
            if best is not None:
                best[1].close()
            best = (nu, h)
        else:
            h.close()
    return best[1], times


@dataclass
class Problem:
    P: object          # CUDA float64 tensor (n, d)
    cfg: object        # nnca.Config
    x: object          # CUDA tensor (nrhs, n) or (n,)


class Batch:
    """A set of independent problems with one batched product.

    tune=True picks each problem's leaf size with ``tune_leaf_size``."""

    def __init__(self, problems: list, precision: int = nnca.PREC_FP32, tune: bool = False,
                 candidates=LEAF_CANDIDATES):
        import torch
        self.precision = precision
        self.handles, self.leaf_times = [], []
        for p in problems:
            if tune:
                h, t = tune_leaf_size(p.P, p.cfg, p.x, precision, candidates)
            else:
                h, t = nnca.H2(p.P, p.cfg), {}
            self.handles.append(h)
            self.leaf_times.append(t)
        self.x = [p.x.contiguous() for p in problems]
        self.y = [torch.empty_like(x) for x in self.x]
        nr = {1 if x.dim() == 1 else x.shape[0] for x in self.x}
        assert len(nr) == 1, "one number of right-hand sides for the whole batch"
        self.nrhs = nr.pop()
        self.graph = None

    def matvec(self, stream=None):
        """y_k = A_k x_k for every problem (asynchronous on the stream)."""
        nnca.nnca_matvec_batch([h.handle for h in self.handles], self.x, self.y, self.nrhs,
                               [h.n for h in self.handles], self.precision, stream)
        return self.y

    def capture(self):
        """Capture one batched product into a CUDA graph (after an uncaptured call,
        which allocates the workspaces). Replay with ``self.graph.replay()``."""
        import torch
        self.matvec()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.matvec()
        self.graph = g
        return g

    def points(self) -> int:
        return sum(h.n for h in self.handles) * self.nrhs

    def close(self):
        for h in self.handles:
            h.close()
        self.handles = []
