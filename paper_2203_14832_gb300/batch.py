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
TILE_CANDIDATES = (0, 128)   # M2L targets per work item (0: 256)


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
                   candidates=LEAF_CANDIDATES, reps: int = 5, tiles=TILE_CANDIDATES):
    """Pick the leaf size and then the M2L tile (targets per work item) by timing.

    Every candidate leaf size is built (default tile) and its product timed on x;
    with the fastest one kept, every tile of `tiles` is built and timed. Returns
    (handle of the best configuration, {"nu/tile": ms})."""
    import torch
    y = torch.empty_like(x)
    times = {}

    def build(nu, tile):
        c = nnca.Config(d=cfg.d, leaf_size=nu, eta2_num=cfg.eta2_num, eta2_den=cfg.eta2_den, aca_tol=cfg.aca_tol,
                        kernel=cfg.kernel, kparam=cfg.kparam, m2l_form=cfg.m2l_form, m2l_item_targets=tile)
        return nnca.H2(P, c)

    best = None   # (ms, nu, tile, handle)
    for nu in candidates:
        h = build(nu, 0)
        t = time_product(h, x, y, precision, reps)
        times[f"{nu}/0"] = t
        if best is None or t < best[0]:
            if best is not None:
                best[3].close()
            best = (t, nu, 0, h)
        else:
            h.close()
    for tile in tiles:
        if tile == 0:
            continue
        h = build(best[1], tile)
        t = time_product(h, x, y, precision, reps)
        times[f"{best[1]}/{tile}"] = t
        if t < best[0]:
            best[3].close()
            best = (t, best[1], tile, h)
        else:
            h.close()
    return best[3], times


@dataclass
class Problem:
    P: object          # CUDA float64 tensor (n, d)
    cfg: object        # nnca.Config
    x: object          # CUDA tensor (nrhs, n) or (n,)


class Batch:
    """A set of independent problems with one batched product.

    tune=True picks each problem's leaf size and M2L tile with ``tune_leaf_size``."""

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
