"""The replica path of bench.py (--gpus N under torchrun) on the CPU: two gloo ranks
join, the barrier passes, the reduction returns the slowest rank's time on every rank,
and the whole-job throughput counts every rank's units over that time."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, _ = bench.dist_init(None)
    assert (w, r) == (ws, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    t = bench.reduce_max(w, 10.0 + 5.0 * rank)      # the ranks' timed totals, ms
    out.put((rank, t, bench.aggregate(w, 1000.0, 4, t)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(ws))
    for rank, t, v in res:
        assert t == 15.0                                  # the slowest rank's time on every rank
        assert abs(v - 2 * 1000.0 * 4 / 0.015) < 1e-6    # both ranks' units over that time


def test_aggregate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(1, 3.5) == 3.5
    assert abs(bench.aggregate(1, 1 << 20, 20, 146.0) - (1 << 20) * 20 / 0.146) < 1e-3
