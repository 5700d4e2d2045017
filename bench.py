#!/usr/bin/env python
"""Benchmark of the NNCA H^2 matrix-vector product on GB300.

Metric: H^2 matvec points/s (N * nrhs / product time) of the FP32-evaluation
form, on the 3D uniform 1/r workload (N = 1,048,576 points i.i.d. uniform in
[0,1]^3, K = 1/r, K(x,x) = 0, leaf size 64, ACA tolerance 1e-6, one vector
x ~ N(0,1)), gated on a relative error <= 1e-6 against the FP64 form of the
same handle.

One step is one H^2 product (Sec. 4 steps 2-5: permutation, P2M, M2M, M2L,
L2L, L2P, P2P, permutation back). The build of the representation (tree,
lists, ACA pivots, bases; Sec. 2-3) runs once per run before the timed
region and is reported in "build". Inputs are resident in HBM when the timed
region starts; L2 is flushed (256 MiB write) before every timed step, outside
the step's CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With --gpus N > 1 (under torchrun) every rank builds and times its own
replica of the workload (independent instances, no data exchange: the
product does not shard); the value is the points of all ranks over the
slowest rank's time. --impl reference times the FP64 CPU oracle's H^2
product on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_14832_gb300 import workloads as W  # noqa: E402

METRIC = "H2 matvec points/s at rel err <=1e-6: mixed-precision vs FP64 form, same GB300"
WORKLOAD = "invr3d_1m"
CPU_SAMPLE_N = 65536          # oracle sample: the same recipe at 65,536 points
MUFU_PER_CLK_SM = 16          # MUFU lanes per SM per clock: one rsqrt per pair
FP32_PER_CLK_SM = 128         # FP32 lanes per SM per clock
NEAR_OPS_PER_PAIR = 13        # FP32 lane-ops per near-field pair (hi/lo differences, squares, rsqrt scale, fma)


# timed arithmetic forms: name -> (nnca precision code, dtype label, description)
PRECISIONS = {
    "fp32": (1, "f32", "FP32 kernel evaluations (M2L, P2P), FP64 bases"),
    "tf32x3": (2, "tf32x3", "tensor-core M2L, 3xTF32 split operands, FP32 accumulation flushed into compensated "
                            "sums; FP32 P2P; FP64 bases"),
    "tf32": (3, "tf32", "tensor-core M2L, TF32 operands, FP32 accumulation; FP32 P2P; FP64 bases"),
    "bf16": (4, "bf16", "tensor-core M2L, BF16 operands, FP32 accumulation; FP32 P2P; FP64 bases"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=0, help="override N (not the benchmark workload)")
    ap.add_argument("--leaf-size", type=int, default=0, help="override the workload's leaf size nu")
    ap.add_argument("--tune", action="store_true",
                    help="pick the leaf size by timing the product (batch.tune_leaf_size over 64, 128, 256)")
    ap.add_argument("--workload", default="invr3d_1m",
                    choices=["invr3d_1m", "log2d_4096", "sphere_512k", "gauss_mix_256k", "cheb2d_102k", "cheb3d_262k",
                             "batch32", "fredholm3d"],
                    help="the headline is invr3d_1m; batch32: 32 independent problems in one captured graph; "
                         "fredholm3d: GMRES on the Nystrom system of the second-kind equation")
    ap.add_argument("--no-tune", action="store_true", help="batch32: keep leaf size 64 instead of tuning it")
    ap.add_argument("--precision", default="fp32", choices=list(PRECISIONS),
                    help="arithmetic of the timed product: fp32 (SIMT FP32 evaluations), or a tensor-core form "
                         "for many right-hand sides (tf32x3, tf32, bf16)")
    return ap.parse_args()


def workload_desc(w):
    if w.name.startswith("invr3d"):
        return (f"{w.name}: N={w.n} i.i.d. uniform in [0,1]^3, K=1/r, K(x,x)=0, leaf size {w.leaf_size}, "
                f"eta=sqrt(2), ACA tol {w.aca_tol:g}, nrhs {w.nrhs}, x~N(0,1)")
    return (f"{w.name}: N={w.n}, d={w.d}, {w.note}, leaf size {w.leaf_size}, eta=sqrt(2), ACA tol {w.aca_tol:g}, "
            f"nrhs {w.nrhs}")


def host_cores():
    return len(os.sched_getaffinity(0))


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_init(args):
    """Replicas: one process per GPU (RANK, LOCAL_RANK, WORLD_SIZE from torchrun), joined
    only for the barrier around the timed region and the slowest rank's time. NCCL on
    GPUs; gloo where no GPU is visible (the CPU tests of this host logic)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo", init_method="env://")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(ws, v: float) -> float:
    """The largest v over the ranks (the slowest replica's time)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ws: int, units_per_rank: float, steps: int, total_ms: float) -> float:
    """Whole-job throughput: the units every rank processed in `steps` steps over the
    slowest rank's time (weak scaling: each replica does the same work)."""
    return ws * units_per_rank * steps / (total_ms / 1e3)


def sample_size(w, n: int) -> int:
    """n, or for grid recipes the largest m^d not above n."""
    if w.points in ("chebyshev", "grid"):
        m = int(n ** (1.0 / w.d) + 1e-9)
        return m ** w.d
    return n


def oracle_sample(n: int, threads: int):
    """Build the oracle's H^2 on the workload recipe at n points; returns (h, x, build_s)."""
    from oracle import oracle as O
    w0 = W.WORKLOADS[WORKLOAD]
    w = w0.scaled(sample_size(w0, n))
    P = w.make_points()
    x = w.make_vector()
    cfg = O.Config(d=w.d, leaf_size=w.leaf_size, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    t0 = time.perf_counter()
    h = O.H2(P, cfg, nthreads=threads)
    return h, x, time.perf_counter() - t0


def cpu_baseline(threads: int) -> dict:
    os.environ["OMP_NUM_THREADS"] = str(threads)
    h, x, tb = oracle_sample(CPU_SAMPLE_N, threads)
    n = h.n
    nrhs = 1 if x.ndim == 1 else x.shape[0]
    h.matvec(x)
    t0 = time.perf_counter()
    reps = 3
    for _ in range(reps):
        h.matvec(x)
    t = (time.perf_counter() - t0) / reps
    # the same product on one thread (one product)
    t1 = time.perf_counter()
    h.matvec(x, nthreads=1)
    t1 = time.perf_counter() - t1
    return {"value": n * nrhs / t, "unit": "points/s", "cores": threads, "kind": "oracle",
            "value_1thread": n * nrhs / t1,
            "sample": f"FP64 oracle H2 product (on-the-fly form) on {n} points of the same recipe "
                      f"(oracle build {tb:.1f} s untimed), mean of {reps} products; value_1thread: one "
                      f"product on one thread"}


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    threads = host_cores()
    os.environ["OMP_NUM_THREADS"] = str(threads)
    h, x, tb = oracle_sample(CPU_SAMPLE_N, threads)
    for _ in range(args.warmup):
        h.matvec(x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        h.matvec(x)
    t = time.perf_counter() - t0
    value = CPU_SAMPLE_N * args.steps / t
    w = W.WORKLOADS[WORKLOAD]
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_desc(w), "sample_n": CPU_SAMPLE_N, "world_size": ws},
           "cpu_baseline": {"value": value, "unit": "points/s", "cores": threads, "kind": "oracle",
                            "sample": f"FP64 oracle H2 product on {CPU_SAMPLE_N} points of the same recipe per step "
                                      f"(build {tb:.1f} s untimed)"},
           "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import torch
    from paper_2203_14832_gb300 import _build, nnca

    ws, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    _build.build()
    w = W.WORKLOADS[WORKLOAD]
    if args.n:
        w = w.scaled(sample_size(w, args.n))
    if args.leaf_size:
        w = W.Workload(w.name, w.n, w.d, w.kernel, w.kparam, args.leaf_size, w.aca_tol, w.nrhs, w.seed, w.points,
                       w.vector, w.note)
    # independent replicas: every rank draws its own instance of the recipe
    if rank:
        w = W.Workload(w.name, w.n, w.d, w.kernel, w.kparam, w.leaf_size, w.aca_tol, w.nrhs, w.seed + 17 * rank,
                       w.points, w.vector, w.note)
    N, nrhs = w.n, w.nrhs
    stream = torch.cuda.current_stream()
    P = torch.as_tensor(w.make_points(), device="cuda")
    xh = w.make_vector()
    cfg = nnca.Config(d=w.d, leaf_size=w.leaf_size, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)

    prec, dtype_label, form = PRECISIONS[args.precision]
    leaf_times = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.tune:
        from paper_2203_14832_gb300 import batch
        h, leaf_times = batch.tune_leaf_size(P, cfg, torch.as_tensor(xh, device="cuda"), prec, (64, 128, 256))
        w = W.Workload(w.name, w.n, w.d, w.kernel, w.kparam, h.cfg.leaf_size, w.aca_tol, w.nrhs, w.seed, w.points,
                       w.vector, w.note)
    else:
        h = nnca.H2(P, cfg)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    st = h.stats()

    x = torch.as_tensor(xh, device="cuda")
    y32 = torch.empty_like(x)
    y64 = torch.empty_like(x)
    h.matvec(x, nnca.PREC_FP64, out=y64)
    h.matvec(x, prec, out=y32)
    torch.cuda.synchronize()
    y64h, y32h = y64.cpu().numpy(), y32.cpu().numpy()
    err32 = float(np.linalg.norm(y32h - y64h) / np.linalg.norm(y64h))

    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    for _ in range(args.warmup):
        h.matvec(x, prec, out=y32)
    torch.cuda.synchronize()

    # timed region: K products, CUDA events around each, L2 flushed before each
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(ws)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    h.set_profiling(True)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        h.matvec(x, prec, out=y32)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(ws)
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    st_prof = h.stats()
    h.set_profiling(False)
    total_ms = reduce_max(ws, float(sum(step_ms)))
    value = aggregate(ws, N * nrhs, args.steps, total_ms)

    # FP64 form of the same handle (a few products)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.fp64_steps):
        h.matvec(x, nnca.PREC_FP64, out=y64)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = e0.elapsed_time(e1) / args.fp64_steps

    # end to end through the C ABI with host buffers (pinned), copies inside
    xpin = torch.empty(N * nrhs, dtype=torch.float64, pin_memory=True)
    ypin = torch.empty(N * nrhs, dtype=torch.float64, pin_memory=True)
    xpin.numpy()[:] = np.asarray(xh, dtype=np.float64).ravel()
    e2e_steps = max(3, args.steps // 2)
    nnca.nnca_matvec_host(h.handle, xpin.numpy(), ypin.numpy(), nrhs, N, prec, stream)
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        nnca.nnca_matvec_host(h.handle, xpin.numpy(), ypin.numpy(), nrhs, N, prec, stream)
    e2e_s = reduce_max(ws, time.perf_counter() - t0)
    e2e_value = ws * N * nrhs * e2e_steps / e2e_s
    yh_e2e = ypin.numpy().copy().reshape((nrhs, N) if nrhs > 1 else (N,))

    if rank != 0:
        h.close()
        return

    # dense check on sampled rows (FP64 oracle dense product, host cores)
    from oracle import oracle as O
    ocfg = O.Config(d=w.d, leaf_size=w.leaf_size, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    # every row for small problems, else 4096 sampled rows
    nrows = N if N <= 16384 else 4096
    rows = np.arange(N) if nrows == N else np.random.default_rng(12345).choice(N, nrows, replace=False)
    os.environ.setdefault("OMP_NUM_THREADS", str(host_cores()))
    x0 = xh if xh.ndim == 1 else xh[0]       # the dense check takes the first right-hand side
    y64f = y64h if y64h.ndim == 1 else y64h[0]
    y32f = y32h if y32h.ndim == 1 else y32h[0]
    yd = O.dense_rows(w.make_points(), rows, x0, ocfg)
    err_dense = float(np.linalg.norm(y64f[rows] - yd) / np.linalg.norm(yd))
    err_dense32 = float(np.linalg.norm(y32f[rows] - yd) / np.linalg.norm(yd))
    e2e_ok = bool(np.array_equal(yh_e2e, y32h))

    # roofline of the dominant kernel (M2L, FP32 evaluation): one rsqrt per pivot pair
    # per product: the profiled region is exactly the K timed products (a product
    # of several right-hand sides records one set of pass events per group)
    calls = max(1, args.steps)
    m2l_ms = st_prof["pass_ms"][2] / calls
    pass_ms = [v / calls for v in st_prof["pass_ms"][:6]]
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak_gpair = MUFU_PER_CLK_SM * sms * sm_max * 1e6 / 1e9
    tc = args.precision != "fp32"
    passes = pass_rooflines(h, st, pass_ms, sms, sm_max, peaks, nrhs, args.precision)
    # kernel evaluations of the pass: each pivot pair once in the symmetric form
    # (a value serves the row and the column sum), else every ordered pair
    evals = st.get("m2l_evals") or st["m2l_pairs"]
    sym = evals < st["m2l_pairs"]
    m2l_kernel = "k_m2l_sym" if sym else "k_m2l_group"
    achieved = evals / (m2l_ms / 1e3) / 1e9
    traffic = None
    tf = os.path.join(ROOT, "profiles", ("m2l_sym" if sym else "m2l_group") + "_traffic_invr3d.json")
    traffic_note = None
    if os.path.exists(tf) and w.name == "invr3d_1m" and w.n == 1 << 20:
        try:
            tj = json.load(open(tf))
            traffic, traffic_note = tj.get("bytes_per_launch"), tj.get("note")
        except Exception:
            traffic = None

    roofline = {"bound": "alu", "kernel": m2l_kernel, "achieved": achieved, "peak": peak_gpair,
                "unit": "G kernel evaluations/s", "frac": achieved / peak_gpair, "traffic": traffic,
                "peak_note": f"one MUFU rsqrt per evaluation: {MUFU_PER_CLK_SM}/clk/SM x {sms} SMs x "
                             f"{sm_max:.0f} MHz",
                "pairs_served_per_s_frac": st["m2l_pairs"] / (m2l_ms / 1e3) / 1e9 / peak_gpair,
                "pairs_note": "symmetric form: each evaluation feeds two ordered pivot pairs (a row and "
                              "a column sum); this fraction counts those pairs against the same peak",
                "traffic_note": ("DRAM bytes read + written by one M2L launch: " + traffic_note) if traffic_note
                else "no full-size ncu DRAM figure for this kernel and workload"}
    if tc or nrhs > 1:
        # several right-hand sides: the M2L pass's own entry (tensor-core flops, or
        # MUFU evaluations of the four-RHS kernel summed over the product's passes)
        p0 = passes[0]
        scale = 1e12 if p0["unit"] == "flops" else 1e9
        roofline = {"bound": p0["bound"], "kernel": p0["kernels"], "achieved": p0["achieved"] / scale,
                    "peak": p0["peak"] / scale, "unit": "TFLOP/s" if p0["unit"] == "flops" else "G kernel evaluations/s",
                    "frac": p0["frac"], "traffic": None, "peak_note": p0["note"],
                    "traffic_note": "no full-size ncu DRAM figure for this kernel and workload"}

    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(host_cores())

    out = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_label, "data": "synthetic",
        "config": {"workload": workload_desc(w), "form": form,
                   "leaf_size_tuning": {str(k): v for k, v in leaf_times.items()} if leaf_times else None,
                   "l2": "flushed (256 MiB write) before every timed step", "parallelism": f"replicas x{ws}"},
        "rel_err_fp32_vs_fp64": err32, "rel_err_fp64_vs_dense": err_dense,
        "rel_err_fp32_vs_dense": err_dense32, "dense_rows": int(nrows),
        "fp64_form": {"value": N * nrhs / (fp64_ms / 1e3), "unit": "points/s", "ms_per_step": fp64_ms},
        "speedup_fp32_vs_fp64": fp64_ms / (total_ms / args.steps),
        "build": {"s": build_s, "ms_phases": st["build_ms"][:6], "kappa": st["kappa"], "lmin": st["lmin"],
                  "ncell": st["ncell"], "n_pivots": st["n_pivots"], "max_rank": st["max_rank"],
                  "aca_retries": st["aca_retries"], "device_bytes": st["device_bytes"]},
        "work": {"m2l_pairs": st["m2l_pairs"], "m2l_evals": evals, "p2p_pairs": st["p2p_pairs"]},
        "pass_ms": {"perm": pass_ms[0], "p2m_m2m": pass_ms[1], "m2l": pass_ms[2], "l2l": pass_ms[3],
                    "l2p_p2p": pass_ms[4], "total": pass_ms[5]},
        "roofline": roofline,
        "roofline_passes": passes,
        "dominant_pass": max((p for p in passes if p.get("ms")), key=lambda p: p["ms"])["pass"],
        "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": N * nrhs * 8,
                "d2h_bytes_per_step": N * nrhs * 8, "matches_device_result": e2e_ok},
        "gpu_launches": int(st_prof["launches_per_product"]) * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "wall_s_timed": wall,
    }
    print(json.dumps(out), flush=True)
    h.close()
    if err32 > 1e-6 and WORKLOAD == "invr3d_1m":
        print(f"error gate failed: FP32 form {err32:.3e} > 1e-6 against FP64", file=sys.stderr)
        sys.exit(3)


def pass_rooflines(h, st, pass_ms, sms, sm_mhz, peaks, nrhs, precision="fp32"):
    """Achieved fraction of its roofline for every pass of one product of nrhs
    right-hand sides (pass times from CUDA events on the launching stream, summed
    over the product's passes; the work below is summed the same way).

    Algorithmic work per pass (counted exactly from the built representation):
      M2L     kernel evaluations (m2l_evals), one MUFU rsqrt each
      P2P+L2P point pairs (p2p_pairs), bound by the FP32 pipe at NEAR_OPS_PER_PAIR
              lane-ops per pair (below the MUFU rate of one rsqrt per pair)
      P2M+M2M operator bytes (FP64 bases of every cell, read once per pass) plus the
              vector in tree order and the multipole coefficients, against HBM
      L2L     FP64 translation operators of the non-leaf cells plus the local
              coefficients (read and written), against HBM
    The build's k_aca (FP64 ACA) is reported from its ncu capture, whose FP64-pipe
    activity is the fraction."""
    lb = h.export("LEVEL_BASE")
    op_off = h.export("OP_OFF")
    op_nonleaf = int(op_off[lb[st["kappa"]]])
    op_all = int(st["op_entries"])
    npiv, n = int(st["n_pivots"]), int(st["n"])
    clk = sm_mhz * 1e6
    hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
    hbm_note = "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"

    def ent(name, kernels, bound, work, unit, ms, peak, note):
        ach = work / (ms / 1e3) if ms > 0 else 0.0
        return {"pass": name, "kernels": kernels, "bound": bound, "work": work, "unit": unit, "ms": ms,
                "achieved": ach, "peak": peak, "frac": ach / peak if peak else None, "note": note}

    # How the product groups its right-hand sides. FP32 form: passes of four (every
    # ordered pivot pair evaluated once for the four; near field and operators once
    # per pass), the rest one at a time (symmetric M2L: each pivot pair once).
    # Tensor-core forms: M2L passes of up to 64, operators in groups of eight (then
    # four, then one), near field in groups of four (then one).
    sym_evals = st.get("m2l_evals") or st["m2l_pairs"]
    if precision == "fp32":
        quads, singles = nrhs // 4, nrhs % 4
        m2l_work = st["m2l_pairs"] * quads + sym_evals * singles
        near_groups = quads + singles
        op_groups = quads + singles
    else:
        near_groups = nrhs // 4 + nrhs % 4
        op_groups = nrhs // 8 + (nrhs % 8) // 4 + nrhs % 4
    if precision != "fp32":
        # tensor-core M2L: useful flops of the contraction (2 per pivot pair and
        # right-hand side, times the products per pair), against the tf32 dense
        # peak = measured bf16 peak x nominal tf32/bf16 ratio (1.1 / 2.25)
        prods = 3 if precision == "tf32x3" else 1
        bf16 = float(peaks.get("bf16_tflops", 1900.0)) * 1e12
        m2l = ent("m2l", "k_m2l_tc (+ pack, unpack)", "tensor", 2.0 * prods * st["m2l_pairs"] * nrhs, "flops",
                  pass_ms[2], bf16 * 1.1 / 2.25, f"{prods} tf32 products per pivot pair and right-hand side, up to "
                  "64 right-hand sides per pass; peak: measured bf16 x 1.1/2.25"
                  + ("" if "bf16_tflops" in peaks else " (fallback)"))
        m2l["mufu_frac"] = st["m2l_pairs"] / (pass_ms[2] / 1e3) / (MUFU_PER_CLK_SM * sms * clk) if pass_ms[2] else None
    else:
        m2l = ent("m2l", "k_m2l_sym + k_m2l_cols" if nrhs == 1 else "k_m2l_group_rhs", "alu", m2l_work,
                  "kernel evaluations", pass_ms[2], MUFU_PER_CLK_SM * sms * clk,
                  "one MUFU rsqrt (or ex2) per kernel evaluation")
    out = [
        m2l,
        ent("l2p_p2p", "k_near_group" if nrhs == 1 else "k_near_rhs", "alu", st["p2p_pairs"] * near_groups,
            "point pairs (evaluations)", pass_ms[4], FP32_PER_CLK_SM / NEAR_OPS_PER_PAIR * sms * clk,
            f"FP32 pipe at {NEAR_OPS_PER_PAIR} lane-ops per pair, one evaluation per pair and group of up to 4 "
            "right-hand sides; includes the FP64 L2P of the same kernel"),
        ent("p2m_m2m", "k_upward", "hbm", 8 * (op_all * op_groups + nrhs * (n + npiv)), "bytes", pass_ms[1], hbm,
            "FP64 operators of every cell (once per group of right-hand sides) + x in tree order + w; " + hbm_note),
        ent("l2l", "k_l2l", "hbm", 8 * (op_nonleaf * op_groups + 2 * nrhs * npiv), "bytes", pass_ms[3], hbm,
            "FP64 translations of the non-leaf cells (once per group) + u read and written; " + hbm_note),
    ]
    af = os.path.join(ROOT, "profiles", "aca_invr3d_131k.json")
    if os.path.exists(af):
        try:
            a = json.load(open(af))
            out.append({"pass": "build_aca", "kernels": "k_aca", "bound": "fp64", "frac": a.get("fp64_pipe_frac"),
                        "note": a.get("note"), "source": "profiles/aca_invr3d_131k.json"})
        except Exception:
            pass
    return out


def run_batch(args):
    """32 independent problems of uneven size (batch32 recipe), FP32 form, 8 RHS each:
    leaf sizes tuned per problem (untimed), one batched product captured into a CUDA
    graph, K replays timed with CUDA events (L2 flushed before each)."""
    import torch
    from paper_2203_14832_gb300 import _build, batch, nnca

    ws_, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    _build.build()
    wls = W.batch_workloads(seed=5000 + 1000 * rank)
    probs = []
    for w in wls:
        P = torch.as_tensor(w.make_points(), device="cuda")
        cfg = nnca.Config(d=w.d, leaf_size=w.leaf_size, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
        probs.append(batch.Problem(P, cfg, torch.as_tensor(np.ascontiguousarray(w.make_vector()), device="cuda")))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prec, dtype_label, form = PRECISIONS[args.precision]
    b = batch.Batch(probs, precision=prec, tune=not args.no_tune)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    # per-problem error of the FP32 form against the FP64 form of the same handle
    y32 = [y.clone() for y in b.matvec()]
    errs = []
    for h, x, y in zip(b.handles, b.x, y32):
        y64 = h.matvec(x, nnca.PREC_FP64)
        errs.append(float(torch.linalg.norm(y - y64) / torch.linalg.norm(y64)))
    g = b.capture()
    for _ in range(args.warmup):
        g.replay()
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(ws_)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        g.replay()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(ws_)
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(c) for a, c in ev]
    total_ms = reduce_max(ws_, sum(step_ms))
    pts = b.points()
    value = aggregate(ws_, pts, args.steps, total_ms)
    # end to end: host inputs copied in, graph replayed, results copied out, every step
    xh = [x.cpu().pin_memory() for x in b.x]
    yh = [torch.empty_like(y, device="cpu").pin_memory() for y in b.y]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for d, hsrc in zip(b.x, xh):
            d.copy_(hsrc, non_blocking=True)
        g.replay()
        for hdst, d in zip(yh, b.y):
            hdst.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = reduce_max(ws_, time.perf_counter() - t0)
    m2l_pairs = sum(h.stats()["m2l_pairs"] for h in b.handles)
    if rank != 0:
        b.close()
        return
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak_gpair = MUFU_PER_CLK_SM * sms * sm_max * 1e6 / 1e9
    achieved = m2l_pairs * b.nrhs / (total_ms / args.steps / 1e3) / 1e9
    out = {
        "metric": f"batched H2 matvec points/s, 32 uneven problems, {args.precision} form", "value": value,
        "unit": "points/s", "n_gpus": ws_, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype_label, "data": "synthetic", "form": form,
        "config": {"workload": "batch32: 32 problems, N log-uniform in [16384, 524288], U[0,1]^3, 16x 1/r + 16x "
                               "Gaussian h=0.2, ACA tol 1e-6, 8 RHS", "sizes": [h.n for h in b.handles],
                   "leaf_sizes": [h.cfg.leaf_size for h in b.handles], "tuned": not args.no_tune,
                   "l2": "flushed (256 MiB write) before every timed step", "graph": "one CUDA graph per step"},
        "rel_err_fp32_vs_fp64": {"max": max(errs), "per_problem": errs},
        "build_s_with_tuning": build_s,
        "roofline": {"bound": "alu", "kernel": "whole step", "achieved": achieved, "peak": peak_gpair,
                     "unit": "Gpair/s", "frac": achieved / peak_gpair, "traffic": None,
                     "note": "all M2L pivot pairs of the batch over the whole step time (a lower bound on the M2L rate)"},
        "e2e": {"value": ws_ * pts * args.steps / e2e_s, "unit": "points/s",
                "h2d_bytes_per_step": sum(x.numel() * x.element_size() for x in b.x),
                "d2h_bytes_per_step": sum(y.numel() * y.element_size() for y in b.y)},
        "gpu_launches": sum(int(h.stats()["launches_per_product"]) for h in b.handles) * args.steps,
        "clocks": clocks,
        "cpu_baseline": None,
    }
    print(json.dumps(out), flush=True)
    b.close()


def run_fredholm(args):
    """Sec. 5 Experiment 5: the Nystrom system (I + h^3 K) sigma = f on the 64^3 grid,
    f = A sigma for a random sigma, solved by GMRES to 1e-10 with the FP64 product."""
    import torch
    from paper_2203_14832_gb300 import _build, nnca
    from paper_2203_14832_gb300.solve import gmres

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if int(os.environ.get("RANK", "0")) != 0:
        return
    _build.build()
    w = W.WORKLOADS["fredholm3d_262k"]
    if args.n:
        w = w.scaled(sample_size(w, args.n))
    P = torch.as_tensor(w.make_points(), device="cuda")
    cfg = nnca.Config(d=w.d, leaf_size=w.leaf_size, aca_tol=w.aca_tol, kernel=w.kernel, kparam=w.kparam)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = nnca.H2(P, cfg)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    sigma = torch.as_tensor(w.make_vector(), device="cuda")
    f = h.matvec(sigma)
    y = torch.empty_like(f)
    for _ in range(args.warmup):
        h.matvec(f, out=y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, it, hist = gmres(lambda v: h.matvec(v), f, tol=1e-10)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    err = float(torch.linalg.norm(x - sigma) / torch.linalg.norm(sigma))
    out = {"metric": "GMRES solve time, second-kind Nystrom system (FP64 H2 products)", "value": solve_s,
           "unit": "s", "n_gpus": 1, "steps": 1, "warmup": args.warmup, "ms_per_step": solve_s * 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"fredholm3d: {w.n} points, cell-centred grid on [-1,1]^3, A = I + h^3/r, "
                                  f"ACA tol {w.aca_tol:g}, GMRES tol 1e-10, sigma ~ N(0,1), f = A sigma"},
           "iterations": it, "relative_forward_error": err, "final_relative_residual": hist[-1] if hist else 0.0,
           "build_s": build_s, "points_per_s_per_product": w.n * it / solve_s}
    print(json.dumps(out), flush=True)
    h.close()


def main():
    global WORKLOAD
    args = parse()
    if args.workload not in ("batch32", "fredholm3d"):
        WORKLOAD = args.workload
    if args.workload == "fredholm3d":
        run_fredholm(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch32":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
