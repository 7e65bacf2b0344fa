#!/usr/bin/env python3
"""Benchmark: overdecomposed 3D 7-point FP64 Jacobi on GB300.

Default workload: 512^3 interior (every cell U[0,1), seed 2), 4096 chares of
32^3, persistent path, 100 timed iterations after warm-up.  A "step" is one
Jacobi iteration over the whole grid (compute + face delivery for every
chare).  The two parity buffers (2 x 2.3 GB) are far larger than the 129 MB
L2, so no flush is needed between iterations.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the host cores instead (the only reference this workload has).  Under
torchrun each rank runs an independent replica on its own GPU (the solve has
no cross-GPU exchange on a one-GPU-per-box pool: weak scaling, replicas).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-pt updates/s & HBM GB/s vs ODF (fused vs per-chare); p50/p99 job latency"
UNIT = "grid-pt updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="odf", choices=["odf", "uneven", "ceiling", "serve", "jacobi2d", "launch", "shards"],
                    help="odf: 512^3 at --odf (default); uneven: 768x512x512 in ~300 uneven chares; "
                         "ceiling: 1024^3 in 4096 chares; serve: Poisson stream of jobs into the server; "
                         "jacobi2d: the 2D 5-point Jacobi on 32768^2 in --odf chares (a power of two); "
                         "launch: the kernel-launch overhead microbenchmarks; shards: 512^3 at ODF 4096 split "
                         "over 1-8 contexts (and 2 processes) exchanging faces through communication endpoints")
    ap.add_argument("--jobs", type=int, default=300, help="serve: number of jobs")
    ap.add_argument("--rate", type=float, default=60.0, help="serve: Poisson arrival rate (jobs/s)")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serve: HBM budget")
    ap.add_argument("--batch-steps", type=int, default=0,
                    help="serve: steps of every running job per batched launch (0 = the server's default)")
    ap.add_argument("--job-streams", type=int, default=-1,
                    help="serve: 0 = batched launches, N > 0 = one persistent launch per job on N streams "
                         "(-1 = the default)")
    ap.add_argument("--odf", type=int, default=4096)
    ap.add_argument("--edge", type=int, default=512)
    ap.add_argument("--edge2d", type=int, default=32768, help="jacobi2d: grid edge (the paper's 32768)")
    ap.add_argument("--path", default="persistent",
                    choices=["per_chare", "fused", "graph", "persistent", "fused_graph"])
    ap.add_argument("--baseline-steps", type=int, default=3,
                    help="timed steps of the per-chare-launch baseline at the same ODF (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="also time every path at every ODF (adds a 'sweep' key; on by default for the odf "
                         "workload at N=1)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the default ODF sweep")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the default run's other workloads (uneven, ceiling, serving)")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (default: od_create times candidate execution shapes first)")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--cpt", type=int, default=0)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--tile-y", type=int, default=0)
    ap.add_argument("--tile-z", type=int, default=0)
    ap.add_argument("--order", type=int, default=0,
                    help="persistent task order (od_config.order: 1 reverse odd steps, 2 Morton chares)")
    ap.add_argument("--arith", type=int, default=-1,
                    help="where the update's operations run (od_config.arith; -1 = library default)")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in a thread."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# GB300 unit counts and clock (profiling recipe): 152 SMs, 2.07 GHz maximum
# SM clock, FP64 1.25 TFLOP/s nominal = 2 FMA lanes per SM per clock.
SMS = 152
SM_MAX_GHZ = 2.07
FP64_LANES_PER_SM = 2
FP64_NOMINAL_GFLOPS = 1250.0
FLOPS_PER_UPDATE = 6  # 5 additions + 1 division
FLOPS_PER_UPDATE_2D = 4  # 3 additions + 1 division


def profiled_kernel(args, plan):
    """The committed ncu summary of the tile kernel (profiles/traffic_*.json:
    DRAM bytes per step, thread instructions per update) when it was taken
    on this exact kernel revision, shape and workload; None otherwise."""
    if args.workload == "jacobi2d":
        name = f"traffic_{args.path}2d_{args.edge2d}sq_odf{args.odf}.json"
    elif args.workload == "odf":
        name = f"traffic_{args.path}_{args.edge}cubed_odf{args.odf}.json"
    else:
        return None
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    rev = KERNEL_REV_2D if args.workload == "jacobi2d" else KERNEL_REV
    if d.get("arith") != plan["arith"] or d.get("threads") != plan["threads"] or \
            d.get("cells_per_thread") != plan["cells_per_thread"] or d.get("kernel_rev") != rev:
        return None
    return d


# bumped whenever a tile kernel changes, so stale profiler counters are not reused
KERNEL_REV = 16     # 3D 7-point
KERNEL_REV_2D = 16  # 2D 5-point


def combine_ranks(ms: float, updates: float, world: int, device: str):
    """Whole-job timing across replicas: the slowest rank's time (max over
    ranks) and the updates of all ranks divided by it.  world == 1 needs no
    process group."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms, updates], dtype=torch.float64, device=device)
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t.clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        ms, updates = float(tmax[0].item()), float(tsum[1].item())
    return ms, updates / (ms * 1e-3)


def workload_config(name: str, dims, odf: int, stencil: str, seed: int, world: int) -> dict:
    """The workload's description, identical in both arms' lines (the
    execution shape of our arm goes under the line's separate "launch")."""
    cells = dims[0] * dims[1] * dims[2]
    return {"workload": name, "nx": dims[0], "ny": dims[1], "nz": dims[2], "odf": odf, "stencil": stencil,
            "seed": seed, "init": "U[0,1) everywhere, Dirichlet shell fixed",
            "l2": f"no flush: the two parity buffers ({2 * 8 * cells / 2**30:.1f} GiB) far exceed the 129 MB L2",
            "parallelism": f"replicas x{world}"}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _time_oracle(sweep, cells: int, target_s: float):
    """Rate of an oracle sweep function sweep(iters): grow the iteration
    count until one call lasts about target_s, then take the rate from the
    difference of the last two calls (their one-off copy and page faults
    cancel).  Returns (updates/s, iterations of the last call, its seconds)."""
    def timed(n):
        t0 = time.perf_counter()
        sweep(n)
        return time.perf_counter() - t0
    n0, t0 = 1, timed(1)
    n1 = max(2, int(target_s / 2 / max(t0, 1e-3)))
    t1 = timed(n1)
    if t1 < target_s / 4:  # the first call was dominated by its one-off cost
        n1 = max(n1 + 1, int(n1 * target_s / 2 / t1))
        t1 = timed(n1)
    n2 = max(n1 + 1, int(n1 * target_s / t1))
    t2 = timed(n2)
    if t2 - t1 < 0.25 * t2 * (n2 - n1) / n2:  # noise swamped the difference: count the whole call
        return n2 * cells / t2, n2, t2
    rate = (n2 - n1) * cells / (t2 - t1)
    return rate, n2, t2


def oracle_cpu_baseline(edge: int, target_s: float = 10.0, e2e_out=None, e2e_iters: int = 100):
    """Time the CPU oracle's monolithic sweep (its OpenMP z-plane split) on a
    bounded sample of the same workload: the full edge^3 field, iterated for
    about target_s seconds.  With e2e_out (the end-to-end run's last result,
    u^e2e_iters of the same field), also solve that job on the oracle and
    compare every cell."""
    import numpy as np
    import oracle
    from paper_2605_12734_gb300 import inputs
    oracle.build()
    threads = oracle.max_threads()
    P = oracle.init_padded(edge, edge, edge, 2, inputs.INIT_UNIFORM)
    ups, iters, dt = _time_oracle(lambda n: oracle.sweep(P, n, threads), edge ** 3, target_s)
    ups1, iters1, dt1 = _time_oracle(lambda n: oracle.sweep(P, n, 1), edge ** 3, target_s / 2)
    out = {"value": ups, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{edge}^3 field (U[0,1), seed 2), undecomposed C oracle sweep on {threads} OpenMP threads; "
                     f"rate from the difference of calls of increasing length, the last {iters} "
                     f"iterations in {dt:.1f} s",
           "single_core": {"value": ups1, "unit": UNIT, "cores": 1,
                           "sample": f"the same on one thread, the last {iters1} iterations in {dt1:.1f} s"}}
    # the method itself on the CPU: the decomposed oracle (per-block arrays,
    # explicit face copies, one thread) at ODF 4096 on the same field, and
    # the small parity case (64^3, interior 0, in 1 or 8 blocks, 10 iterations)
    ez = oracle.split(edge, 16)
    upsd, itd, dtd = _time_oracle(lambda n: oracle.sweep_decomposed(P, ez, ez, ez, n), edge ** 3, target_s / 3)
    out["decomposed_odf4096"] = {"value": upsd, "unit": UNIT, "cores": 1,
                                 "sample": f"{edge}^3 in 16^3 blocks, decomposed C oracle on one thread, the last "
                                           f"{itd} iterations in {dtd:.1f} s"}
    P64 = oracle.init_padded(64, 64, 64, 1, inputs.INIT_ZERO_INTERIOR)
    e64 = oracle.split(64, 2)
    small = {}
    for key, fn in (("odf1", lambda: oracle.sweep(P64, 10, 1)),
                    ("odf8", lambda: oracle.sweep_decomposed(P64, e64, e64, e64, 10))):
        best = float("inf")
        for _ in range(5):
            t0 = time.perf_counter()
            fn()
            best = min(best, time.perf_counter() - t0)
        small[key] = 64 ** 3 * 10 / best
    out["small_64cubed"] = {"odf1_updates_per_s": small["odf1"], "odf8_updates_per_s": small["odf8"], "cores": 1,
                            "sample": "64^3 (interior 0, shell U[0,1) seed 1), 10 iterations, best of 5 calls "
                                      "(one-off copy included)"}
    if e2e_out is not None:
        t0 = time.perf_counter()
        want = oracle.solve(edge, edge, edge, 2, inputs.INIT_UNIFORM, e2e_iters, threads)
        out["e2e_oracle_seconds"] = time.perf_counter() - t0
        diff = int(np.count_nonzero(np.ascontiguousarray(e2e_out).view(np.uint64) != want.view(np.uint64)))
        out["e2e_cells_differing_from_oracle"] = diff
    return out


def oracle_cpu_baseline_2d(edge: int, target_s: float = 10.0):
    """The same for the 2D workload: the C oracle's 2D sweep of the full
    edge^2 field."""
    import oracle
    from paper_2605_12734_gb300 import inputs
    oracle.build()
    threads = oracle.max_threads()
    P = oracle.init_padded_2d(edge, edge, 9, inputs.INIT_UNIFORM)
    ups, iters, dt = _time_oracle(lambda n: oracle.sweep_2d(P, n, threads), edge ** 2, target_s)
    return {"value": ups, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{edge}^2 field (U[0,1), seed 9), undecomposed C oracle 2D sweep on {threads} OpenMP "
                      f"threads; rate from the difference of calls of increasing length, the last {iters} "
                      f"iterations in {dt:.1f} s"}


# ----------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    edge = args.edge
    import oracle
    from paper_2605_12734_gb300 import inputs
    oracle.build()
    threads = oracle.max_threads()
    P = oracle.init_padded(edge, edge, edge, 2, inputs.INIT_UNIFORM)
    # Each "step" is a bounded sample: m oracle iterations over the full grid,
    # m sized to about a second of CPU work.  Every oracle call copies the
    # field and touches fresh pages, so the rate comes from calls of growing
    # length (the difference of the last two cancels that one-off cost),
    # over about K seconds of oracle work in all (4 at least, 40 at most).
    K = max(1, args.steps)
    W = max(0, args.warmup)
    oracle.sweep(P, max(1, min(W, 3)), threads)  # warm-up: OpenMP threads, the library's pages
    ups, _, _ = _time_oracle(lambda n: oracle.sweep(P, n, threads), edge ** 3, float(min(max(K, 4), 40)))
    m = max(1, int(round(ups / edge ** 3)))  # iterations in about a second
    dt = K * m * edge ** 3 / ups
    line = {"impl": "reference", "metric": METRIC, "value": ups, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": dt * 1e3 / K, "higher_is_better": True,
            "iters_per_step": m,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(f"jacobi3d-{edge}^3-odf{args.odf}", (edge, edge, edge), args.odf, "3d7", 2,
                                      args.gpus),
            "note": "CPU oracle: the undecomposed sweep, which gives the same bits for any ODF; a step is "
                    f"{m} oracle iterations (about a second)",
            "cpu_baseline": {"value": ups, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{edge}^3 field, steps of {m} iterations on {threads} threads; rate "
                                       f"from the difference of oracle calls of growing length over about "
                                       f"{min(max(K, 4), 40)} s"},
            "e2e": {"value": ups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- our arm

def time_path(pkg, edge, odf, path, steps, warmup, stream, tune_kw, make=None):
    """Device-resident timing of `steps` iterations; returns (ms/step, stats).
    make(path, **kw) builds the solver (default: edge^3 in odf cubic chares)."""
    import torch
    if make is None:
        p = round(odf ** (1 / 3))
        s = pkg.Jacobi3D(edge, edge, edge, split=(p, p, p), seed=2, init_mode=1, path=path,
                         stream=stream.cuda_stream, **tune_kw)
    else:
        s = make(path, stream=stream.cuda_stream, **tune_kw)
    try:
        s.step(warmup)
        s.sync()
        st0 = s.stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        st1 = s.stats()
    finally:
        s.close()
    return ms / steps, st0, st1


def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_2605_12734_gb300 as pkg
    from paper_2605_12734_gb300 import build as od_build

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    # one rank per node compiles (if anything is stale); the others wait for it
    if world > 1 and local != 0:
        dist.barrier()
    od_build.build()
    if world > 1 and local == 0:
        dist.barrier()
    dev = local
    if args.workload == "serve":
        return run_serve(args, pkg, torch, rank, world, dev)
    if args.workload == "launch":
        return run_launch(args, pkg, rank, dev)
    if args.workload == "shards":
        return run_shards(args, pkg, torch, rank, dev)
    edge, odf = args.edge, args.odf
    p = round(odf ** (1 / 3))
    if p ** 3 != odf and args.workload != "jacobi2d":
        raise SystemExit("--odf must be a cube")
    stream = torch.cuda.Stream(device=dev)
    tune_kw = dict(threads=args.threads, cells_per_thread=args.cpt, stages=args.stages,
                   tile_y=args.tile_y, tile_z=args.tile_z, arith=args.arith, order=args.order,
                   autotune=not args.no_tune and not (args.threads or args.cpt or args.stages or args.arith >= 0),
                   device=dev)
    from paper_2605_12734_gb300 import inputs
    if args.workload == "uneven":
        w = inputs.uneven_768()
        dims, dec, name = (w.nx, w.ny, w.nz), dict(cuts=w.cuts), w.name
    elif args.workload == "ceiling":
        w = inputs.ceiling_1024()
        dims, dec, name = (w.nx, w.ny, w.nz), dict(split=w.split), w.name
    elif args.workload == "jacobi2d":
        w = inputs.jacobi2d_32768(odf, edge=args.edge2d)
        dims, dec, name = (w.nx, w.ny, 1), dict(split=w.split[:2]), w.name
    else:
        dims, dec, name = (edge, edge, edge), dict(split=(p, p, p)), f"jacobi3d-{edge}^3-odf{odf}"
    seed = 2 if args.workload == "odf" else w.seed
    two_d = args.workload == "jacobi2d"

    def make(path, **kw):
        if two_d:
            return pkg.Jacobi2D(dims[0], dims[1], seed=seed, init_mode=1, path=path, **dec, **kw)
        return pkg.Jacobi3D(*dims, seed=seed, init_mode=1, path=path, **dec, **kw)

    # under torchrun rank 0 tunes first and writes the tuning cache; the other
    # ranks (identical GPUs) then find their shape there instead of all tuning
    # at once and appending to the same file
    if world > 1 and rank != 0:
        dist.barrier()
    solver = make(args.path, stream=stream.cuda_stream, **tune_kw)
    if world > 1 and rank == 0:
        dist.barrier()
    plan = solver.stats()["plan"]
    solver.step(args.warmup)
    solver.sync()
    st0 = solver.stats()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    st1 = solver.stats()
    ms, value = combine_ranks(ms, plan["cells"] * args.steps, world, f"cuda:{dev}")
    ms_step = ms / args.steps
    updates_step = plan["cells"]
    launches = st1["kernel_launches"] - st0["kernel_launches"]

    # roofline of the tile kernel (it does all of a step's arithmetic and all
    # of its HBM traffic): the stencil's own roof is HBM, with the
    # algorithmic bytes of a step (16 B per cell + 16 B per internal ghost
    # cell + 8 B per Dirichlet ghost cell) over the measured copy bandwidth.
    # Beside it, flat keys for the two pipes the exact FP64 arithmetic loads:
    # the FP64 pipe (adds issued there, 1 per lane-cycle, 2 lanes per SM) and
    # the issue ports (thread instructions per update from the kernel's ncu
    # capture, 4 x 32 per SM-cycle), both at the SM clock sampled under load.
    if two_d:
        fp64_adds = {0: 3, 1: 3, 2: 2, 3: 1, 4: 0, 5: 0, 6: 0, 7: 1.5, 8: 1.75, 9: 2, 10: 1, 11: 1.5,
                     12: 1, 13: 0, 14: 0.5, 15: 2}[plan["arith"]]
    else:
        fp64_adds = {0: 5, 1: 5, 2: 4, 3: 3, 4: 2, 5: 1, 6: 0, 7: 3.5, 8: 3.75, 9: 4, 10: 3,
                     11: 3.5, 12: 2, 13: 1, 14: 1.5, 15: 1.75}[plan["arith"]]
    if plan["arith"] == 0:
        fp64_adds += 8  # the IEEE division is a sequence of FP64 instructions
    ghz = (clk.get("sm_mhz") or SM_MAX_GHZ * 1e3) / 1e3
    hbm_peak, peak_kind = measured_peaks()
    bytes_step = plan["bytes_per_step"]
    ups = updates_step / (ms_step * 1e-3)
    achieved = bytes_step / (ms_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                "bytes_per_step": bytes_step,
                "note": "algorithmic bytes per step: 16 B/cell + 16 B per internal ghost cell + 8 B per Dirichlet "
                        "ghost cell; peak: measured copy bandwidth (MEASURED_PEAKS.json)"}
    prof = profiled_kernel(args, plan)
    if prof is not None and prof.get("dram_bytes_per_step"):
        # the timed region is one persistent launch of args.steps iterations
        per_launch = args.steps if args.path == "persistent" else 1
        roofline["traffic"] = prof["dram_bytes_per_step"] * per_launch
        roofline["traffic_per_step"] = prof["dram_bytes_per_step"]
        roofline["traffic_vs_algorithmic"] = prof["dram_bytes_per_step"] / bytes_step
    fp64_peak = FP64_LANES_PER_SM * SMS * ghz  # G FP64 lane-operations per second
    flat = {"hbm_frac": achieved / hbm_peak, "hbm_achieved_gbps": achieved,
            "alu_fp64_frac": fp64_adds * ups / 1e9 / fp64_peak, "fp64_ops_per_update": fp64_adds,
            "issue_frac": None, "inst_per_update": None, "sm_ghz_used": ghz}
    if prof is not None and prof.get("thread_inst_per_update"):
        flat["inst_per_update"] = prof["thread_inst_per_update"]
        flat["issue_frac"] = prof["thread_inst_per_update"] * ups / (SMS * 4 * 32 * ghz * 1e9)

    # end to end through the public API with pinned host buffers: each e2e
    # step is a whole solve of 100 iterations from the config's initial
    # field: import it (H2D), iterate, export the result (D2H).  Three
    # contexts run as a pipeline, as a serving loop would: one job's copies
    # (copy engines) run under another job's iterations, and the host waits
    # only for the job three back, so a stall of the (shared) host or host
    # link up to two jobs long leaves the device busy.  A job's iterations
    # start after the previous job's gather kernel (an event), so that short
    # kernel is not left queued behind a whole persistent launch.  Every job
    # computes u^100 of the same field, which the CPU baseline's oracle solve
    # checks below.
    e2e, e2e_flat, e2e_last = None, {}, None
    if not args.no_e2e:
        import numpy as np
        n = plan["cells"]
        depth = 3                          # contexts in the pipeline
        host_in = torch.empty(n, dtype=torch.float64, pin_memory=True)
        outs = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(depth)]
        iters_job = 100
        reps = 16                          # the pipeline's fill and drain amortised over 16 jobs
        strm = [stream] + [torch.cuda.Stream(dev) for _ in range(depth - 1)]
        twins = [make(args.path, stream=st.cuda_stream, **tune_kw) for st in strm[1:]]
        twins[0].read(host_in.numpy())     # the initial field u^0
        ctx = [solver] + twins
        # the host link's bandwidth right now (the host is shared): one copy each way
        probe = torch.empty(min(n, 1 << 27), dtype=torch.float64, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            probe.copy_(host_in[:probe.numel()], non_blocking=True)
            ev[1].record(stream)
            outs[0][:probe.numel()].copy_(probe, non_blocking=True)
            ev[2].record(stream)
        ev[2].synchronize()
        link = (probe.numel() * 8 / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e9,
                probe.numel() * 8 / (ev[1].elapsed_time(ev[2]) * 1e-3) / 1e9)
        del probe
        first = None
        for c, o in zip(ctx, outs):        # warm-up job on each context
            c.write_async(host_in)
            c.step(iters_job)
            c.read_async(o)
            c.sync()
            if first is None:
                first = o.numpy().copy()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ctx[0].write_async(host_in)
        ctx[0].step(iters_job)
        spans = []                         # each job's iterations, as the device ran them
        for j in range(1, reps):
            cur, prev = ctx[j % depth], ctx[(j - 1) % depth]
            if j >= depth:
                cur.sync()                 # this context's job j - depth: exported
            cur.write_async(host_in)
            prev.read_async(outs[(j - 1) % depth])
            gathered = torch.cuda.Event()
            gathered.record(strm[(j - 1) % depth])
            strm[j % depth].wait_event(gathered)
            k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k0.record(strm[j % depth])
            cur.step(iters_job)
            k1.record(strm[j % depth])
            spans.append((k0, k1))
        last = (reps - 1) % depth
        ctx[last].read_async(outs[last])
        for c in ctx:
            c.sync()
        dt = time.perf_counter() - t0
        e2e_last = outs[last].numpy().copy()
        same = bool(np.array_equal(e2e_last.view(np.uint64), first.view(np.uint64)))
        for t in twins:
            t.close()
        it_ms = sum(a.elapsed_time(b) for a, b in spans) / len(spans)
        # the device's job intervals: from one job's end of iterations to the next one's
        gaps = np.array([spans[q][1].elapsed_time(spans[q + 1][1]) for q in range(len(spans) - 1)])
        e2e = {"value": n * iters_job * reps * world / dt, "unit": UNIT,
               "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8,
               "iters_per_step": iters_job, "jobs": reps, "results_identical": same, "pipeline_contexts": depth,
               "job_intervals_ms": [round(float(g), 2) for g in gaps],
               "iterations_ms": [round(a.elapsed_time(b), 2) for a, b in spans],
               "note": "e2e step = od_write_async(pinned host u^0) + od_step(100) + od_read_async(pinned host); "
                       "three contexts pipelined, so one job's host copies overlap another's iterations"}
        e2e_flat = {"e2e_host_link_h2d_gbps": round(link[0], 1), "e2e_host_link_d2h_gbps": round(link[1], 1),
                    "e2e_iterations_ms_per_job": round(it_ms, 3), "e2e_wall_ms_per_job": round(dt / reps * 1e3, 3),
                    "e2e_job_interval_median_ms": round(float(np.median(gaps)), 3),
                    "e2e_job_interval_max_ms": round(float(np.max(gaps)), 3),
                    "e2e_first_interval_ms": round(float(gaps[0]), 3),
                    "e2e_jobs_identical": same}
    solver.close()

    baseline = None
    if args.baseline_steps > 0 and rank == 0 and args.workload in ("odf", "jacobi2d"):
        ms_b, b0, b1 = time_path(pkg, edge, odf, "per_chare", args.baseline_steps, 1, stream,
                                 dict(device=dev), make=make if two_d else None)
        baseline = {"path": "per_chare", "ms_per_step": ms_b, "value": updates_step / (ms_b * 1e-3),
                    "steps": args.baseline_steps,
                    "api_calls_per_step": (b1["api_calls"] - b0["api_calls"]) / args.baseline_steps,
                    "kernels_per_step": (b1["kernel_launches"] - b0["kernel_launches"]) / args.baseline_steps}
        # the paper's runtime remedy: several host threads (PEs) submit the chares' work
        for pe in (2, 4, 8):
            ms_pe, _, _ = time_path(pkg, edge, odf, "per_chare", args.baseline_steps, 1, stream,
                                    dict(device=dev, pe_threads=pe), make=make if two_d else None)
            baseline[f"ms_per_step_pe{pe}"] = ms_pe

    sweep = None
    if args.workload == "odf" and world == 1 and not args.no_sweep:
        args.sweep = True  # the metric is throughput vs ODF: sweep every path at every ODF
    if args.sweep and rank == 0 and two_d:
        sweep = []
        for o in (1, 4, 16, 64, 256, 1024, 4096):
            w2 = inputs.jacobi2d_32768(o, edge=args.edge2d)
            for path in ("fused", "persistent", "fused_graph", "graph", "per_chare"):
                k = args.steps if path in ("fused", "persistent", "fused_graph") else max(2, min(10, args.steps))
                if path in ("graph", "per_chare") and o >= 1024:
                    k = 2

                def make_o(pth, **kw):
                    return pkg.Jacobi2D(w2.nx, w2.ny, seed=seed, init_mode=1, path=pth, split=w2.split[:2], **kw)
                ms_p, _, _ = time_path(pkg, edge, o, path, k, 2, stream, dict(device=dev), make=make_o)
                info = pkg.plan_2d(w2.nx, w2.ny, split=w2.split[:2])
                sweep.append({"odf": o, "path": path, "ms_per_step": ms_p, "steps": k,
                              "updates_per_s": info["cells"] / (ms_p * 1e-3),
                              "alg_GBps": info["bytes_per_step"] / (ms_p * 1e-3) / 1e9})
    elif args.sweep and rank == 0:
        sweep = []
        for o in (1, 8, 64, 512, 4096):
            for path in ("fused", "persistent", "fused_graph", "graph", "per_chare"):
                k = args.steps if path in ("fused", "persistent", "fused_graph") else max(2, min(10, args.steps))
                if path in ("graph", "per_chare") and o >= 4096:
                    k = 2
                ms_p, _, _ = time_path(pkg, edge, o, path, k, 2, stream, dict(device=dev))
                info = pkg.plan(edge, edge, edge, split=(round(o ** (1 / 3)),) * 3)
                sweep.append({"odf": o, "path": path, "ms_per_step": ms_p, "steps": k,
                              "updates_per_s": info["cells"] / (ms_p * 1e-3),
                              "eff_GBps": 16 * info["cells"] / (ms_p * 1e-3) / 1e9,
                              "alg_GBps": info["bytes_per_step"] / (ms_p * 1e-3) / 1e9})

    # the metric's other workloads, one short run each beside the headline:
    # the uneven 300-chare grid and the 1024^3 ceiling (same path, tuned),
    # and a serving stream at a rate near saturation
    legs = {}
    if args.workload == "odf" and rank == 0 and world == 1 and not args.no_legs:
        for key, w in (("uneven", inputs.uneven_768()), ("ceiling", inputs.ceiling_1024())):
            def make_w(path, w=w, **kw):
                dec_w = {"cuts": w.cuts} if w.cuts else {"split": w.split}
                return pkg.Jacobi3D(w.nx, w.ny, w.nz, seed=w.seed, init_mode=1, path=path, **dec_w, **kw)
            ms_w, _, st_w = time_path(pkg, 0, 0, args.path, args.steps, args.warmup, stream,
                                      dict(device=dev, autotune=not args.no_tune), make=make_w)
            info = st_w["plan"]
            legs[f"{key}_updates_per_s"] = info["cells"] / (ms_w * 1e-3)
            legs[f"{key}_ms_per_step"] = ms_w
            legs[f"{key}_hbm_frac"] = info["bytes_per_step"] / (ms_w * 1e-3) / 1e9 / hbm_peak
            legs[f"{key}_arith"] = info["arith"]
        r = serve_stream(pkg, dev, 150, 120.0, args.budget_gb, job_streams=serve_job_streams(args))
        alone = jobs_alone_rate(pkg, dev, 150, 120.0)
        legs.update({"serve_job_streams": serve_job_streams(args),
                     "serve_jobs_alone_updates_per_s": alone,
                     # the server's rate while the device is busy, against the same jobs run alone
                     "serve_busy_vs_jobs_alone": r["updates_per_s"] / max(r["device_busy_frac"], 1e-9) / alone,
                     "serve_p50_ms": r["p50_s"] * 1e3, "serve_p99_ms": r["p99_s"] * 1e3,
                     "serve_updates_per_s": r["updates_per_s"], "serve_rate_per_s": r["rate_per_s"],
                     "serve_jobs": r["jobs"], "serve_device_busy_frac": r["device_busy_frac"],
                     "serve_offered_updates_per_s": r["offered_updates_per_s"]})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if two_d:
            cpu = oracle_cpu_baseline_2d(dims[0])
        else:
            cpu = oracle_cpu_baseline(edge if args.workload == "odf" else 512,
                                      e2e_out=e2e_last if args.workload == "odf" else None)
            if "e2e_cells_differing_from_oracle" in cpu:
                e2e_flat["e2e_matches_oracle"] = cpu["e2e_cells_differing_from_oracle"] == 0

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(name, dims, plan["nchares"], "2d5" if two_d else "3d7", seed, world),
                "launch": {"path": args.path, "tuned": bool(st1.get("tuned")),
                           "chare_edge": (edge // p) if args.workload == "odf" else None,
                           **{k: plan[k] for k in ("threads", "cells_per_thread", "stages", "arith", "tile_y",
                                                   "tile_z", "smem_bytes", "ntiles")}},
                "roofline": roofline, **flat, "cpu_baseline": cpu, "e2e": e2e, **e2e_flat,
                "e2e_frac_of_device": (e2e["value"] / value) if e2e else None, **legs,
                "gpu_launches": launches, "clocks": clk, "eff_GBps": 16 * updates_step / (ms_step * 1e-3) / 1e9,
                "per_chare_baseline": baseline}
        if sweep is not None:
            line["sweep"] = sweep
            by = {(r["odf"], r["path"]): r["ms_per_step"] for r in sweep}
            odfs = sorted({r["odf"] for r in sweep})
            for pth in ("persistent", "fused", "fused_graph", "graph", "per_chare"):
                if (odfs[0], pth) in by and (odfs[-1], pth) in by:
                    line[f"sweep_{pth}_maxodf_vs_odf1"] = by[(odfs[-1], pth)] / by[(odfs[0], pth)]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_launch(args, pkg, rank, dev):
    """The paper's launch-overhead measurements (Sec. III) on this GPU: the
    round trip of one empty kernel, a fixed amount of work split over 1..1024
    pre-enqueued kernels released together, and the kernel rate of 1-4 host
    threads driving 1-8 chares each."""
    if rank != 0:
        return 0
    clocks = ClockSampler(dev)
    clocks.start()
    lat = {w: pkg.bench_launch_latency(w, reps=5000, device=dev) for w in ("sync", "event", "callback")}
    work = 4096
    release = []
    for total in (256 * 1024, 4 * 1024 * 1024):
        for nk in (1, 2, 4, 8, 16, 32, 64, 256, 1024):
            t = sorted(pkg.bench_release(total, nk, work, device=dev) for _ in range(5))
            release.append({"total_threads": total, "kernels": nk, "us_median": t[2], "us_min": t[0]})
    rate = []
    for ht in (1, 2, 4):
        for ch in (1, 2, 4, 8):
            rate.append({"host_threads": ht, "chares_per_thread": ch,
                         "kernels_per_s": pkg.bench_launch_rate(ht, ch, kernels=max(200, 4000 // (ht * ch)),
                                                                 device=dev)})
    clk = clocks.stop()
    line = {"metric": "kernel launch round trip (empty kernel, cudaStreamSynchronize)", "value": lat["sync"],
            "unit": "us", "n_gpus": 1, "higher_is_better": False, "dtype": "none", "data": "synthetic",
            "config": {"workload": "launch-overhead-microbenchmarks", "release_work_lcg_steps": work,
                       "rate_kernel": "empty, one block of 32 threads per SM"},
            "latency_us": lat, "release": release, "launch_rate": rate, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


SHARD_SHAPE = dict(threads=128, cells_per_thread=4, stages=4, arith=7, tile_z=32)


def _shard_worker(rank, world, port, edge, steps, warmup, path, out):
    """One process of the two-process shard measurement (spawned)."""
    import torch
    import torch.distributed as dist
    import paper_2605_12734_gb300 as pkg
    from paper_2605_12734_gb300.shard import IpcTransport, ProcessShard, ShardPlan, _make_solver
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plan = ShardPlan((edge, edge, edge), (1, 1, world))
    stream = torch.cuda.Stream(device=0)
    p = 16
    solver = _make_solver(pkg, plan, rank, (p, p, p // world), stream.cuda_stream, seed=2, init_mode=1, path=path,
                          device=0, **SHARD_SHAPE)
    tr = IpcTransport(plan, rank, 0, stream.cuda_stream)
    sh = ProcessShard(plan, rank, solver, tr)
    sh.step(warmup)
    stream.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    sh.step(steps)
    stream.synchronize()
    dt = time.perf_counter() - t0
    dist.barrier()
    sh.drain()
    out[rank] = dt
    dist.barrier()
    solver.close()
    tr.close()
    dist.destroy_process_group()


def run_shards(args, pkg, torch, rank, dev):
    """The paper's process-width trade-off (Sec. III "Performance
    trade-offs") on one GPU: the 512^3 grid at ODF 4096 held by one context,
    or split along z into 2, 4, 8 shards (contexts on their own streams) whose
    boundary faces move every iteration through communication endpoints (two
    device copies and an event per face, the inter-process transport), or
    held by two processes sharing the GPU through CUDA IPC endpoints."""
    if rank != 0:
        return 0
    import socket
    import torch.multiprocessing as mp
    from paper_2605_12734_gb300.shard import ShardedJacobi
    edge, steps, warmup = args.edge, args.steps, args.warmup
    rows = []
    clocks = ClockSampler(dev)
    clocks.start()
    for S in (1, 2, 4, 8):
        sj = ShardedJacobi((edge, edge, edge), (1, 1, S), (16, 16, 16 // S), seed=2, init_mode=1, path=args.path,
                           device=dev, **SHARD_SHAPE)
        sj.step(warmup)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sj.step(steps)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        sj.close()
        rows.append({"shards": S, "processes": 1, "ms_per_step": dt * 1e3 / steps,
                     "updates_per_s": edge ** 3 * steps / dt})
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        mp.spawn(_shard_worker, args=(2, port, edge, steps, warmup, args.path, out), nprocs=2, join=True)
        dt = max(dict(out).values())
    rows.append({"shards": 2, "processes": 2, "ms_per_step": dt * 1e3 / steps,
                 "updates_per_s": edge ** 3 * steps / dt})
    clk = clocks.stop()
    base = rows[0]["ms_per_step"]
    for r in rows:
        r["vs_one_context"] = r["ms_per_step"] / base
    line = {"metric": "grid-pt updates/s of 512^3 at ODF 4096 split over shards exchanging faces",
            "value": rows[1]["updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"jacobi3d-{edge}^3-odf4096-shards", "path": args.path, "shape": SHARD_SHAPE,
                       "timing": "host wall clock around the steps, device synchronised on both sides"},
            "shards": rows, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def jobs_alone_rate(pkg, dev, n_jobs, rate):
    """The serving stream's jobs run one at a time, each alone on the GPU in
    its own context (persistent path, the planner's shape): total updates
    over the sum of the jobs' device times (CUDA events around each job's
    steps).  The rate the server would reach if it only queued the jobs --
    the yardstick for what running them side by side gains."""
    import torch
    from paper_2605_12734_gb300 import inputs
    stream = torch.cuda.Stream(device=dev)
    upd, ms = 0.0, 0.0
    for j in inputs.serving_stream(n_jobs, rate, seed=6):
        with pkg.Jacobi3D(j.edge, j.edge, j.edge, split=(j.p, j.p, j.p), seed=j.seed, init_mode=1,
                          path="persistent", device=dev, stream=stream.cuda_stream) as s:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(j.iters)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            upd += j.updates
    return upd / (ms * 1e-3)


def serve_stream(pkg, dev, n_jobs, rate, budget_gb, threads=0, cpt=0, stages=0, arith=-1, batch_steps=0,
                 job_streams=0):
    """Poisson arrivals of independent jobs into one server: each a cubic
    grid with edge log-uniform in [64, 384], ODF in {8, 27, 64, 216} and
    10..200 iterations (seeded); returns aggregate updates/s and the job
    latencies (completion - arrival)."""
    from paper_2605_12734_gb300 import inputs
    jobs = inputs.serving_stream(n_jobs, rate, seed=6)
    budget = int(budget_gb * (1 << 30))
    srv = pkg.Server(budget, device=dev, threads=threads, cells_per_thread=cpt, stages=stages, arith=arith,
                     batch_steps=batch_steps, job_streams=job_streams)
    # warm-up: one small job through the whole path
    w = srv.submit(64, 64, 64, 3, split=(2, 2, 2), seed=1)
    srv.wait(w, 60.0)
    srv.release(w)
    while srv.next_completion(0.0) is not None:  # the warm-up job's completion
        pass
    # the client releases every job as soon as it ends (the server's
    # completion queue, drained by a second thread), as a serving client
    # would, so finished jobs do not hold the HBM budget against new arrivals
    ids, lock = {}, threading.Lock()
    lat, upd, span, failed = [], [0.0], [None, 0.0], []

    def reap():
        left = n_jobs
        while left:
            jid = srv.next_completion(0.05)
            if jid is None:
                continue
            with lock:
                j = ids.pop(jid, None)
            if j is None:  # not one of this stream's jobs: stop, the check below reports it
                failed.append((jid, "unknown"))
                return
            info = srv.info(jid)
            if info["state"] != 2:
                failed.append((jid, info["state"]))
            lat.append(info["t_done"] - info["t_submit"])
            span[0] = info["t_submit"] if span[0] is None else min(span[0], info["t_submit"])
            span[1] = max(span[1], info["t_done"])
            upd[0] += j.updates
            srv.release(jid)
            left -= 1

    reaper = threading.Thread(target=reap, daemon=True)
    t0 = time.perf_counter()
    busy0 = srv.stats()["busy_seconds"]
    reaper.start()
    for j in jobs:
        delay = t0 + j.arrival_s - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        with lock:
            jid = srv.submit(j.edge, j.edge, j.edge, j.iters, split=(j.p, j.p, j.p), seed=j.seed)
            ids[jid] = j
    reaper.join(timeout=1200.0)
    if reaper.is_alive() or failed:
        raise SystemExit(f"serving stream did not complete: {len(ids)} jobs unreaped, failed {failed[:5]}")
    first_submit, last_done, upd = span[0], span[1], upd[0]
    st = srv.stats()
    srv.close()
    wall = last_done - first_submit
    lat_sorted = sorted(lat)

    def pct(q):
        return lat_sorted[min(len(lat_sorted) - 1, int(round(q * (len(lat_sorted) - 1))))]
    return {"updates_per_s": upd / wall, "p50_s": pct(0.50), "p99_s": pct(0.99), "mean_s": sum(lat) / len(lat),
            "max_s": lat_sorted[-1], "wall_s": wall, "launches": st["launches"],
            "pool_peak_gb": st["pool_peak"] / (1 << 30), "offered_updates_per_s": upd / jobs[-1].arrival_s,
            "admit_seconds": st["admit_seconds"], "device_busy_frac": (st["busy_seconds"] - busy0) / wall,
            "jobs": n_jobs, "rate_per_s": rate}


SERVE_JOB_STREAMS = 16  # the serving leg's default: one persistent launch per job on 16 streams


def serve_job_streams(args):
    return SERVE_JOB_STREAMS if args.job_streams < 0 else args.job_streams


def run_serve(args, pkg, torch, rank, world, dev):
    """Serving stream: independent jobs arrive as a Poisson process (seeded),
    each a cubic grid with edge log-uniform in [64, 384], ODF in {8, 27, 64,
    216} and 10..200 iterations; the server admits them under the HBM budget
    and batches every running job into one launch per iteration.  Reports
    aggregate updates/s and p50/p99 job latency (completion - arrival)."""
    clocks = ClockSampler(dev)
    clocks.start()
    r = serve_stream(pkg, dev, args.jobs, args.rate, args.budget_gb, args.threads, args.cpt, args.stages, args.arith,
                     args.batch_steps, serve_job_streams(args))
    clk = clocks.stop()
    alone = jobs_alone_rate(pkg, dev, args.jobs, args.rate)
    line = {"metric": METRIC, "value": r["updates_per_s"], "unit": UNIT, "n_gpus": world, "steps": args.jobs,
            "warmup": 1, "ms_per_step": r["wall_s"] * 1e3 / args.jobs, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "jacobi3d-serving-poisson", "jobs": args.jobs, "rate_per_s": args.rate,
                       "edge": "log-uniform [64,384]", "odf": "{8,27,64,216}", "iters": "U[10,200]",
                       "budget_gb": args.budget_gb, "seed": 6, "batch_steps": args.batch_steps,
                       "job_streams": serve_job_streams(args),
                       "note": "a step here is one job"},
            "latency_p50_s": r["p50_s"], "latency_p99_s": r["p99_s"], "latency_mean_s": r["mean_s"],
            "latency_max_s": r["max_s"], "wall_s": r["wall_s"], "launches": r["launches"],
            "pool_peak_gb": r["pool_peak_gb"], "offered_updates_per_s": r["offered_updates_per_s"],
            "admit_seconds": r["admit_seconds"], "device_busy_frac": r["device_busy_frac"],
            "jobs_alone_updates_per_s": alone, "vs_jobs_alone": r["updates_per_s"] / alone,
            "busy_vs_jobs_alone": r["updates_per_s"] / max(r["device_busy_frac"], 1e-9) / alone, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
