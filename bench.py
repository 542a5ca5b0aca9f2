#!/usr/bin/env python3
"""Benchmark of the GB300 feasible-triplet sweep (Heineman et al., arXiv 2407.10925).

Workload (default): sigma = d = 2, h = 16 -- 2^32 states, the zero start of
Algorithm 2, three resident fixed-point iterate vectors (complement-symmetric
storage: 3 x 16 GiB).  One *step* is one check period of Algorithm 2 as the
library runs it: C sweeps v_t = F(v_{t-1}, v_{t-2}) (the last one with the
fused min/argmin of the increment), then the feasibility check of that
iterate and the device-side keep test.  value = state-updates/s = (states x
sweeps) / time over all ranks.

Arms:
  --impl ours (default)  the CUDA library through its C ABI
  --impl reference       the CPU oracle as it stands, on a bounded sample of
                         the same workload (no GPU work)

Multi-GPU: the path has no exchange step across GPUs, so N ranks run N
independent replicas (weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BATCH_SHAPES = [(2, 2, 10), (2, 2, 12), (3, 2, 6), (3, 2, 7), (4, 2, 5), (2, 3, 6), (2, 3, 7), (2, 4, 5)]
CONFIGS = {
    "batch": dict(sigma=0, d=0, h=0, shapes=BATCH_SHAPES),
    "warm": dict(sigma=2, d=2, h=14, train_h=[10, 11, 12], ref_iters=4000, train_steps=3000),
    "warm16": dict(sigma=2, d=2, h=16, train_h=[10, 11, 12], ref_iters=1000, train_steps=3000),
    "fp32": dict(sigma=0, d=0, h=0, shapes=[(2, 3, 8), (3, 2, 8)], iters=1500),
    "h17": dict(sigma=2, d=2, h=17, bound_iters=400),  # 2^34 states: 3 x 64 GiB resident (Table 2's l = 17); use --no-e2e
    "h16": dict(sigma=2, d=2, h=16, bound_iters=2000),
    "d3h11": dict(sigma=2, d=3, h=11, bound_iters=400),  # 2^33 states, 4 x 32 GiB: beyond Table 3's l = 10 for d = 3
    "d3h9": dict(sigma=2, d=3, h=9),  # 2^27 states (2 GiB resident): profiling size of the d = 3 kernels
    "h14": dict(sigma=2, d=2, h=14),
    "h12": dict(sigma=2, d=2, h=12),
    "h8": dict(sigma=2, d=2, h=8),
    # out of core: 32-bit offset-normalised rows, one of the three in pinned host memory
    "h18": dict(sigma=2, d=2, h=18, frac_bits=26, outofcore=True, check=25, max_iters=800, target=0.790668),
    "h16x": dict(sigma=2, d=2, h=16, frac_bits=26, outofcore=True, check=25, max_iters=400, target=0.789021),
    # the same 32-bit rows, all three in device memory (h = 17: 3 x 32 GiB)
    "h17n": dict(sigma=2, d=2, h=17, frac_bits=26, storage=1, bound_iters=400),
    # shapes of the general kernels (every shape without a specialised kernel)
    # (sums of sigma^d values need fewer fractional bits than the default 44)
    "s3d8h2": dict(sigma=3, d=8, h=2, frac_bits=36, general=True),  # 3^16 states
    "s10d2h4": dict(sigma=10, d=2, h=4, general=True),  # 10^8 states
    "s2d12h2": dict(sigma=2, d=12, h=2, frac_bits=36, general=True),  # 2^24 states, one warp per state
}
METRIC = "state-updates/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="h16")
    ap.add_argument("--check-every", type=int, default=10, help="sweeps per step (one check per step)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--bound-iters", type=int, default=None,
                    help="iterations of the wall-time-to-bound run (default: the config's, 2000 for h16; 0 skips)")
    ap.add_argument("--symmetry", type=int, default=1)
    ap.add_argument("--batch-mode", choices=["auto", "0", "1", "2"], default="auto",
                    help="batch config: the autotuner's mode, or force 0 (persistent launch), 1 (concurrent, "
                         "graph-captured), 2 (concurrent, enqueued call by call)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU side: the oracle on a bounded sample (spawned workers, before any CUDA use)
#
# The oracle's plain F (orc_F_fx) over a window of W = sigma^(d m) consecutive
# states, aligned to W, with its arguments resident in host memory.  Such a
# window varies only the last m letters of every string, so the states F reads
# for one set of advanced strings lie in one aligned block of sigma^d W states
# (the block of the window's first state advanced with the letters 0).  Each
# argument is a full-length vector whose pages exist only where written (an
# anonymous mapping without reservation); the blocks the window reads hold
# seeded values like converged iterates (200 units, spread over 4).


def _sparse_vector(n):
    """(numpy int64 view of n values, munmap callback): pages are allocated only where written"""
    import ctypes

    import numpy as np

    libc = ctypes.CDLL(None, use_errno=True)
    libc.mmap.restype = ctypes.c_void_p
    libc.mmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long]
    libc.munmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    prot_rw, map_private, map_anonymous, map_noreserve = 0x3, 0x02, 0x20, 0x4000
    p = libc.mmap(None, n * 8, prot_rw, map_private | map_anonymous | map_noreserve, -1, 0)
    if p is None or p == ctypes.c_void_p(-1).value:
        raise OSError(ctypes.get_errno(), "mmap of the oracle's sparse argument vector failed")
    arr = np.ctypeslib.as_array((ctypes.c_int64 * n).from_address(p))
    return arr, (lambda: libc.munmap(p, n * 8))


def window_arguments(sigma, d, h, x0, m, seed, vs):
    """Fill, in the d argument vectors vs, the blocks that F reads for the window of sigma^(d m) states at x0."""
    import itertools

    import numpy as np

    import oracle

    B = sigma ** (d * (m + 1))
    one = 1 << oracle.DEFAULT_FRAC_BITS
    rng = np.random.default_rng(seed)
    X = oracle.decode(sigma, d, h, x0)
    for adv in itertools.chain.from_iterable(itertools.combinations(range(d), k) for k in range(1, d + 1)):
        Y = X.copy()
        for j in adv:  # string j loses its head and gains the letter 0
            Y[:-1, j] = X[1:, j]
            Y[-1, j] = 0
        base = oracle.encode(sigma, d, h, Y) // B * B
        vs[len(adv) - 1][base:base + B] = (200 - len(adv)) * one + rng.integers(0, 4 * one, size=B)


_BARRIER = None


def _init_worker(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_window(args):
    """(start, end) wall-clock seconds of the oracle's F plus the increment minimum over one window.

    The arguments are filled first; with `together`, every worker of the step
    then meets at a barrier, so the timed parts of a step run side by side."""
    sigma, d, h, x0, m, seed, together = args
    import oracle

    n = sigma ** (d * h)
    W = sigma ** (d * m)
    vs, frees = zip(*[_sparse_vector(n) for _ in range(d)])
    window_arguments(sigma, d, h, x0, m, seed, vs)
    if together:
        _BARRIER.wait(timeout=600)
    t0 = time.time()
    out = oracle.F(sigma, d, h, list(vs), arith="fx", x0=x0, x1=x0 + W)
    int((out - vs[0][x0:x0 + W]).min())
    t1 = time.time()
    del out
    for f in frees:
        f()
    return t0, t1


def oracle_sample(cfg, workers=None, steps=1, m=None):
    """Time the oracle's plain F on windows of consecutive states of the workload.

    Returns (per-step dicts of states and seconds on all workers, the 1-core rate, cores, sample text).
    """
    import oracle

    oracle.build()
    sigma, d, h = cfg["sigma"], cfg["d"], cfg["h"]
    n = sigma ** (d * h)
    workers = workers or os.cpu_count() or 1
    if m is None:  # about a second of F per window (4^11 states for sigma = d = 2)
        m = max(1, min(h - 1, round(22 / (d * math.log2(sigma)))))
    W = sigma ** (d * m)
    n_windows = n // W
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    with ctx.Pool(workers, initializer=_init_worker, initargs=(barrier,)) as pool:
        pool.map(_oracle_window, [(sigma, d, h, 0, 1, 0, True)] * workers, chunksize=1)  # import + build
        a, b = pool.apply(_oracle_window, ((sigma, d, h, (n_windows // 3) * W, m, 1, False),))  # one core alone
        t1 = b - a
        steps_out = []
        for s in range(steps):
            args = [(sigma, d, h, ((s * workers + i) * 7919 % n_windows) * W, m, 100 + s * workers + i, True)
                    for i in range(workers)]
            spans = pool.map(_oracle_window, args, chunksize=1)
            steps_out.append({"states": workers * W,
                              "seconds": max(e for _, e in spans) - min(st for st, _ in spans)})
    sample = (f"the oracle's plain F (orc_F_fx, fixed point) and the increment minimum over {workers} windows of "
              f"{W} consecutive states of sigma={sigma} d={d} h={h} per step, one window per spawned process, "
              f"arguments resident in host memory (seeded values in the blocks each window reads), the "
              f"processes starting together after filling them; 1-core figure: one window alone")
    return steps_out, W / t1, workers, sample


# ---------------------------------------------------------------------------
# GPU helpers


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to LCS_CLOCKS_DIR (default: the temporary directory)
        out_dir = os.environ.get("LCS_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"lcs_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(files):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2407_10925_gb300", "csrc")
    for name in files:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(config_name, kernel):
    """dram bytes per launch from the committed ncu summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            j = json.load(f)
        entry = j.get(kernel, {}).get(config_name)
        if not entry or entry.get("source_hash") != kernel_source_hash(entry["source_files"]):
            return None
        return entry.get("dram_bytes_per_launch")
    except (OSError, ValueError, KeyError):
        return None


# ---------------------------------------------------------------------------
# ranks: replicas only; the slowest rank's time is the job's time


def reduce_max(x: float, dist=None, device=None) -> float:
    """max of x over all ranks (x itself without a process group)."""
    if dist is None or not dist.is_initialized():
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, cfg, rank):
    if rank != 0:
        return
    steps, rate_1core, cores, sample = oracle_sample(cfg, steps=args.warmup + args.steps)
    timed = steps[args.warmup:]
    states = sum(st["states"] for st in timed)
    seconds = sum(st["seconds"] for st in timed)
    value = states / seconds
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "state-updates/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * seconds / len(timed),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": workload_name(cfg, args), "states": cfg["sigma"] ** (cfg["d"] * cfg["h"]),
                   "states_per_step": timed[0]["states"],
                   "step": "one bounded sample: F and the increment minimum over one window of consecutive "
                           "states on each host core (the GPU arm's step sweeps every state 10 times)"},
        "cpu_baseline": {"value": value, "unit": "state-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample, "value_1core": rate_1core, "value_all_cores": value},
        "e2e": {"value": value, "unit": "state-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def general_terms_per_state(sigma, d):
    """Mean terms of F per state (every candidate's sum over sigma^|N| values),
    counting each sum once per tail tuple: the block form forms each once."""
    import math

    # a sum M(z, S) for every letter z and every proper S whose complement is
    # not empty, sigma^|N| terms each, shared by the sigma^d head combinations
    tot = sum(math.comb(d, k) * sigma ** k for k in range(1, d)) * sigma + sigma ** d
    return tot / sigma ** d


def workload_name(cfg, args):
    return (f"feasible-triplet sweep sigma={cfg['sigma']} d={cfg['d']} h={cfg['h']} "
            f"({cfg['sigma'] ** (cfg['d'] * cfg['h'])} states), zero start, fixed-point int64 iterates, "
            f"{args.check_every} sweeps + 1 check per step")


def run_batch(args, cfg, world, rank, local_rank):
    """Config 3: the eight instances in one persistent launch vs one after another."""
    import torch

    import paper_2407_10925_gb300 as lb

    torch.cuda.set_device(local_rank)
    shapes = cfg["shapes"]
    n_states = [s ** (d * h) for s, d, h in shapes]
    C = args.check_every
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    total_iters = 1000

    # wall time to the rigorous bounds, batched: create (with autotuning) .. read
    torch.cuda.synchronize()
    t0_batch = time.perf_counter()
    b = lb.LcsBatch(shapes, check_every=C, stream=stream.cuda_stream)
    if args.batch_mode != "auto":
        b.set_mode(int(args.batch_mode))
    t_created = time.perf_counter()
    b.iterate(total_iters)
    bounds_batch = [b.read(i)[0] for i in range(len(shapes))]
    t_batch = time.perf_counter() - t0_batch
    info = b.info()

    # the timed steady state: steps of C iterations after warm-up
    for _ in range(args.warmup):
        b.iterate(C)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            b.iterate(C)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = reduce_max(ev0.elapsed_time(ev1), None)
    b.close()

    # the concurrent mode with its calls captured in CUDA graphs (1) against
    # the same mode enqueued call by call (2), in the same steady state.  A
    # schedule (call length, check phase, every ring's newest slot) is
    # captured the second time it comes; with 10-iteration calls the rings of
    # 3, 4 and 5 slots repeat after 6 calls, so 24 warm-up calls capture all.
    conc = {}
    for mode in (1, 2):
        bm = lb.LcsBatch(shapes, check_every=C, stream=stream.cuda_stream)
        bm.set_mode(mode)
        for _ in range(max(args.warmup, 24)):
            bm.iterate(C)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            bm.iterate(C)
        e1.record(stream)
        torch.cuda.synchronize()
        mi = bm.info()
        conc[f"mode{mode}"] = {"ms_per_step": reduce_max(e0.elapsed_time(e1), None) / args.steps,
                               "graph_captured": mi["graph_captured"], "graph_replays": mi["graph_replays"],
                               "bounds": [bm.read(i)[0] for i in range(len(shapes))]}
        bm.close()
    conc["captured_speedup"] = conc["mode2"]["ms_per_step"] / conc["mode1"]["ms_per_step"]
    conc["bounds_equal"] = conc["mode1"].pop("bounds") == conc["mode2"].pop("bounds")

    # the plain path: each instance alone through the single-instance API
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bounds_plain = []
    for s_, d_, h_ in shapes:
        with lb.LcsBound(s_, d_, h_, check_every=C, stream=stream.cuda_stream) as one:
            one.iterate(total_iters)
            bounds_plain.append(one.read()[0])
    t_plain = time.perf_counter() - t0
    value = world * sum(n_states) * C * args.steps / (ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "state-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "8 instances (sigma,d,h) " + str(shapes) + " in one batch handle ("
                   + ("concurrent single-instance kernels" if info["mode"] >= 1 else "one persistent launch")
                   + f", the autotuner's choice unless forced), {C} iterations per step",
                   "states": sum(n_states), "sweeps_per_step": C,
                   "l2": "working set of the batch (about 0.6 GB) is larger than L2"},
        "batch": {"time_to_bounds_s": t_batch, "create_and_tune_s": t_created - t0_batch,
                  "plain_sequential_time_to_bounds_s": t_plain, "speedup_vs_plain": t_plain / t_batch,
                  "iterations": total_iters, "bounds_equal_plain": bounds_batch == bounds_plain,
                  "bounds": dict(zip([str(s) for s in shapes], bounds_batch)), "tuning": info,
                  "concurrent_modes": conc},
        "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_warm(args, cfg, world, rank, local_rank):
    """Config 5: iterations and wall time to a bound within 1e-7 of the zero-start
    converged bound at h = 14, from the zero start, a prefix-truncation start and
    the learned (MLP) start trained on converged iterates of h = 10, 11, 12."""
    import torch

    import paper_2407_10925_gb300 as lb

    torch.cuda.set_device(local_rank)
    H, train_h, chunk, tol = cfg["h"], cfg["train_h"], 10, 1e-7

    def sync():
        torch.cuda.synchronize()

    def converged_vector(h, iters=1500):
        with lb.LcsBound(2, 2, h, check_every=100) as hnd:
            hnd.iterate(iters)
            v = torch.empty(4 ** h, dtype=torch.int64, device="cuda")
            lb.lcs_bound_export_fx(hnd.hnd, 0, v)
            return v, hnd.read()

    def run_to(target, start=None, limit=6000, stored=False):
        """iterations (a multiple of `chunk`) and seconds until the bound reaches target"""
        sync()
        t0 = time.perf_counter()
        with lb.LcsBound(2, 2, H, check_every=chunk) as hnd:
            if start is not None and stored:
                hnd.set_start_stored_fx(start)
            elif start is not None:
                hnd.set_start(start)
            it, bound = 0, 0.0
            while it < limit:
                hnd.iterate(chunk)
                it += chunk
                bound = hnd.read()[0]
                if target is not None and bound >= target:
                    break
        return it, time.perf_counter() - t0, bound

    # the zero-start reference: run long, the converged bound is the target
    it_ref, t_ref, bound_ref = run_to(None, limit=cfg["ref_iters"])
    target = bound_ref - tol
    it_zero, t_zero, b_zero = run_to(target)

    # training data: converged iterates of smaller h
    sync()
    t0 = time.perf_counter()
    data = {h: converged_vector(h) for h in train_h}
    t_data = time.perf_counter() - t0
    r_hat = data[max(train_h)][1][2]

    sync()
    t0 = time.perf_counter()
    mlp = lb.LcsMlp(seed=2024)
    loss0 = mlp.train([data[h][0] for h in train_h], train_h, steps=0, batch=4096)
    loss = mlp.train([data[h][0] for h in train_h], train_h, steps=cfg["train_steps"], batch=4096, lr=1e-3)
    t_train = time.perf_counter() - t0

    # the learned start goes straight into the handle's stored form (fixed point)
    newest_fx = torch.empty(4 ** H // 2, dtype=torch.int64, device="cuda")
    older_fx = torch.empty(4 ** H // 2, dtype=torch.int64, device="cuda")
    sync()
    t0 = time.perf_counter()
    mlp.start_vectors_stored_fx(H, r_hat, newest_fx, older_fx)
    t_infer = time.perf_counter() - t0
    dummy = torch.empty(1, dtype=torch.float32, device="cuda")
    t_tab = []
    for _ in range(3):  # the tensor-core table kernel alone (the gather reads it for each state)
        sync()
        t0 = time.perf_counter()
        mlp.predict_bf16(H, 0, 0, dummy)
        t_tab.append(time.perf_counter() - t0)
    it_mlp, t_mlp, b_mlp = run_to(target, start=[newest_fx, older_fx], stored=True)
    del newest_fx, older_fx
    newest = torch.empty(4 ** H, dtype=torch.float64, device="cuda")
    older = torch.empty(4 ** H, dtype=torch.float64, device="cuda")

    sync()
    t0 = time.perf_counter()
    lb.lcs_lift_prefix(max(train_h), H, data[max(train_h)][0], r_hat, newest, older)
    t_lift = time.perf_counter() - t0
    it_lift, t_lift_run, b_lift = run_to(target, start=[newest, older])
    mlp.close()

    line = {
        "metric": "iterations and wall time to a bound within 1e-7 of the zero-start converged bound",
        "value": t_infer + t_mlp, "unit": "s", "n_gpus": world, "steps": 1, "warmup": 0,
        "higher_is_better": False, "dtype": "int64", "data": "synthetic (the method's own iterates)",
        "config": {"workload": f"sigma=2 d=2 h={H} ({4 ** H} states); MLP trained on converged iterates of h="
                               f"{train_h}; checks every {chunk} iterations", "tolerance": tol},
        "reference": {"zero_start_iterations": it_ref, "bound": bound_ref},
        "zero_start": {"iterations": it_zero, "seconds": t_zero, "bound": b_zero},
        "truncation_lift": {"iterations": it_lift, "seconds": t_lift + t_lift_run, "bound": b_lift},
        "mlp": {"iterations": it_mlp, "seconds_iterating": t_mlp, "seconds_inference_bf16": t_infer,
                "seconds_table_kernel_min_of_3": min(t_tab), "table_rows": 2 ** (2 * min(H, 12) - 1),
                "start_form": "stored half, fixed point (lcs_mlp_start_vectors_stored_fx + set_start_stored_fx)",
                "seconds_total_with_inference": t_infer + t_mlp, "bound": b_mlp,
                "train_seconds": t_train, "train_steps": cfg["train_steps"], "loss_before": loss0,
                "loss_after": loss, "training_data_seconds": t_data},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_fp32(args, cfg, world, rank, local_rank):
    """Config 4: (2,3,8) and (3,2,8), 1500 iterations from zero, exact fixed point vs float32 storage."""
    import torch

    import paper_2407_10925_gb300 as lb

    torch.cuda.set_device(local_rank)
    results = {}
    for s_, d_, h_ in cfg["shapes"]:
        n = s_ ** (d_ * h_)
        iters = cfg["iters"]
        with lb.LcsBound(s_, d_, h_, check_every=100, timing=1, symmetry=0) as hnd:
            hnd.iterate(iters)
            st = hnd.stats()
            exact = torch.empty(n, dtype=torch.int64, device="cuda")
            lb.lcs_bound_export_fx(hnd.hnd, 0, exact)
            bound, _, r, eps, _ = hnd.read()
        f32 = torch.empty(n, dtype=torch.float64, device="cuda")
        ms32 = lb.lcs_fp32_experiment(s_, d_, h_, iters, r, f32)
        ex = exact.double() / 2.0 ** 44
        err = (f32 - ex).abs()
        results[f"({s_},{d_},{h_})"] = {
            "states": n, "iterations": iters, "bound_fixed_point": bound,
            "fixed_point_ms_per_sweep": st["sweep_ms"] / max(1, st["sweep_launches"]),
            "float32_ms_per_sweep": ms32,
            "float32_max_abs_error": float(err.max()), "float32_max_rel_error": float((err / ex.abs()).max()),
            "float32_mean_abs_error": float(err.mean()),
        }
        del exact, f32, ex, err
        torch.cuda.empty_cache()
        # the library's default path for the shape (symmetric storage where it
        # applies) and, for d >= 3, the max over every non-empty advance set
        variants = [("default_storage", {})]
        if d_ >= 3:
            variants.append(("all_advance_sets", {"f_mode": 1}))
        for name, kw in variants:
            # wall time to the rigorous bound without per-launch events, then
            # the same run with them for the per-sweep time
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with lb.LcsBound(s_, d_, h_, check_every=100, **kw) as hnd:
                hnd.iterate(iters)
                b_rd = hnd.read()[0]
            seconds = time.perf_counter() - t0
            with lb.LcsBound(s_, d_, h_, check_every=100, timing=1, **kw) as hnd:
                hnd.iterate(iters)
                st = hnd.stats()
                bound = hnd.read()[0]
                assert bound == b_rd
                results[f"({s_},{d_},{h_})"][name] = {
                    "ms_per_sweep": st["sweep_ms"] / max(1, st["sweep_launches"]), "bound": bound,
                    "seconds_to_bound": seconds, "stored_states": hnd.n_stored, **kw}
    if rank == 0:
        print(json.dumps({"metric": "float32 storage experiment: error vs exact iterates and sweep time",
                          "config": {"workload": "zero start, 1500 iterations; float32 vs fixed point with full "
                                                 "storage (no symmetry), plus the library's default storage and "
                                                 "(d >= 3) the all-advance-sets F"},
                          "results": results, "note": "no bound is derived from float32 iterates"}), flush=True)


def link_rates(nbytes=1 << 32):
    """host <-> device copy rates of a pinned buffer through PyTorch (GB/s)"""
    import torch

    host = torch.empty(nbytes // 8, dtype=torch.int64, pin_memory=True)
    dev = torch.empty(nbytes // 8, dtype=torch.int64, device="cuda")
    out = {}
    for name, dst, src in (("h2d_gbs", dev, host), ("d2h_gbs", host, dev)):
        best = 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            best = max(best, nbytes / (time.perf_counter() - t0) / 1e9)
        out[name] = best
    del host, dev
    torch.cuda.empty_cache()
    return out


def run_outofcore(args, cfg, world, rank, local_rank):
    """Table 2 beyond device memory: sigma = d = 2 with 32-bit offset-normalised
    rows, one of the three in pinned host memory, from the zero start until the
    bound reaches the paper's printed value (checks every cfg['check'])."""
    import torch

    import paper_2407_10925_gb300 as lb

    torch.cuda.set_device(local_rank)
    H, K, C = cfg["h"], cfg["frac_bits"], cfg["check"]
    rates = link_rates()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hnd = lb.LcsBound(2, 2, H, check_every=C, frac_bits=K, storage=1, host_slots=1, timing=1,
                      stream=stream.cuda_stream)
    t_create = time.perf_counter() - t0
    n_stored = hnd.n_stored
    it, bound, history, reached = 0, 0.0, [], None
    max_iters = args.bound_iters if args.bound_iters is not None else cfg["max_iters"]
    with ClockSampler(local_rank) as clk:
        while it < max_iters:
            hnd.iterate(C)
            it += C
            bound = hnd.read()[0]
            history.append((it, bound, time.perf_counter() - t0))
            if reached is None and math.floor(bound * 1e6 + 1e-9) / 1e6 >= cfg["target"]:
                reached = (it, time.perf_counter() - t0)
                break
    t_total = time.perf_counter() - t0
    st = hnd.stats()
    rep = hnd.report()
    hnd.close()
    sweep_ms = st["sweep_ms"] / max(1, st["sweep_launches"])
    # over three sweeps the host row is written once, read whole once (as the
    # newest input) and read in its distinct half once (as the older input)
    link_bytes = (4 + 4 + 2) * n_stored / 3
    line = {
        "metric": "wall time to Table 2's printed bound out of core", "unit": "s", "value": t_total,
        "higher_is_better": False, "n_gpus": world, "dtype": "int32 storage, int64 arithmetic",
        "data": "the method's own iterates from the zero start",
        "config": {"workload": f"sigma=2 d=2 h={H} ({4 ** H} states, {n_stored} stored): three 32-bit offset-normalised "
                               f"rows of {n_stored * 4 / 2 ** 30:.0f} GiB, one in pinned host memory; {K} fractional "
                               f"bits; a check every {C} iterations", "target": cfg["target"]},
        "result": {"bound_rd": bound, "iterations": it, "reached_target": reached is not None,
                   "iterations_to_target": reached[0] if reached else None,
                   "seconds_to_target": reached[1] if reached else None, "r": rep["r"] / 2 ** K,
                   "eps": rep["eps"] / 2 ** K, "kept_iter": rep["kept_iter"]},
        "create_s": t_create,
        "sweep_ms_mean": sweep_ms, "check_ms_mean": st["check_ms"] / max(1, st["check_launches"]),
        "link": {"algorithmic_bytes_per_sweep": link_bytes, "achieved_gbs": link_bytes / (sweep_ms / 1e3) / 1e9,
                 "copy_rates_gbs": rates},
        "history": history, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    cfg = CONFIGS[args.config]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, cfg, rank)
        return
    if args.config == "batch":
        run_batch(args, cfg, world, rank, local_rank)
        return
    if args.config in ("warm", "warm16"):
        run_warm(args, cfg, world, rank, local_rank)
        return
    if args.config == "fp32":
        run_fp32(args, cfg, world, rank, local_rank)
        return
    if cfg.get("outofcore"):
        run_outofcore(args, cfg, world, rank, local_rank)
        return

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        steps, rate_1core, cores, sample = oracle_sample(cfg, steps=2)
        value = sum(st["states"] for st in steps) / sum(st["seconds"] for st in steps)
        cpu = {"value": value, "unit": "state-updates/s", "cores": cores, "kind": "oracle", "sample": sample,
               "value_1core": rate_1core, "value_all_cores": value}

    import torch

    import paper_2407_10925_gb300 as lb

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    sigma, d, h = cfg["sigma"], cfg["d"], cfg["h"]
    C = args.check_every
    # a dedicated stream: every kernel of the library and the timing events go here
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    K = cfg.get("frac_bits", 44)
    storage = cfg.get("storage", 0)
    hnd = lb.LcsBound(sigma, d, h, check_every=C, timing=1, symmetry=args.symmetry, frac_bits=K, storage=storage,
                      stream=stream.cuda_stream)
    n = hnd.n_states
    for _ in range(args.warmup):
        hnd.iterate(C)
    torch.cuda.synchronize()
    hnd.stats(reset=True)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            hnd.iterate(C)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = reduce_max(ev0.elapsed_time(ev1), dist, "cuda")
    st = hnd.stats(reset=True)
    bound, argmin, r, eps, at_iter = hnd.read()
    rep = hnd.report()

    sweeps = args.steps * C
    value = world * n * sweeps / (ms / 1e3)
    peak, peak_src = measured_peaks()
    achieved = st["sweep_bytes"] / (st["sweep_ms"] / 1e3) / 1e9 if st["sweep_ms"] > 0 else None
    per_launch_bytes = st["sweep_bytes"] / max(1, st["sweep_launches"])
    traffic = profiled_traffic(args.config, "sweep")

    # end to end through the public API from pinned host memory: set the start
    # vectors from the host, run one check period, read the bound.  The start
    # goes in the most compact form the handle takes: the orbit form (sigma =
    # d = 2 with the complement and the swap: a quarter of the states) where
    # it applies, else the stored form (lcs_bound_set_start_stored_fx: the
    # complement half under symmetry).  The same step with the stored form and
    # with full vectors (lcs_bound_set_start_fx, which also verifies the
    # symmetry) is reported beside it.
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        def e2e_run(set_start):
            """the slowest step's time, and the phases of every step (host clock; each phase ends synchronised)"""
            times, phases = [], []
            for i in range(args.e2e_steps + 1):
                barrier()
                torch.cuda.synchronize()
                hnd.stats(reset=True)
                t0 = time.perf_counter()
                set_start()  # synchronous for host vectors
                t1 = time.perf_counter()
                hnd.iterate(C)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                hnd.read()
                torch.cuda.synchronize()
                t3 = time.perf_counter()
                if i > 0:
                    times.append((t3 - t0) * 1e3)
                    x = hnd.stats(reset=True)  # the library's events: copies and the kernels on their values
                    phases.append({"set_start_ms": (t1 - t0) * 1e3, "iterate_ms": (t2 - t1) * 1e3,
                                   "read_ms": (t3 - t2) * 1e3, "h2d_copy_ms": x["h2d_ms"],
                                   "h2d_copy_gbs": x["h2d_bytes"] / max(x["h2d_ms"], 1e-9) / 1e6,
                                   "transfer_kernel_ms": x["xfer_kernel_ms"], "sweep_ms": x["sweep_ms"],
                                   "check_ms": x["check_ms"]})
            return reduce_max(max(times), dist, "cuda"), phases

        def entry(run, h2d, what, host):
            ms, phases = run
            rate = buffer_rate(host)
            return {"value": world * n * C / (ms / 1e3), "ms_per_step": ms, "h2d_bytes_per_step": h2d, "what": what,
                    "host_buffer_h2d_gbs": rate, "phases": phases,
                    "link_ms_at_buffer_rate": h2d / (rate["median"] * 1e9) * 1e3}

        def buffer_rate(host):
            # the plain copy rate of this pinned buffer, 1 GiB segment by
            # segment (min and median over the whole buffer), so that a slow
            # e2e step can be told from a slow host buffer
            m = 1 << 27
            dev = torch.empty(m, dtype=torch.int64, device="cuda")
            rates = []
            for a in range(0, host.numel() - m + 1, m):  # whole segments; each the better of two copies
                best = 0.0
                for _ in range(2):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    dev.copy_(host[a:a + m], non_blocking=True)
                    torch.cuda.synchronize()
                    best = max(best, m * 8 / (time.perf_counter() - t0) / 1e9)
                rates.append(best)
            del dev
            return {"min": min(rates), "median": statistics.median(rates), "segments": len(rates)}

        read_what = " + lcs_bound_iterate(C) + lcs_bound_read"
        try:
            n_orb = hnd.n_orbit
        except lb.LcsError:
            n_orb = None
        forms = {}
        # the host vectors come from lcs_host_alloc (pinned, huge-page advised)
        if n_orb:
            with lb.HostBuffer(n_orb) as buf:
                start_orb = torch.from_numpy(hnd.export_orbit_fx(0, out=buf.array))
                forms["orbit_form"] = entry(e2e_run(lambda: hnd.set_start_orbit_fx([start_orb] * d)), d * n_orb * 8,
                                            "lcs_bound_set_start_orbit_fx from pinned host (d vectors in orbit form)"
                                            + read_what, start_orb)
                del start_orb
        n_st = hnd.n_stored
        with lb.HostBuffer(n_st) as buf:
            start_st = torch.from_numpy(hnd.export_stored_fx(0, out=buf.array))
            forms["stored_form"] = entry(e2e_run(lambda: hnd.set_start_stored_fx([start_st] * d)), d * n_st * 8,
                                         "lcs_bound_set_start_stored_fx from pinned host (d vectors in stored form)"
                                         + read_what, start_st)
            del start_st
        with lb.HostBuffer(n) as buf:
            start = torch.from_numpy(hnd.export_fx(0, out=buf.array))
            forms["full_vectors"] = entry(e2e_run(lambda: hnd.set_start_fx([start] * d)), d * n * 8,
                                          "lcs_bound_set_start_fx from pinned host (every state, symmetry verified "
                                          "on the device)" + read_what, start)
            del start
        head = "orbit_form" if n_orb else "stored_form"
        e2e = {"unit": "state-updates/s", "d2h_bytes_per_step": 80, **forms.pop(head), "form": head,
               "host_buffers": "lcs_host_alloc: pinned, mapped, advised for huge pages", **forms}

    # wall time to the rigorous bound: a fresh handle from the zero start,
    # create .. iterate(bound_iters) .. read, checks every 100 iterations
    n_stored = hnd.n_stored
    hnd.close()
    bound_iters = args.bound_iters if args.bound_iters is not None else cfg.get("bound_iters", 0)
    to_bound = None
    if bound_iters > 0:
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        with lb.LcsBound(sigma, d, h, check_every=100, symmetry=args.symmetry, frac_bits=K, storage=storage,
                         stream=stream.cuda_stream) as hb:
            hb.iterate(bound_iters)
            b_rd = hb.read()[0]
        t_bound = reduce_max(time.perf_counter() - t0, dist, "cuda")
        to_bound = {"iterations": bound_iters, "check_every": 100, "seconds": t_bound, "bound_rd": b_rd,
                    "what": "wall time from lcs_bound_create to lcs_bound_read (zero start), allocation included"}

    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "state-updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "int64",
            "data": "synthetic",
            "config": {
                "workload": workload_name(cfg, args),
                "states": n,
                "stored_states": n_stored,
                "sweeps_per_step": C,
                "symmetry": bool(args.symmetry and n_stored < n),
                "l2": "inputs larger than L2 (each iterate vector is %.1f GiB)" % (n_stored * 8 / 2 ** 30),
                "parallelism": f"replicas x{world}",
            },
            "roofline": {
                "bound": "hbm",
                "kernel": "sweep",
                "achieved": achieved,
                "peak": peak,
                "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                "traffic": traffic,
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "sweep_ms_per_launch": st["sweep_ms"] / max(1, st["sweep_launches"]),
                "check_ms_per_launch": st["check_ms"] / max(1, st["check_launches"]),
                "check": ("each check runs inside the next sweep (the first of the next step), which reads "
                          "4 more bytes per stored state; those bytes count in the sweep's"
                          if st["check_launches"] == 0 else "a kernel of its own per check"),
                **({"note": "general kernels in block form: two launches per sweep, bound by the sums of "
                            "Algorithm 1 formed in shared memory (%.1f terms per state), not by DRAM"
                            % general_terms_per_state(sigma, d)}
                   if cfg.get("general") else {}),
            },
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": st["kernel_launches"],
            "clocks": clocks,
            "result": {"bound_rd": bound, "r": r, "eps": eps, "kept_iter": at_iter, "argmin_state": argmin,
                       "iterations": rep["iters_done"]},
            "time_to_bound": to_bound,
        }
        print(json.dumps(line), flush=True)
    hnd.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
