#!/usr/bin/env python3
"""Throughput benchmark of the SneakySnake filter on GB300; prints one JSON
line.

Workload (short-read threshold sweep): 30,000,000 read/reference pairs of
100 bp, seeded and synthetic -- even pairs carry Poisson(3) random edits,
odd pairs are independent random sequences (the shape of the paper's
100 bp datasets, Section 3.1) -- filtered at E = 0, 2, 4, 6, 8, 10.

One step = the whole hot path over the batch: pack the resident ASCII reads
and references to 2 bits (2 launches) and run one plain filter launch per
threshold (6 launches).  ``value`` counts pair decisions (pairs x
thresholds) per second with the inputs resident in HBM; the inputs (6 GB
ASCII + 1.7 GB packed) are far larger than L2, so no flush is needed.
``e2e`` runs the same sweep through ``ss_filter_host`` from pinned host
buffers (copies inside the timed region).  ``cpu_baseline`` times the CPU
oracle on a bounded sample on the host cores.

``--impl reference`` times the CPU oracle alone on the same workload (the
reference arm).  Under torchrun each rank filters its own 30M pairs (weak
scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_PAIRS = 30_000_000
M = 100
SWEEP = [0, 2, 4, 6, 8, 10]
SEED = 1910_09020 + 2
WORKLOAD = ("short-read threshold sweep: 30M synthetic pairs x 100 bp "
            "(even pairs Poisson(3) edits, odd pairs random), "
            "E in {0,2,4,6,8,10}, plain one-launch-per-threshold form")
METRIC = "sequence pairs/sec (and Gbases/s) per GB300 vs roofline"
# algorithmic bytes of one pair decision: both sequences at 2 bits per base
# plus the accept byte and the int32 obstacle count
FILTER_BYTES_PER_PAIR = 2 * ((M + 3) // 4) + 1 + 4
# pack: both sequences read as ASCII, written at 2 bits per base
PACK_BYTES_PER_PAIR = 2 * M + 2 * ((M + 3) // 4)
# op model of the method per the lazy maze of Section 2.4: per evaluated
# 32-column row word 7 logic/shift ops + 1 find-first; per iteration one
# max per row plus 4 bookkeeping ops
K_WORD, K_RED, K_ITER = 7, 1, 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pairs", type=int, default=N_PAIRS,
                    help="pairs per GPU (default: the full workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


# ---- distributed plumbing ----------------------------------------------------

def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(local)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks --------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device),
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---- peaks ---------------------------------------------------------------------

def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "hbm_source": "measured"}
    return {"hbm_gbs": 6800.0, "hbm_source": "fallback"}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1910_09020_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str) -> float | None:
    """DRAM bytes per pair of a kernel from the committed ncu summary, or
    None if the kernels changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("source_sha") != kernel_source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else float(k["dram_bytes_per_pair"])


# ---- CPU oracle (baseline leg and reference arm) --------------------------------

def oracle_sample(n: int, first: int = 0):
    from paper_1910_09020_gb300 import synth
    return synth.pairs_fixed(SEED, first, n, M, synth.SHORT_POISSON)


def time_oracle(reads, refs, threads: int = 0):
    """Oracle over every threshold of the sweep; returns (seconds, per-E
    stats (cells, words, iterations) summed over pairs)."""
    import oracle
    stats = {}
    t0 = time.perf_counter()
    for E in SWEEP:
        _, _, st = oracle.filter_batch(reads, refs, M, E, threads=threads,
                                       with_stats=True)
        stats[E] = st
    return time.perf_counter() - t0, stats


def cpu_baseline(target_s: float):
    import oracle
    cores = oracle.default_threads()
    probe_n = 20000
    r, f = oracle_sample(probe_n)
    dt, _ = time_oracle(r, f)
    n = int(min(N_PAIRS, max(probe_n, probe_n * target_s / max(dt, 1e-6))))
    r, f = oracle_sample(n)
    dt, stats = time_oracle(r, f)
    value = n * len(SWEEP) / dt
    return {
        "value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
        "sample": f"first {n} pairs of the workload x {len(SWEEP)} thresholds "
                  f"({dt:.1f} s, {cores} host threads)",
    }, stats, n


def op_model(stats: dict, n: int) -> dict:
    """Per-pair algorithmic ALU and find-first ops of each threshold."""
    out = {}
    for E, (cells, words, iters) in stats.items():
        alu = (words * K_WORD + iters * (2 * E + 1) * K_RED + iters * K_ITER)
        out[E] = {"alu_ops_per_pair": alu / n, "xu_ops_per_pair": words / n,
                  "iterations_per_pair": iters / n,
                  "cells_per_pair": cells / n}
    return out


# ---- reference arm ----------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    cores = oracle.default_threads()
    r, f = oracle_sample(20000)
    dt, _ = time_oracle(r, f)
    per_step_s = 1.5
    total_budget = 150.0
    steps_total = args.steps + args.warmup
    per_step_s = min(per_step_s, total_budget / max(steps_total, 1))
    n = int(max(2000, 20000 * per_step_s / max(dt, 1e-6)))
    times = []
    for s in range(steps_total):
        rr, ff = oracle_sample(n, first=s * n)
        dt, _ = time_oracle(rr, ff)
        if s >= args.warmup:
            times.append(dt)
    t = float(np.sum(times))
    value = n * len(SWEEP) * len(times) / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "pairs/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic",
        "config": config_dict(args.gpus, n_override=n),
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{n} pairs x {len(SWEEP)} thresholds "
                                   f"per step"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_dict(world: int, n_override: int | None = None) -> dict:
    return {"workload": WORKLOAD, "pairs_per_gpu": n_override or N_PAIRS,
            "read_length": M, "thresholds": SWEEP, "format": "ASCII resident, "
            "packed to 2 bits in the step", "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (6 GB ASCII + 1.7 GB packed)"}


# ---- our arm ---------------------------------------------------------------------

def run_ours(args):
    import torch

    from paper_1910_09020_gb300 import binding, synth
    from paper_1910_09020_gb300.peaks import measure as measure_int_peaks

    rank, world, local = dist_setup()
    n = args.pairs
    dev = torch.device("cuda", local)

    # inputs: generated into pinned host memory, copied once to HBM
    t0 = time.perf_counter()
    hq = torch.empty(n * M, dtype=torch.uint8, pin_memory=True)
    hr = torch.empty(n * M, dtype=torch.uint8, pin_memory=True)
    synth.pairs_fixed(SEED, rank * n, n, M, synth.SHORT_POISSON,
                      out=(hq.numpy(), hr.numpy()))
    gen_s = time.perf_counter() - t0
    dq = hq.to(dev, non_blocking=True)
    dr = hr.to(dev, non_blocking=True)
    torch.cuda.synchronize()

    F = binding.Filter(local, workspace_bytes=8 << 30)
    W16 = binding.ss_packed_words(M)
    pq = torch.empty(n * W16, dtype=torch.int32, device=dev)
    pr = torch.empty(n * W16, dtype=torch.int32, device=dev)
    acc = torch.empty((len(SWEEP), n), dtype=torch.uint8, device=dev)
    obs = torch.empty((len(SWEEP), n), dtype=torch.int32, device=dev)
    # events on the stream the kernels are launched on (torch's current
    # stream, passed to the library), one set per timed step
    nev = 2 + 2 * len(SWEEP)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)]
           for _ in range(args.steps)]
    launch_ms = {"pack": [], **{E: [] for E in SWEEP}}

    def step(ev):
        if ev:
            ev[0].record()
        F.pack(dq, m=M, n=n, out=pq)
        F.pack(dr, m=M, n=n, out=pr)
        if ev:
            ev[1].record()
        for t, E in enumerate(SWEEP):
            if ev:
                ev[2 + 2 * t].record()
            F.filter(pq, pr, m=M, e=E, n=n, out_accept=acc[t],
                     out_obstacles=obs[t])
            if ev:
                ev[3 + 2 * t].record()

    for _ in range(args.warmup):
        step(None)
    F.sync()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    start, stop = (torch.cuda.Event(enable_timing=True),
                   torch.cuda.Event(enable_timing=True))
    start.record()
    for s in range(args.steps):
        step(evs[s])
    stop.record()
    torch.cuda.synchronize()
    for ev in evs:
        launch_ms["pack"].append(ev[0].elapsed_time(ev[1]))
        for t, E in enumerate(SWEEP):
            launch_ms[E].append(ev[2 + 2 * t].elapsed_time(ev[3 + 2 * t]))
    barrier(world)
    clk = clocks.stop()
    elapsed_ms = start.elapsed_time(stop)
    F.sync()
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    pairs_per_step = n * len(SWEEP)
    value = world * pairs_per_step * args.steps / (elapsed_ms * 1e-3)

    # e2e: the public host-buffer call, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hacc = torch.empty((len(SWEEP), n), dtype=torch.uint8, pin_memory=True)
        hobs = torch.empty((len(SWEEP), n), dtype=torch.int32, pin_memory=True)
        hq2, hr2 = hq.view(n, M), hr.view(n, M)
        F.filter_host(hq2, hr2, m=M, e=SWEEP, fmt=binding.SS_FMT_ASCII,
                      out_accept=hacc, out_obstacles=hobs)
        e2e_steps = max(3, args.steps // 6)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            F.filter_host(hq2, hr2, m=M, e=SWEEP, fmt=binding.SS_FMT_ASCII,
                          out_accept=hacc, out_obstacles=hobs)
        dt = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": world * pairs_per_step * e2e_steps / dt,
               "unit": "pairs/s", "h2d_bytes_per_step": 2 * n * M,
               "d2h_bytes_per_step": 5 * n * len(SWEEP),
               "ms_per_step": 1e3 * dt / e2e_steps}
        # the device path and the host path must agree
        same = (torch.equal(hacc, acc.cpu()) and torch.equal(hobs, obs.cpu()))
        e2e["matches_device_path"] = bool(same)

    if rank != 0:
        F.close()
        return 0

    # roofline of the dominant kernel: the filter launches of the sweep
    peaks = measured_peaks()
    ipk = measure_int_peaks(local)
    cpu = None
    model = None
    if not args.no_cpu and world == 1:
        cpu, stats, sample_n = cpu_baseline(args.cpu_seconds)
        model = op_model(stats, sample_n)
    hbm = peaks["hbm_gbs"] * 1e9
    per_launch = []
    roof_total = meas_total = 0.0
    for E in SWEEP:
        ms = float(np.mean(launch_ms[E]))
        t_hbm = n * FILTER_BYTES_PER_PAIR / hbm
        d = {"E": E, "ms": ms, "pairs_per_s": n / (ms * 1e-3),
             "hbm_gbs": n * FILTER_BYTES_PER_PAIR / (ms * 1e-3) / 1e9,
             "t_hbm_ms": 1e3 * t_hbm}
        t_bound, bound = t_hbm, "hbm"
        if model:
            t_alu = n * model[E]["alu_ops_per_pair"] / ipk["lop3"]
            t_xu = n * model[E]["xu_ops_per_pair"] / ipk["bfind"]
            d.update({"t_alu_ms": 1e3 * t_alu, "t_xu_ms": 1e3 * t_xu,
                      "alu_ops_per_pair": model[E]["alu_ops_per_pair"],
                      "tops": n * model[E]["alu_ops_per_pair"] / (ms * 1e-3)
                      / 1e12})
            if max(t_alu, t_xu) > t_bound:
                t_bound, bound = max(t_alu, t_xu), ("alu" if t_alu >= t_xu
                                                    else "xu")
        d["bound"] = bound
        d["frac"] = 1e3 * t_bound / ms
        roof_total += 1e3 * t_bound
        meas_total += ms
        per_launch.append(d)
    filter_ms = sum(float(np.mean(launch_ms[E])) for E in SWEEP)
    pack_ms = float(np.mean(launch_ms["pack"]))
    alu_share = sum(d["ms"] for d in per_launch if d["bound"] != "hbm")
    dom_bound = "alu" if alu_share > filter_ms / 2 else "hbm"
    if dom_bound == "hbm":
        achieved = n * FILTER_BYTES_PER_PAIR * len(SWEEP) / (filter_ms * 1e-3) / 1e9
        peak, unit = peaks["hbm_gbs"], "GB/s"
    else:
        ops = sum(n * model[E]["alu_ops_per_pair"] for E in SWEEP)
        achieved = ops / (filter_ms * 1e-3) / 1e12
        peak, unit = ipk["lop3"] / 1e12, "Tops/s"
    traffic = ncu_traffic("k_rw_uniform")
    roofline = {
        "kernel": "k_rw_uniform (plain filter, one launch per E)",
        "bound": dom_bound, "achieved": achieved, "peak": peak, "unit": unit,
        "frac": roof_total / meas_total,
        "frac_note": "sum over the sweep of max(HBM, ALU, find-first) "
                     "roofline time / measured time",
        "traffic": None if traffic is None else traffic * n,
        "algorithmic_bytes_per_launch": n * FILTER_BYTES_PER_PAIR,
        "peak_source": f"HBM {peaks['hbm_source']} ({peaks['hbm_gbs']} GB/s); "
                       "integer pipes measured live by microbenchmark",
        "int_peaks_tops": {k: v / 1e12 for k, v in ipk.items()},
        "per_launch": per_launch,
    }
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s",
        "gbases_per_s": value * M / 1e9, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": config_dict(world, n),
        "clocks": clk, "e2e": e2e,
        "gpu_launches": (2 + len(SWEEP)) * args.steps,
        "roofline": roofline, "cpu_baseline": cpu,
        "breakdown": {"pack_ms": pack_ms, "filter_ms": filter_ms,
                      "pack_gbs": n * PACK_BYTES_PER_PAIR / (pack_ms * 1e-3)
                      / 1e9, "generate_s": gen_s},
    }
    print(json.dumps(line), flush=True)
    F.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
