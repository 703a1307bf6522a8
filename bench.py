#!/usr/bin/env python
"""Throughput benchmark of the solidification time step on GB300.

One benchmark step is one time step of Algorithm 1 (momentum predictor,
pressure projection, solute, two-step energy with the lever rule) on the 3D
box workload: 0.10 x 0.06 x 0.06 m at 128 x 96 x 96 cells (1.18 M), Sn-Pb-like
alloy, left wall Robin-cooled, pressure PCG rel tol 1e-10, transport
BiCGSTAB rel tol 1e-12. Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
    python bench.py --impl reference ...    # the FP64 CPU oracle on host cores

Multi-GPU (torchrun): every rank steps its own independent replica of the
workload (cases shard with no data-path collective); a process-group barrier
brackets the timed region and the time is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2303_10783_gb300 import cases  # noqa: E402

WORKLOAD = "box_3d_128x96x96"
# algorithmic work of the pressure solve (matrix-free 7-point PCG, per cell per iteration):
#   flops: A p 13, (p,q) 2, x += a p 2, r -= a q 2, z = M^-1 r 1, (r,z) 2, (r,r) 2, p = z + b p 2  -> 26
#   bytes (FP64): A p reads p, writes q (16); x/r update reads x p r q, writes x r (48);
#                 p update reads r p, writes p (24)                                  -> 88
PCG_FLOPS_PER_CELL_IT = 26.0
PCG_BYTES_PER_CELL_IT = 88.0
FP64_FLOP_PER_CLK_PER_SM = 4.0   # 2 DFMA per clock per SM (1.25 TFLOP/s nominal at 2070 MHz, 152 SMs)
NUM_SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp64", "mixed"), default="fp64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--ny", type=int, default=96)
    ap.add_argument("--nz", type=int, default=96)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args, rank=0):
    """The benchmark case; rank r gets seed 1 + r (independent replica)."""
    return cases.box_3d(args.nx, args.ny, args.nz, seed=1 + rank)


def init_group(world):
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group("gloo")
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def kernel_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    summary was taken on the current source (its sha256 matches); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = os.path.join(ROOT, "paper_2303_10783_gb300", "csrc", "krylov.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    for line in open(path):
        m = re.match(r"\s*(\S+)\s+sha256=(\w+)\s+bytes_per_launch=([0-9.eE+]+)\s+workload=(\S+)", line)
        if m and m.group(1) == kernel and m.group(2) == sha:
            return float(m.group(3)), m.group(4)
    return None


def cpu_baseline(args):
    """The FP64 oracle as it stands, one full step of the same workload on the host."""
    import oracle
    case = workload(args)
    f = cases.initial_fields(case)
    g = oracle.Grid(case)
    st = oracle.initial_state(case, f["T"], f["C"])
    t = time.perf_counter()
    oracle.step(g, st, case)
    dt = time.perf_counter() - t
    return {"value": g.ncell / dt, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
            "sample": "one full time step of %s (%d cells) from the seeded initial state, numpy/scipy FP64, "
                      "single thread, %.1f s" % (WORKLOAD, g.ncell, dt)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    # bounded sample of the workload: the same box at half resolution per axis
    case = cases.box_3d(max(args.nx // 2, 2), max(args.ny // 2, 2), max(args.nz // 2, 2), seed=1)
    f = cases.initial_fields(case)
    g = oracle.Grid(case)
    st = oracle.initial_state(case, f["T"], f["C"])
    for _ in range(args.warmup):
        st = oracle.step(g, st, case)
    t = time.perf_counter()
    for _ in range(args.steps):
        st = oracle.step(g, st, case)
    dt = time.perf_counter() - t
    value = g.ncell * args.steps / dt
    sample = ("the %s workload's box at half resolution per axis (%dx%dx%d = %d cells), %d timed steps after %d "
              "warm-up, numpy/scipy FP64, single thread" % (WORKLOAD, g.n[0], g.n[1], g.n[2], g.ncell, args.steps,
                                                            args.warmup))
    out = {"metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "sample_cells": g.ncell, "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_ours(args):
    import torch
    from paper_2303_10783_gb300 import solid
    rank, world, local = dist_env()
    dist = init_group(world)
    torch.cuda.set_device(local)
    solid.load()
    precision = solid.SS_MIXED if args.precision == "mixed" else solid.SS_FP64
    case = workload(args, rank)
    f = cases.initial_fields(case)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c = solid.Case(case, precision=precision, stream=stream)
        c.initialize(f["T"], f["C"])
        c.step(args.warmup)
        c.sync()
        c.get_profile()   # reset accumulators
        c.set_profiling(True)
        sampler = ClockSampler(local)
        barrier(dist)
        stream.synchronize()
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(args.steps)
        e1.record(stream)
        stream.synchronize()
        clocks = sampler.stop()
        barrier(dist)
        ms = e0.elapsed_time(e1)
        status = c.sync(allow=(solid.SS_ENOTCONV,))
        prof = c.get_profile()
        stats = c.stats()
        c.set_profiling(False)

        # end to end through the public API with host buffers: every step uploads
        # its full input state from pinned host memory, steps, and reads back all fields
        e2e = None
        if not args.no_e2e:
            state = c.get_fields()
            host = {k: torch.from_numpy(v).pin_memory() for k, v in state.items() if not (k == "w" and case["dim"] == 2)}
            out = {k: torch.empty_like(v).pin_memory() for k, v in host.items()}
            h2d = sum(v.numel() * 8 for v in host.values())
            d2h = h2d
            ke = max(2, min(args.steps, 5))
            barrier(dist)
            stream.synchronize()
            t0 = time.perf_counter()
            for _ in range(ke):
                c.set_fields({k: v.numpy() for k, v in host.items()})
                c.step(1)
                c.get_fields(tuple(out.keys()), out=out)
            stream.synchronize()
            e2e_s = time.perf_counter() - t0
            barrier(dist)
            e2e_s = max_over_ranks(dist, e2e_s)
            e2e = {"value": sum_over_ranks(dist, case["nx"] * case["ny"] * case["nz"] * ke) / e2e_s,
                   "unit": "cell-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "steps": ke, "path": "ss_set_fields(host) + ss_step(1) + ss_get_fields(host) per step"}
        c.close()

    ms_max = max_over_ranks(dist, ms)
    ncell = case["nx"] * case["ny"] * case["nz"]
    total_cells = sum_over_ranks(dist, ncell * args.steps)
    value = total_cells / (ms_max * 1e-3)

    # roofline of the dominant stage (device time measured by the library's events on the case stream)
    stage_ms = prof["ms"]
    top = max(stage_ms, key=stage_ms.get)
    peaks = measured_peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roof = None
    if top == "solve_p":
        its = prof["iters"]["p"]
        launches = max(prof["launches"]["solve_p"], 1)
        t_launch = stage_ms[top] * 1e-3 / launches
        flops = PCG_FLOPS_PER_CELL_IT * ncell * its / launches
        bytes_ = PCG_BYTES_PER_CELL_IT * ncell * its / launches
        if args.precision == "fp64":
            peak = FP64_FLOP_PER_CLK_PER_SM * NUM_SMS * sm_mhz * 1e6 / 1e12
            ach = flops / t_launch / 1e12
            roof = {"bound": "alu", "kernel": "k_pcg_poisson", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak,
                    "peak_basis": "FP64 pipe: 4 flop/clk/SM x 152 SMs x %.0f MHz median SM clock under load" % sm_mhz,
                    "hbm_achieved_GBps": bytes_ / t_launch / 1e9,
                    "hbm_frac_of_measured": bytes_ / t_launch / 1e9 / peaks.get("hbm_gbs", 6687.1)}
        else:
            hbm = peaks.get("hbm_gbs", 6687.1)
            ach = bytes_ / 2 / t_launch / 1e9
            roof = {"bound": "hbm", "kernel": "k_pcg_poisson", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm}
        tr = kernel_traffic("k_pcg_poisson")
        roof["traffic"] = tr[0] if tr else None
        roof["algorithmic_per_launch"] = {"flops": flops, "bytes": bytes_, "iterations": its / launches,
                                          "cells": ncell}
        roof["launch_ms"] = t_launch * 1e3
    if rank != 0:
        return 0
    out = {
        "metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": ncell, "precision": args.precision, "tol_p": case["tol_p"],
                   "tol_t": case["tol_t"], "dt": case["dt"], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: each step streams ~0.5 GB of fields and DIA planes (L2 129 MB); "
                         "no flush"},
        "status": solid.STATUS_NAMES.get(status, status),
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": prof["kernels"],
        "roofline": roof,
        "stage_ms_per_step": {k: v / args.steps for k, v in stage_ms.items() if v > 0},
        "iters_per_step": {k: v / args.steps for k, v in prof["iters"].items()},
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
