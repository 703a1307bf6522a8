#!/usr/bin/env python
"""Throughput benchmark of the solidification time step on GB300.

One benchmark step is one time step of Algorithm 1 (momentum predictor,
pressure projection, solute, two-step energy with the lever rule) on the 3D
box workload: 0.10 x 0.06 x 0.06 m at 128 x 96 x 96 cells (1.18 M), Sn-Pb-like
alloy, left wall Robin-cooled, pressure solve rel tol 1e-10, transport solves
rel tol 1e-12. The headline is the mixed-precision path (FP32 inner
iterations in FP64 refinement); the FP64 path is measured beside it at the
same tolerances. Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision both|mixed|fp64]
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2303_10783_gb300 import cases  # noqa: E402

# Algorithmic work per unit of the kernels whose roofline the line reports (the
# dominant stage of a step). Bytes are what the method must move per cell or row;
# flops are arithmetic operations (FMA = 2) in the kernel's own precision.
#
# k_pcg_mg (multigrid-preconditioned CG), per fine cell:
#   one CG iteration with a V(2,2)-cycle moves, at the fine level, A p (8 B in FP32), the x/r
#   update with the first smoothing sweep (32), second pre-sweep (12), residual (12),
#   restriction (5), prolongation (8.5), two post-sweeps (24), the dot products (8) and the
#   p update (12) = 121.5 B, plus ~10 B on the coarser levels -> 131 B in FP32, 262 B in FP64.
#   One FP64 refinement sweep of the mixed path adds 44 B (r = b - A x: 24, x += d: 20).
#   FP64 flops per CG iteration: A p and (p,q) 12, updates 5, pre-sweep 13, residual 11,
#   restriction 21, prolongation 15, post-sweeps 26, dots 6, p update 3 = 112, coarse levels
#   ~13 -> 125.
MG_BYTES_PER_CELL_IT = {"mixed": 131.0, "fp64": 262.0}
MG_BYTES_PER_CELL_REFINE = 44.0
MG_FLOPS_PER_CELL_IT = 125.0
# k_poisson_dct (cosine-transform solver in FP64 refinement), per cell, with E the size in
# bytes of the transform type (4 mixed, 8 FP64):
#   per sweep: pass A reads the FP64 residual (8) and writes T1 (E); pass B reads T1 (E),
#   writes T2 (E), reads and writes it in the tridiagonal solves (2E), reads it (E) and writes
#   T1 (E); pass C reads T1 (E) and reads and writes x (16); the FP64 residual reads x and b
#   and writes r (24): 48 + 8E B. Once per launch: the mean of b (8), b and x set (24), the
#   gauge (24): 56 B.
#   flops per sweep: the forward and inverse transforms are 2 (Mx + My) multiply-adds
#   (4 (Mx + My) flops, My = 0 in 2D) and the tridiagonal solve ~8, in the transform type;
#   the FP64 residual ~16.
DCT_BYTES_PER_CELL_SWEEP_BASE = 48.0
DCT_BYTES_PER_CELL_LAUNCH = 56.0
DCT_THOMAS_FLOPS = 8.0
# k_bicgstab_ir (mixed transport: FP32 inner solve in FP64 refinement), per row:
#   the first FP64 residual reads 7 FP64 planes, x and b and writes r and its FP32 copy (84);
#   each sweep adds the correction (x read and written, d read: 20) and forms the next
#   residual (7 planes, x, b read, r and its copy written: 84): 104; a BiCGSTAB inner
#   iteration moves 7 FP32 planes twice (56) and ~80 B of FP32 vectors: 136.
BCG_IR_BYTES_ROW = 84.0
BCG_IR_BYTES_ROW_SWEEP = 104.0
BCG_IR_BYTES_ROW_IT = 136.0
# k_helmholtz_dct (the T* pre-solve of the mixed path), per cell: the first FP64 residual with
#   the system's 7 FP64 planes, x and b, staged in FP32 (76 B); per sweep the transforms move
#   the staged residual and T1 (4 + 4 + 8 in passes A and B), pass C reads T1 and reads and
#   writes x (20), the FP64 residual again (76): 112 B; 4 (n_x + n_y) + 8 FP32 flop per sweep.
HELM_BYTES_PER_CELL = 76.0
HELM_BYTES_PER_CELL_SWEEP = 112.0
# k_bicgstab (FP64 transport), per row and iteration: two SpMVs over 7 FP64 planes (2 x 72)
# and the vector updates (~156 B): 300 B; 2 x 13 + 20 = 46 FP64 flops.
# Jacobi sweep of a transport solve, per row: mixed (FP32, inside the refinement) 7 FP32
#   planes, the inverse diagonal, the staged residual and d read, d written: 44 B, ~16 FP32
#   flop; FP64: 7 FP64 planes, x, b and the inverse diagonal read, x written: 88 B, 19 FP64 flop.
JAC_BYTES_ROW = {"mixed": 44.0, "fp64": 88.0}
JAC_FLOPS_ROW = {"mixed": 16.0, "fp64": 19.0}
BCG_BYTES_ROW_IT = 300.0
# assembly of one transport row (a1, a6, a8): ~6 inputs read (48 B) and 7 FP64 planes, the
#   right-hand side and 8 FP32 planes written (96 B) on the mixed path; the FP64 path writes
#   7 FP64 planes, b and the FP64 inverse diagonal (72 B)
ASM_BYTES_ROW = {"mixed": 144.0, "fp64": 120.0}
# pressure right-hand side: u*, v*, w* read at each cell's faces (24 B), b written (8 B)
RHS_BYTES_CELL = 32.0
# lever rule: T*, g_l, C and the T* increment read, T, g_l, C_l, C_s, K^-1, A_g, increment written
LEVER_BYTES_CELL = 88.0
BCG_FLOPS_ROW_IT = 46.0
FP64_FLOP_PER_CLK_PER_SM = 4.0    # 2 DFMA per clock per SM (1.26 TFLOP/s at 2070 MHz, 152 SMs)
FP32_FLOP_PER_CLK_PER_SM = 256.0  # 128 FP32 FMA per clock per SM (80.6 TFLOP/s at 2070 MHz)
NUM_SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("both", "mixed", "fp64"), default="both",
                    help="both: headline = mixed path, FP64 path measured alongside")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=("box", "batched", "serving", "ingot"), default="box",
                    help="box: the 128x96x96 headline; batched: 64 independent cavities; serving: request stream; "
                         "ingot: 384x256x256")
    ap.add_argument("--requests", type=int, default=120, help="serving: requests in the sample")
    ap.add_argument("--request-steps", type=int, default=50, help="serving: steps per request in the sample")
    ap.add_argument("--no-extras", action="store_true",
                    help="box workload only: skip the cavity, ingot, batched and serving legs of the default line")
    ap.add_argument("--slots", type=int, default=16, help="serving: requests on the GPU at once at most (0: budget only)")
    ap.add_argument("--block-cap", type=int, default=-1,
                    help="serving: blocks per cooperative solver launch of each request (0: no cap; "
                         "-1: in proportion to the request's cells)")
    ap.add_argument("--precond", choices=("dct", "mg", "jacobi"), default=None,
                    help="pressure solver (default: the workload's own)")
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--ny", type=int, default=96)
    ap.add_argument("--nz", type=int, default=96)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args, rank=0, k=1):
    """The benchmark case; rank r gets seed 1 + r (independent replica). k > 1:
    the same case at 1/k of the resolution per axis (a bounded oracle sample)."""
    nx, ny, nz = max(args.nx // k, 2), max(args.ny // k, 2), max(args.nz // k, 2)
    if getattr(args, "workload", "box") == "ingot":
        case = cases.ingot_3d(nx, ny, nz, seed=4 + rank)
    else:
        case = cases.box_3d(nx, ny, nz, seed=1 + rank)
    if getattr(args, "precond", None):
        case["precond_p"] = args.precond
    return case


def workload_name(args):
    kind = "ingot" if getattr(args, "workload", "box") == "ingot" else "box"
    return "%s_3d_%dx%dx%d" % (kind, args.nx, args.ny, args.nz)


# Oracle samples are bounded: the workload's own case at the smallest
# per-axis reduction k that keeps it within a cell budget (the oracle runs
# ~1e5 cell-steps/s on one host core, so 1.3 M cells is ~12 s per step).
CPU_BASELINE_MAX_CELLS = 1_300_000     # one step (cpu_baseline leg)
REFERENCE_MAX_CELLS = 160_000          # warm-up + timed steps (--impl reference)


def sample_case(args, max_cells):
    """(case, k): the workload at 1/k resolution per axis, k the smallest with <= max_cells cells."""
    k = 1
    while max(args.nx // k, 2) * max(args.ny // k, 2) * max(args.nz // k, 2) > max_cells:
        k += 1
    return workload(args, k=k), k


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
        self.path = os.path.join(tempfile.gettempdir(), "solid_clocks_%d.csv" % os.getpid())

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


KERNEL_SOURCES = {"k_pcg_mg": ("mg.cu",), "k_poisson_dct": ("dct.cu", "umma.cuh"),
                  "k_helmholtz_dct": ("dct.cu", "umma.cuh"), "k_bicgstab_ir": ("krylov.cu",),
                  "k_bicgstab": ("krylov.cu",), "k_pcg_poisson": ("krylov.cu",)}


def kernel_source_sha(kernel="k_bicgstab_ir"):
    """sha256 over the source files of `kernel` and the shared header."""
    h = hashlib.sha256()
    base = kernel.split("<")[0]
    for f in KERNEL_SOURCES.get(base, ("krylov.cu",)) + ("solid_internal.cuh",):
        h.update(open(os.path.join(ROOT, "paper_2303_10783_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kernel_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    summary was taken on the current source (its sha256 matches) and on this
    workload; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(kernel)
    for line in open(path):
        m = re.match(r"\s*(\S+)\s+sha256=(\w+)\s+bytes_per_launch=([0-9.eE+]+)\s+workload=(\S+)", line)
        if m and m.group(1) == kernel and m.group(2) == sha and m.group(4) == workload:
            return float(m.group(3)), m.group(4)
    return None


def cpu_baseline(args):
    """The FP64 oracle as it stands, one full step of the same workload on the host."""
    import oracle
    case, k = sample_case(args, CPU_BASELINE_MAX_CELLS)
    f = cases.initial_fields(case)
    g = oracle.Grid(case)
    st = oracle.initial_state(case, f["T"], f["C"])
    t = time.perf_counter()
    oracle.step(g, st, case)
    dt = time.perf_counter() - t
    res = "" if k == 1 else " at 1/%d resolution per axis (%dx%dx%d)" % (k, g.n[0], g.n[1], g.n[2])
    return {"value": g.ncell / dt, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
            "sample": "one full time step of %s%s (%d cells) from the seeded initial state, numpy/scipy FP64, "
                      "single thread, %.1f s" % (workload_name(args), res, g.ncell, dt)}


def _oracle_step_at(job):
    """One oracle step of the box workload at (nx, ny, nz), started at wall time
    `start` (so that every process steps at once); returns (cells, begin, end)."""
    nx, ny, nz, seed, start = job
    import oracle
    from paper_2303_10783_gb300 import cases as cs
    case = cs.box_3d(nx, ny, nz, seed=seed)
    f = cs.initial_fields(case)
    g = oracle.Grid(case)
    st = oracle.initial_state(case, f["T"], f["C"])
    while time.time() < start:
        time.sleep(0.01)
    t0 = time.time()
    oracle.step(g, st, case)
    return g.ncell, t0, time.time()


def cpu_all_cores(args, delay=8.0):
    """The oracle as it stands on every host core at once: one independent
    replica per core (spawned processes, one thread each), each taking one
    step of the workload at half its resolution per axis; throughput = the
    replicas' cells over the span from the first start to the last end."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    nx, ny, nz = max(args.nx // 2, 2), max(args.ny // 2, 2), max(args.nz // 2, 2)
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        start = time.time() + delay        # after every process has imported numpy and scipy
        with ctx.Pool(ncores) as pool:
            res = pool.map(_oracle_step_at, [(nx, ny, nz, 100 + q, start) for q in range(ncores)])
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    cells = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    try:
        import platform
        model = platform.processor() or platform.machine()
    except Exception:
        model = "unknown"
    return {"value": cells / span, "unit": "cell-steps/s", "cores": ncores, "kind": "oracle",
            "cpu": model,
            "sample": "%d independent replicas (one per core, one thread each), one step each of %s at 1/2 "
                      "resolution per axis (%dx%dx%d), numpy/scipy FP64, %.1f s span"
                      % (ncores, workload_name(args), nx, ny, nz, span)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    # bounded sample of the workload: the same case at reduced resolution per axis
    case, k = sample_case(args, REFERENCE_MAX_CELLS)
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
    sample = ("the %s workload at 1/%d resolution per axis (%dx%dx%d = %d cells), %d timed steps after %d "
              "warm-up, numpy/scipy FP64, single thread" % (workload_name(args), k, g.n[0], g.n[1], g.n[2], g.ncell,
                                                            args.steps, args.warmup))
    out = {"metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": workload_name(args), "sample_cells": g.ncell, "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def measure(args, precision_name, case, dist, local):
    """Warm up, then time args.steps steps of one case on its own stream.
    Returns the measured quantities (max over ranks applied by the caller)."""
    import torch
    from paper_2303_10783_gb300 import solid
    precision = solid.SS_MIXED if precision_name == "mixed" else solid.SS_FP64
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
        # fields after warm-up + timed steps (outside the timed region), to state the
        # mixed path's per-field error against the FP64 path on the full workload
        fields = c.get_fields(("u", "v", "w", "p", "T", "C", "gl"))
        e2e = None
        if not args.no_e2e:
            # end to end through the public API with host buffers: every step uploads its full
            # input state from pinned host memory, steps, and reads every field back to pinned
            # host memory. The copies run on a side stream, double-buffered through device
            # buffers: step k+1's upload and step k's read-back overlap the compute of the
            # neighbouring step; every byte still crosses inside the timed region.
            state = c.get_fields()
            host = {k: torch.from_numpy(v).pin_memory() for k, v in state.items() if not (k == "w" and case["dim"] == 2)}
            out = {k: torch.empty_like(v).pin_memory() for k, v in host.items()}
            names = tuple(host.keys())
            nbytes = sum(v.numel() * 8 for v in host.values())
            dev_in = [{k: torch.empty(v.shape, dtype=torch.float64, device="cuda") for k, v in host.items()}
                      for _ in range(2)]
            dev_out = [{k: torch.empty(v.shape, dtype=torch.float64, device="cuda") for k, v in host.items()}
                       for _ in range(2)]
            side = torch.cuda.Stream()
            up = [torch.cuda.Event() for _ in range(2)]     # input buffer q holds its step's upload
            used = [torch.cuda.Event() for _ in range(2)]   # input buffer q has been consumed
            down = [torch.cuda.Event() for _ in range(2)]   # output buffer q has been read back

            def upload(q):
                with torch.cuda.stream(side):
                    side.wait_event(used[q])
                    for k in names:
                        dev_in[q][k].copy_(host[k], non_blocking=True)
                    up[q].record(side)

            ke = max(2, args.steps)
            barrier(dist)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            upload(0)
            for k_step in range(ke):
                q = k_step % 2
                stream.wait_event(up[q])
                c.set_fields(dev_in[q])                      # device to device on the case stream
                used[q].record(stream)
                if k_step + 1 < ke:
                    upload(1 - q)                            # the next step's input, during this step
                c.step(1)
                stream.wait_event(down[q])
                c.get_fields(names, device=True, out=dev_out[q])
                with torch.cuda.stream(side):
                    side.wait_stream(stream)
                    for k in names:
                        out[k].copy_(dev_out[q][k], non_blocking=True)
                    down[q].record(side)
            side.synchronize()
            stream.synchronize()
            e2e_s = time.perf_counter() - t0
            barrier(dist)
            e2e = dict(seconds=e2e_s, steps=ke, h2d=nbytes, d2h=nbytes)
        c.close()
    return dict(ms=ms, status=solid.STATUS_NAMES.get(status, status), prof=prof, stats=stats, clocks=clocks, e2e=e2e,
                fields=fields)


def field_errors(a, b, dim):
    """Relative L-inf difference of fields a against b: scalars against their own
    largest value, the velocity as one vector field against its largest component."""
    import numpy as np
    out = {}
    for k in ("p", "T", "C", "gl"):
        out[k] = float(np.abs(a[k] - b[k]).max() / max(np.abs(b[k]).max(), 1e-300))
    comps = ("u", "v", "w")[:dim]
    vmax = max(float(np.abs(b[k]).max()) for k in comps)
    out["velocity"] = max(float(np.abs(a[k] - b[k]).max()) for k in comps) / max(vmax, 1e-300)
    return out


def _rows(case, sysname):
    nx, ny, nz = case["nx"], case["ny"], case["nz"] if case["dim"] == 3 else 1
    return {"u": (nx + 1) * ny * nz, "v": nx * (ny + 1) * nz, "w": nx * ny * (nz + 1)}.get(sysname, nx * ny * nz)


def kernel_work(stage, precision_name, case, prof, stats):
    """Algorithmic work of the launches of `stage` in the timed steps (from the
    per-unit figures above and the measured iterations): (kernel, launches,
    bytes, flops, flop type, counts), bytes and flops summed over its launches."""
    mixed = precision_name == "mixed"
    launches = prof["launches"][stage]
    ncell = _rows(case, "p")
    precond = case.get("precond_p", "dct")
    modes = case["nx"] + (case["ny"] if case["dim"] == 3 else 0)
    if stage == "presolve_T":
        sweeps = prof.get("presolve_sweeps", 0)
        nbytes = ncell * (HELM_BYTES_PER_CELL * launches + HELM_BYTES_PER_CELL_SWEEP * sweeps)
        flops = ncell * sweeps * (4.0 * modes + DCT_THOMAS_FLOPS)
        return "k_helmholtz_dct", launches, nbytes, flops, "fp32", {"sweeps": sweeps, "cells": ncell}
    sysname = stage.split("_", 1)[1]
    if sysname == "p":
        its = prof["iters"]["p"]
        if precond == "dct":
            E = 4.0 if mixed else 8.0
            nbytes = ncell * (DCT_BYTES_PER_CELL_LAUNCH * launches + its * (DCT_BYTES_PER_CELL_SWEEP_BASE + 8.0 * E))
            flops = ncell * its * (4.0 * modes + DCT_THOMAS_FLOPS)
            kern = "k_poisson_dct<%s>" % ("float" if mixed else "double")
            return kern, launches, nbytes, flops, "fp32" if mixed else "fp64", {"sweeps": its, "cells": ncell}
        refs = stats["refinements"]["p"] * launches
        nbytes = ncell * (MG_BYTES_PER_CELL_IT[precision_name] * its + MG_BYTES_PER_CELL_REFINE * refs)
        flops = MG_FLOPS_PER_CELL_IT * ncell * its
        kern = "k_pcg_mg<%s>" % ("float" if mixed else "double")
        return kern, launches, nbytes, flops, "fp64", {"iterations": its, "cells": ncell}
    systems = [sysname]
    if stage == "solve_u" and prof["launches"].get("solve_v", 0) == 0:
        systems = list("uvw"[: case["dim"]])     # the joint momentum launch, counted under solve_u
    nbytes = flops = 0.0
    counts = {}
    for q in systems:
        rows = _rows(case, q)
        its = prof["iters"][q]
        jac = prof.get("jacobi", {}).get(q, 0)
        nbytes += rows * JAC_BYTES_ROW[precision_name] * jac
        if not mixed:
            flops += rows * JAC_FLOPS_ROW["fp64"] * jac
        if mixed:
            sweeps = stats["refinements"][q] * launches    # sweeps of the last step, for each launch
            # a launch with no sweeps, iterations or Jacobi sweeps found its system solved
            # (the T* pre-solve met the tolerance) and read nothing per row
            active = launches if (sweeps or its or jac) else 0
            nbytes += rows * (BCG_IR_BYTES_ROW * active + BCG_IR_BYTES_ROW_SWEEP * sweeps + BCG_IR_BYTES_ROW_IT * its)
            counts[q] = {"rows": rows, "jacobi_sweeps": jac, "inner_iterations": its, "sweeps": sweeps}
        else:
            nbytes += rows * BCG_BYTES_ROW_IT * its
            flops += rows * BCG_FLOPS_ROW_IT * its
            counts[q] = {"rows": rows, "jacobi_sweeps": jac, "iterations": its}
    return ("k_bicgstab_ir" if mixed else "k_bicgstab"), launches, nbytes, flops, "fp64", counts


def roofline(precision_name, m, case, steps, wname):
    """Roofline of the step's dominant kernel: the solver kernel with the most
    device time per step, its launches summed over the stages that run it.
    Achieved = its algorithmic bytes (or flops, when those take longer at
    their peak) over its device time (CUDA events on the case stream), against
    the measured HBM copy bandwidth or the FP32 / FP64 pipe's peak at the
    median SM clock sampled during the timed region."""
    prof = m["prof"]
    stage_ms = prof["ms"]
    peaks = measured_peaks()
    sm_mhz = m["clocks"].get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    hbm = peaks.get("hbm_gbs", 6687.1)
    kernels = {}
    for st in stage_ms:
        if not (st.startswith("solve_") or st == "presolve_T") or prof["launches"].get(st, 0) <= 0:
            continue
        kern, launches, nbytes, flops, ftype, counts = kernel_work(st, precision_name, case, prof, m["stats"])
        k = kernels.setdefault(kern, {"ms": 0.0, "launches": 0, "bytes": 0.0, "flops": 0.0, "flop_type": ftype,
                                      "stages": {}})
        k["ms"] += stage_ms[st]
        k["launches"] += launches
        k["bytes"] += nbytes
        k["flops"] += flops
        k["stages"][st] = counts
    top = max(kernels, key=lambda q: kernels[q]["ms"])
    detail = {}
    for kern, k in kernels.items():
        t = k["ms"] * 1e-3
        per_clk = FP32_FLOP_PER_CLK_PER_SM if k["flop_type"] == "fp32" else FP64_FLOP_PER_CLK_PER_SM
        fpeak = per_clk * NUM_SMS * sm_mhz * 1e6 / 1e12
        d = {"ms_per_step": k["ms"] / steps, "launch_ms": k["ms"] / max(k["launches"], 1),
             "bytes_per_launch": k["bytes"] / max(k["launches"], 1), "flops_per_launch": k["flops"] / max(k["launches"], 1),
             "flop_type": k["flop_type"], "hbm_frac": k["bytes"] / t / 1e9 / hbm,
             "alu_frac": k["flops"] / t / 1e12 / fpeak, "stages": k["stages"]}
        if k["bytes"] / (hbm * 1e9) >= k["flops"] / (fpeak * 1e12):
            ach = k["bytes"] / t / 1e9
            d.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                     peak_basis="measured HBM copy bandwidth (MEASURED_PEAKS.json)")
        else:
            ach = k["flops"] / t / 1e12
            d.update(bound="alu", achieved=ach, peak=fpeak, unit="TFLOP/s", frac=ach / fpeak,
                     peak_basis="%s pipe: %.0f flop/clk/SM x %d SMs x %.0f MHz median SM clock under load"
                                % (k["flop_type"].upper(), per_clk, NUM_SMS, sm_mhz))
        tr = kernel_traffic(kern, wname)
        d["traffic"] = tr[0] if tr else None
        detail[kern] = d
    out = dict(detail[top])
    out["kernel"] = top
    out["all_kernels"] = {k: {q: v for q, v in d.items() if q != "stages"} for k, d in detail.items() if k != top}
    # the assembly and pointwise kernels against the HBM roof by their algorithmic bytes
    point = {}
    for st, ms in stage_ms.items():
        if ms <= 0 or not (st.startswith("assemble_") or st == "lever"):
            continue
        if st == "lever":
            kern, per, rows = "k_lever", LEVER_BYTES_CELL, _rows(case, "p")
        elif st == "assemble_p":
            kern, per, rows = "k_poisson_rhs", RHS_BYTES_CELL, _rows(case, "p")
        else:
            q = st.split("_", 1)[1]
            mom = q in ("u", "v", "w")
            kern = ("k_assemble_momentum" if mom else "k_assemble_cells") + ("_df" if precision_name == "mixed" else "")
            per, rows = ASM_BYTES_ROW[precision_name], _rows(case, q)
        launches = max(prof["launches"].get(st, 1), 1)
        ach = rows * per * launches / (ms * 1e-3) / 1e9
        point[st] = {"kernel": kern, "bytes_per_launch": rows * per, "launch_ms": ms / launches, "achieved": ach,
                     "unit": "GB/s", "hbm_frac": ach / hbm}
    out["pointwise_kernels"] = point
    return out


def run_ours(args):
    import torch
    from paper_2303_10783_gb300 import solid
    rank, world, local = dist_env()
    dist = init_group(world)
    torch.cuda.set_device(local)
    solid.load()
    case = workload(args, rank)
    ncell = case["nx"] * case["ny"] * case["nz"]
    names = ["mixed", "fp64"] if args.precision == "both" else [args.precision]
    res = {}
    for name in names:
        m = measure(args, name, case, dist, local)
        ms_max = max_over_ranks(dist, m["ms"])
        total_cells = sum_over_ranks(dist, ncell * args.steps)
        m["value"] = total_cells / (ms_max * 1e-3)
        m["ms_max"] = ms_max
        if m["e2e"]:
            e2e_s = max_over_ranks(dist, m["e2e"]["seconds"])
            m["e2e_value"] = sum_over_ranks(dist, ncell * m["e2e"]["steps"]) / e2e_s
        res[name] = m
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    head = names[0]
    h = res[head]
    out = {
        "metric": "cell-steps/s", "value": h["value"], "unit": "cell-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h["ms_max"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if head == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": workload_name(args),
                   "cells": ncell, "precision": head, "tol_p": case["tol_p"],
                   "tol_t": case["tol_t"], "dt": case["dt"], "pressure_preconditioner": case.get("precond_p", "dct"),
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: each step streams ~0.5 GB of fields and DIA planes (L2 129 MB); "
                         "no flush"},
        "status": h["status"],
        "clocks": h["clocks"],
        "e2e": ({"value": h["e2e_value"], "unit": "cell-steps/s", "h2d_bytes_per_step": h["e2e"]["h2d"],
                 "d2h_bytes_per_step": h["e2e"]["d2h"], "steps": h["e2e"]["steps"],
                 "path": "per step: pinned host -> device buffer (side stream, during the previous step), "
                         "ss_set_fields(device) + ss_step(1) + ss_get_fields(device), device buffer -> pinned "
                         "host (side stream, during the next step)"} if h["e2e"] else None),
        "gpu_launches": h["prof"]["kernels"],
        "roofline": roofline(head, h, case, args.steps, workload_name(args)),
        "stage_ms_per_step": {k: v / args.steps for k, v in h["prof"]["ms"].items() if v > 0},
        "iters_per_step": {k: v / args.steps for k, v in h["prof"]["iters"].items()},
        "jacobi_sweeps_per_step": {k: v / args.steps for k, v in h["prof"]["jacobi"].items()},
        "refinements_last_step": dict(h["stats"]["refinements"]),
    }
    for name in names[1:]:
        m = res[name]
        out[name] = {"value": m["value"], "ms_per_step": m["ms_max"] / args.steps, "status": m["status"],
                     "dtype": "f64" if name == "fp64" else "f32+f64",
                     "e2e_value": m.get("e2e_value"), "gpu_launches": m["prof"]["kernels"],
                     "roofline": roofline(name, m, case, args.steps, workload_name(args)),
                     "stage_ms_per_step": {k: v / args.steps for k, v in m["prof"]["ms"].items() if v > 0},
                     "iters_per_step": {k: v / args.steps for k, v in m["prof"]["iters"].items()}}
    if "mixed" in res and "fp64" in res:
        out["mixed_vs_fp64"] = {"after_steps": args.warmup + args.steps, "bound": 1e-6, "bounded_fields": ["T", "C", "gl"],
                                "rel_linf": field_errors(res["mixed"]["fields"], res["fp64"]["fields"], case["dim"])}
    if world == 1 and not args.no_extras and args.workload == "box":
        for leg in (cavity_leg, ingot_leg, batched_leg, serving_leg):
            name, val = leg(args, local)
            out[name] = val
            torch.cuda.empty_cache()
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
        out["cpu_baseline"]["all_cores"] = cpu_all_cores(args)
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _time_case(case, precision, steps, warmup, local):
    """Warm up, then time `steps` steps of one case on its own stream (CUDA
    events on that stream); returns (ms, status, profile, stats, clocks)."""
    import torch
    from paper_2303_10783_gb300 import solid
    f = cases.initial_fields(case)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        c = solid.Case(case, precision=solid.SS_MIXED if precision == "mixed" else solid.SS_FP64, stream=stream)
        c.initialize(f["T"], f["C"])
        c.step(warmup)
        c.sync()
        c.get_profile()
        c.set_profiling(True)
        sampler = ClockSampler(local)
        stream.synchronize()
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.step(steps)
        e1.record(stream)
        stream.synchronize()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        status = c.sync(allow=(solid.SS_ENOTCONV,))
        prof = c.get_profile()
        stats = c.stats()
        c.close()
    return ms, solid.STATUS_NAMES.get(status, status), prof, stats, clocks


def cavity_leg(args, local):
    """The 2D cavity (0.10 x 0.06 m, 50 x 30 cells, FP64 plain scheme), 300 steps."""
    case = cases.cavity_2d()
    if args.precond:
        case["precond_p"] = args.precond
    ms, status, prof, _, clocks = _time_case(case, "fp64", 300, 3, local)
    n = case["nx"] * case["ny"]
    return "cavity", {"workload": "cavity_2d_50x30", "precision": "fp64", "steps": 300, "warmup": 3,
                      "value": n * 300 / (ms * 1e-3), "unit": "cell-steps/s", "ms_per_step": ms / 300,
                      "status": status, "gpu_launches": prof["kernels"], "clocks": clocks,
                      "stage_ms_per_step": {k: v / 300 for k, v in prof["ms"].items() if v > 0},
                      "iters_per_step": {k: v / 300 for k, v in prof["iters"].items()},
                      "note": "1500 cells: latency-bound, no roofline claimed"}


def ingot_leg(args, local):
    """The 3D ingot (0.2 x 0.1 x 0.1 m, 384 x 256 x 256 = 25.2 M cells, Fe-C-like
    alloy, bottom cooling), mixed and FP64, each with the roofline of its
    dominant solve: at this size the vectors do not fit L2."""
    out = {"workload": "ingot_3d_384x256x256", "cells": 384 * 256 * 256}
    steps, warmup = 5, 2
    for prec in ("mixed", "fp64"):
        case = cases.ingot_3d(seed=4)
        if args.precond:
            case["precond_p"] = args.precond
        ms, status, prof, stats, clocks = _time_case(case, prec, steps, warmup, local)
        m = {"prof": prof, "stats": stats, "clocks": clocks}
        out[prec] = {"value": out["cells"] * steps / (ms * 1e-3), "unit": "cell-steps/s", "ms_per_step": ms / steps,
                     "steps": steps, "warmup": warmup, "status": status, "gpu_launches": prof["kernels"],
                     "clocks": clocks, "pressure_solver": case.get("precond_p", "dct"),
                     "roofline": roofline(prec, m, case, steps, "ingot_3d_384x256x256"),
                     "stage_ms_per_step": {k: v / steps for k, v in prof["ms"].items() if v > 0},
                     "iters_per_step": {k: v / steps for k, v in prof["iters"].items()}}
    return "ingot", out


def batched_leg(args, local, steps=5, warmup=2):
    """64 independent cavities stepped side by side; see run_batched."""
    return "batched", _batched(args, local, steps, warmup, None)


def serving_leg(args, local):
    """A bounded sample of the request stream served under the 150 GB budget; see run_serving."""
    return "serving", _serving(args)


def _batched_one(args, local, steps, warmup, dist, packed):
    """64 independent cavities (2D and 3D, uneven sizes) stepped side by side,
    either one stream and one captured step graph per case (solver block cap
    autotuned) or packed (one launch per stage for all cases, team sizes and
    tile rows autotuned); the autotuner's trials run from a saved and restored
    state, outside the timed region. Returns the measured quantities
    (rank-local timing, max over ranks applied)."""
    import torch
    from paper_2303_10783_gb300 import solid
    from paper_2303_10783_gb300.batch import Batch
    rank = dist_env()[0]
    cs = cases.batch_cases(64, seed=2 + 100 * rank)
    if args.precond:
        cs = [dict(c, precond_p=args.precond) for c in cs]
    b = Batch(cs, precision=solid.SS_MIXED, packed=packed)
    sampler = ClockSampler(local)
    b.step(warmup)
    b.sync()
    best, trials = b.autotune()
    k0 = b.kernels()   # count launches of the timed region only
    barrier(dist)
    sampler.start()
    dt, _ = b.run(steps)
    clocks = sampler.stop()
    dt = max_over_ranks(dist, dt)
    total = sum_over_ranks(dist, b.cells * steps)
    status = b.sync()
    kernels = b.kernels() - (k0 if packed else 0)
    cells = b.cells
    teams = b.packed.teams() if packed else None
    b.close()
    torch.cuda.empty_cache()
    out = {"value": total / dt, "unit": "cell-steps/s", "ms_per_step": 1e3 * dt / steps,
           "status": solid.STATUS_NAMES.get(status, status), "graphs": True,
           "autotune_ms_per_step": {str(k): 1e3 * v for k, v in trials.items()},
           "clocks": clocks, "gpu_launches": kernels, "cells": cells, "cases": len(cs),
           "pressure_solver": cs[0].get("precond_p", "dct")}
    if packed:
        out.update(mode="packed", schedule={"gamma": best[0], "tile_rows": best[1]}, team_blocks=teams,
                   launches_per_step=kernels / steps)
    else:
        out.update(mode="streams", streams=len(cs), block_cap=best)
    return out


def _batched(args, local, steps, warmup, dist):
    """The batched workload, stepped both ways; the leg's value is the faster."""
    modes = {m: _batched_one(args, local, steps, warmup, dist, m == "packed") for m in ("packed", "streams")}
    best = max(modes, key=lambda m: modes[m]["value"])
    h = modes[best]
    return {"workload": "batched_64_cavities", "value": h["value"], "unit": "cell-steps/s",
            "ms_per_step": h["ms_per_step"], "mode": best, "steps": steps, "warmup": warmup, "cases": h["cases"],
            "cells": h["cells"], "precision": "mixed", "pressure_solver": h["pressure_solver"], "status": h["status"],
            "timing": "host wall clock over the steps of all cases (enqueue to the last stream synchronised)",
            "clocks": h["clocks"], "gpu_launches": h["gpu_launches"], "modes": modes}


def run_batched(args):
    """64 independent cavities stepped side by side (one stream each, graph-replayed steps)."""
    import torch
    rank, world, local = dist_env()
    dist = init_group(world)
    torch.cuda.set_device(local)
    r = _batched(args, local, args.steps, args.warmup, dist)
    if rank == 0:
        print(json.dumps({"metric": "cell-steps/s", "value": r["value"], "unit": "cell-steps/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                          "data": "synthetic", "status": r["status"],
                          "config": {k: r[k] for k in ("workload", "cases", "cells", "precision", "mode",
                                                        "pressure_solver")},
                          "modes": r["modes"],
                          "clocks": r["clocks"], "gpu_launches": r["gpu_launches"]}))
    return 0


def _serving(args):
    """The first `args.requests` requests of the seeded stream (Poisson arrivals
    at 20/s, grids 32^3..192^3), `args.request_steps` steps each, served under
    the 150 GB budget with continuous batching."""
    from paper_2303_10783_gb300.serve import Server
    reqs = cases.serving_requests(n=args.requests, steps=args.request_steps)
    srv = Server(budget_bytes=150 * 10 ** 9, chunk=10, block_cap=args.block_cap, precond=args.precond,
                 slots=args.slots)
    rep = srv.run(reqs)
    waits = sorted(p["admitted"] - p["arrival"] for p in rep["per_request"])
    return {"workload": "serving_requests", "value": rep["cell_steps_per_s"], "unit": "cell-steps/s",
            "requests": rep["requests"], "steps_per_request": args.request_steps, "arrival_rate_per_s": 20.0,
            "budget_bytes": rep["budget_bytes"],
            "sample": "first %d requests of the seeded stream (grids 32^3..192^3), %d steps each"
                      % (args.requests, args.request_steps),
            "latency": "per 100 steps, from admission to completion (service) and from arrival (total)",
            "slots": args.slots,
            "p50_ms_per_100_steps": rep["p50_ms_per_100_steps"], "p99_ms_per_100_steps": rep["p99_ms_per_100_steps"],
            "p50_total_ms_per_100_steps": rep["p50_total_ms_per_100_steps"],
            "p99_total_ms_per_100_steps": rep["p99_total_ms_per_100_steps"],
            "p50_queue_s": rep["p50_queue_s"], "p99_queue_s": rep["p99_queue_s"],
            "requests_that_waited": sum(1 for w in waits if w > 0.05),
            "max_active": rep["max_active"], "max_used_bytes": rep["max_used_bytes"], "wall_s": rep["wall_s"],
            "pressure_solver": srv.precond or reqs[0][1].get("precond_p", "dct")}


def run_serving(args):
    """A bounded sample of the request stream served under the 150 GB budget."""
    import torch
    torch.cuda.set_device(0)
    r = _serving(args)
    print(json.dumps({"metric": "cell-steps/s", "value": r["value"], "unit": "cell-steps/s",
                      "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                      "dtype": "f32+f64", "data": "synthetic",
                      "config": {k: r[k] for k in ("workload", "requests", "steps_per_request", "arrival_rate_per_s",
                                                    "budget_bytes", "sample", "pressure_solver")},
                      **{k: r[k] for k in ("p50_ms_per_100_steps", "p99_ms_per_100_steps", "p50_total_ms_per_100_steps",
                                           "p99_total_ms_per_100_steps", "slots", "p50_queue_s",
                                           "p99_queue_s", "requests_that_waited", "max_active", "max_used_bytes",
                                           "wall_s")}}))
    return 0


def main():
    args = parse()
    if args.workload == "ingot" and (args.nx, args.ny, args.nz) == (128, 96, 96):
        args.nx, args.ny, args.nz = 384, 256, 256     # the ingot's own size unless given
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
