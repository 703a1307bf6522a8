"""The multi-GPU path of bench.py is replicas only: every rank steps its own
case and the ranks meet only to bracket the timed region and to reduce the
timings. This checks that host logic with two gloo ranks on the CPU."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_env()
    dist = bench.init_group(w)
    bench.barrier(dist)
    args = type("A", (), {"nx": 16, "ny": 12, "nz": 8})()
    case = bench.workload(args, r)
    res = {"rank": r, "world": w, "max": bench.max_over_ranks(dist, float(r + 1)),
           "sum": bench.sum_over_ranks(dist, 10.0 * (r + 1)), "seed": case["seed"],
           "cells": case["nx"] * case["ny"] * case["nz"]}
    bench.barrier(dist)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks_reduce_timings_and_own_distinct_replicas(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for r in res:
        assert r["world"] == 2 and r["max"] == 2.0 and r["sum"] == 30.0
    # each rank owns an independent replica of the workload (its own seed, same size)
    assert res[0]["seed"] != res[1]["seed"] and res[0]["cells"] == res[1]["cells"]
