"""Host logic of bench.py that needs no GPU: workload names, the bounded
oracle samples and the lookup of committed DRAM traffic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(kind, nx, ny, nz):
    return type("A", (), {"workload": kind, "nx": nx, "ny": ny, "nz": nz})()


def test_workload_name_follows_sizes():
    assert bench.workload_name(_args("box", 128, 96, 96)) == "box_3d_128x96x96"
    assert bench.workload_name(_args("ingot", 384, 256, 256)) == "ingot_3d_384x256x256"
    assert bench.workload_name(_args("box", 64, 48, 32)) == "box_3d_64x48x32"


def test_oracle_samples_are_bounded_and_keep_the_case():
    for kind, n in (("box", (128, 96, 96)), ("ingot", (384, 256, 256))):
        a = _args(kind, *n)
        for budget in (bench.CPU_BASELINE_MAX_CELLS, bench.REFERENCE_MAX_CELLS):
            case, k = bench.sample_case(a, budget)
            cells = case["nx"] * case["ny"] * case["nz"]
            assert cells <= budget
            # k is the smallest reduction that fits
            if k > 1:
                prev = max(n[0] // (k - 1), 2) * max(n[1] // (k - 1), 2) * max(n[2] // (k - 1), 2)
                assert prev > budget
            assert (case["nx"], case["ny"], case["nz"]) == tuple(max(v // k, 2) for v in n)
            # the sample is the workload's own case (domain and cooling), only coarser
            full = bench.workload(a)
            assert case["lx"] == full["lx"] and case["ly"] == full["ly"] and case["lz"] == full["lz"]
            assert case["dt"] == full["dt"]
    # the box workload's one-step CPU baseline runs at full size
    assert bench.sample_case(_args("box", 128, 96, 96), bench.CPU_BASELINE_MAX_CELLS)[1] == 1


def test_traffic_record_is_keyed_by_workload():
    """Every record of the committed DRAM traffic is looked up by its kernel,
    source hash and workload; a record taken on other sources or another
    workload is not reported."""
    recs = []
    for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
        if line.strip() and not line.startswith("#"):
            kern = line.split()[0]
            recs.append((kern, dict(f.split("=", 1) for f in line.split()[1:])))
    assert recs
    for kern, rec in recs:
        got = bench.kernel_traffic(kern, rec["workload"])
        if rec["sha256"] == bench.kernel_source_sha(kern):
            assert got is not None and got[0] == float(rec["bytes_per_launch"])
        else:
            assert got is None
        assert bench.kernel_traffic(kern, "some_other_workload") is None


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the host and prints one
    JSON line with the contract's keys (run here on a tiny box)."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--nx", "16",
                        "--ny", "12", "--nz", "12", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "cell-steps/s" and d["unit"] == "cell-steps/s"
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "box_3d_16x12x12"


def test_all_core_oracle_timing_runs_one_replica_per_core():
    """The all-core oracle leg spawns one single-threaded replica per host core
    and reports their combined throughput with the core count."""
    d = bench.cpu_all_cores(_args("box", 16, 12, 12), delay=4.0)
    assert d["cores"] == (os.cpu_count() or 1) and d["kind"] == "oracle" and d["value"] > 0
    assert "8x6x6" in d["sample"]
