"""Host-side logic of bench.py that needs no GPU."""
import json
import shutil
from pathlib import Path

import bench

ROOT = Path(__file__).resolve().parents[1]


def test_source_digest_tracks_the_kernel_sources(tmp_path):
    src = ROOT / "paper_1107_5300_gb300" / "csrc"
    copy = tmp_path / "csrc"
    shutil.copytree(src, copy, ignore=shutil.ignore_patterns("*.o", "*.so"))
    d0 = bench.kernel_sources_digest(copy)
    assert d0 == bench.kernel_sources_digest(src) == bench.kernel_sources_digest()
    f = copy / "rgf_tc.cuh"
    f.write_bytes(f.read_bytes() + b"\n")
    assert bench.kernel_sources_digest(copy) != d0


def test_traffic_record_names_its_sources():
    rec = json.loads((ROOT / "profiles" / "traffic.json").read_text())
    assert len(rec["_sources_sha256"]) == 64
    assert all(isinstance(v, int) and v > 0 for k, v in rec.items() if not k.startswith("_"))


def _run_bench(args, env=None):
    import os
    import subprocess
    import sys
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, str(ROOT / "bench.py"), *args], capture_output=True,
                          text=True, timeout=300, env=e, cwd=str(ROOT))


def test_reference_arm_prints_one_contract_line():
    # the oracle on a 2-cell sample of the bench workload (a few seconds)
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-cells", "2"])
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["value"] > 0 and out["higher_is_better"] is True
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"]["value"] == out["value"] and out["e2e"]["h2d_bytes_per_step"] == 0
    assert out["config"]["workload"] == "agnr245_L4000_anderson"


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-cells", "2"],
                   env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_flop_counts_per_slice_step():
    # N = 245 (M = 490): the column recursion's count and the unit-cell count
    # (LU + boundary solve + strip), 5.63e8
    assert abs(bench.flops_per_cell(245) - 1.18e8) < 0.01e8
    assert abs(bench.cell_slicing_flops_per_step(245) - 5.628e8) < 0.001e8
    # N = 101 (M = 202): 3.9e7 by the unit-cell count
    assert abs(bench.cell_slicing_flops_per_step(101) - 3.9e7) < 0.1e7
