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
