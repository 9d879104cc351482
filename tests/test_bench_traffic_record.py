"""bench.py's DRAM-traffic record for the roofline object: per operator variant, reported only
while the hashed kernel sources are unchanged, never for a variant that was not captured."""
import json
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record():
    return json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))


def test_record_is_consistent():
    rec = _record()
    assert rec["alg_bytes_per_step"] == 4 * (6 * 32 ** 3 * 512 + 7 * (32 * 7 + 1) ** 3)
    assert rec["variants"]
    for v, entry in rec["variants"].items():
        kern = entry["kernels"]
        total = sum(k["dram_read"] + k["dram_write"] for k in kern.values())
        assert total == entry["traffic_bytes_per_step"], v
        # the reads are the algorithmic count (G + 7n); the writes come on top
        reads = sum(k["dram_read"] for k in kern.values())
        assert abs(reads - rec["alg_bytes_per_step"]) < 0.01 * rec["alg_bytes_per_step"], v
        assert "--clock-control none" in entry["command"] and "python bench.py" in entry["command"]


def test_lookup_by_variant_and_source_hash(tmp_path, monkeypatch):
    rec = _record()
    v = next(iter(rec["variants"]))
    fresh = bench.recorded_traffic(int(v))
    assert fresh in (None, rec["variants"][v]["traffic_bytes_per_step"])   # None once a source changes
    assert bench.recorded_traffic(999) is None                             # never captured
    # a copy of the tree with one hashed source edited: the record no longer applies
    root = tmp_path / "tree"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "profiles", "roofline_traffic.json"), root / "profiles")
    for f in rec["source_files"]:
        (root / f).parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), root / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.recorded_traffic(int(v)) == fresh
    with open(root / rec["source_files"][-1], "a") as fh:
        fh.write("\n// edited\n")
    assert bench.recorded_traffic(int(v)) is None
