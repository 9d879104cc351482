"""bench.py's reference arm on the CPU: the FP64 oracle timed on a bounded sample, one JSON line
in the bench's metric and unit; ranks other than 0 exit without work."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    env.pop("RANK", None)
    if extra_env:
        env.update(extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                          timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_line_in_the_bench_unit():
    sys.path.insert(0, ROOT)
    import bench
    out = _run()
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["dtype"] == "f64" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert "E=16^3" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # the config names what was solved: the benchmark's recipe and cycle at E = 16^3
    c = d["config"]
    assert c["E"] == 16 ** 3 and c["n_dof"] == 1_442_897 and c["N"] == bench.NORDER
    assert c["sample_of"] == {"E": 32 ** 3, "n_dof": 11_390_625} and c["iterations"] >= 1
    for key in ("orders", "smoother", "k", "sided", "rtol"):
        assert c[key] == bench.config()[key]
    assert cb["config"] == c
    # value = DOFs of the sample / seconds per solve
    assert abs(d["value"] - 1_442_897 / (d["ms_per_step"] / 1e3) / 1e9) <= 1e-9 * d["value"] + 1e-15


def test_reference_arm_other_ranks_do_no_work():
    out = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.returncode == 0 and out.stdout.strip() == ""
