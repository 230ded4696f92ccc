"""bench.py --impl reference (the oracle as the reference arm), on CPU: one JSON line with
every key of the line format, the reference's own end-to-end entry, and silence on ranks
other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return p.stdout


def test_reference_line():
    out = _run({})
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("laplace3d_128")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["setup_ms"] > 0 and cb["solve_ms"] > 0 and cb["iterations"] == d["iterations"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_are_silent():
    out = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert not [l for l in out.splitlines() if l.startswith("{")]


def test_all_cores_oracle_baseline():
    """The all-core oracle leg: spawned workers, one independent setup + solve each, timed
    from the first start to the last finish."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench

    d = bench.run_cpu_baseline_allcores(side=20, max_workers=2)
    assert d["kind"] == "oracle" and d["unit"] == "solves/s"
    assert 1 <= d["cores"] <= 2 and d["value"] > 0 and "20^3" in d["sample"]
