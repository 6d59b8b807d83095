"""The benchmark's reference arm (the float64 oracle on host cores) prints one
JSON line with the contract's keys; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "c1",
                          "--steps", "2", "--warmup", "0", "--ref-side", "0.5"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["unit"] == "particles/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the step time and the rate describe the same sample
    per_step = float(d["cpu_baseline"]["sample"].split("(")[1].split(" ")[0])
    assert abs(per_step / (d["ms_per_step"] * 1e-3) - d["value"]) <= 1e-6 * d["value"]
    assert "workload" in d["config"]


def test_per_group_sample_selection():
    """The per-group comparison's sample: seeded, ascending, distinct, the
    largest tenth included, and all groups when the sample asks for more."""
    import importlib.util
    import numpy as np
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    sizes = np.random.default_rng(3).integers(10, 100000, 5000)
    a, k = bench.sample_groups(sizes, 200, 7)
    b, _ = bench.sample_groups(sizes, 200, 7)
    assert np.array_equal(a, b) and len(a) == 200 and k == 20
    assert np.all(np.diff(a) > 0)
    assert set(np.argsort(sizes)[::-1][:20]) <= set(a.tolist())
    c, _ = bench.sample_groups(sizes, 10000, 7)
    assert np.array_equal(c, np.arange(5000))


def test_stream_chunk_plan():
    """The streamed batching benchmark's plan: chunks of whole consecutive
    groups within the particle cap (or one oversized group alone), tasks
    tiling each chunk, every group exactly once."""
    import importlib.util
    import numpy as np
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    sizes = np.random.default_rng(5).integers(20, 5000, 3000)
    sizes[100] = 50_000  # larger than a chunk
    chunks, tasks, tchunk = bench.plan_chunks(sizes, 40_000, task_particles=7000)
    assert chunks[0][0] == 0 and chunks[-1][1] == len(sizes)
    for (a, b), (c, d) in zip(chunks, chunks[1:]):
        assert b == c
    for a, b in chunks:
        assert sizes[a:b].sum() <= 40_000 or b - a == 1
    covered = []
    for (a, b), k in zip(tasks, tchunk):
        assert chunks[k][0] <= a < b <= chunks[k][1]
        covered += list(range(a, b))
    assert covered == list(range(len(sizes)))
    assert bench.plan_chunks(np.zeros(0, np.int64), 10) == ([], [], [])


def test_shipped_tuning_record_equals_the_library_defaults():
    """The library starts with the table the tuner's committed record
    (coordinate descent on the 134M workload on a GB300) chose; every trial
    kept the result unchanged."""
    import json
    pytest = __import__("pytest")
    torch = pytest.importorskip("torch")  # noqa: F841 (the binding imports torch)
    from paper_1110_4372_gb300 import rsgpu
    rec = json.load(open(rsgpu.TUNING_FILE))
    assert rec["tuned"] == rsgpu.rs_tuning_default()
    assert all(t.get("same_result", True) for t in rec["trials"])
    assert rec["tuned_ms"] <= min(t["ms"] for t in rec["trials"]) * 1.005


def test_tuner_descent():
    """The tuner's coordinate descent: keeps a candidate only when it beats
    the best by the margin, measures no table twice in a sweep, ends after a
    sweep that keeps nothing, and stops when a candidate changes the result."""
    import pytest
    from paper_1110_4372_gb300 import tune
    space = {"a": [1, 2, 3], "b": [10, 20], "c": [0, 1]}
    cost = {("a", 1): 0.0, ("a", 2): -5.0, ("a", 3): -4.0, ("b", 10): 0.0, ("b", 20): -0.2,
            ("c", 0): 0.0, ("c", 1): -2.0}
    seen = []

    def measure(t):
        seen.append(dict(t))
        return 100.0 + sum(cost[(k, v)] for k, v in t.items()), True

    best, best_ms, base_ms, trials = tune.descend({"a": 1, "b": 10, "c": 0}, space, measure, sweeps=3,
                                                  log=lambda m: None)
    # b=20 saves 0.2 ms of ~95: inside the 0.5% margin, so not kept
    assert best == {"a": 2, "b": 10, "c": 1} and best_ms == 93.0 and base_ms == 100.0
    assert len(trials) == len(seen)
    # sweep 0 moves a and c, sweep 1 keeps nothing and ends the descent
    assert len(seen) == 1 + 4 + 4
    with pytest.raises(RuntimeError, match="changed the result"):
        tune.descend({"a": 1, "b": 10, "c": 0}, space, lambda t: (100.0, t["b"] != 20), log=lambda m: None)
