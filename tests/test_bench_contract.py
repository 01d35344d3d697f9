"""The reference arm of bench.py on the CPU: one JSON line with the keys the benchmark contract
names (the FP64 oracle timed on the host cores, no device bytes), printed by rank 0 only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "64", "--steps", "1",
        "--warmup", "0"]


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run(ARGS, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_line_keys():
    p = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["dtype"] == "f64" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"] and d["config"]["N"] == 64


def test_reference_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_candidate_selection_gates_and_fallback():
    sel = _bench().select_candidates
    c = lambda S, ms, err, rel, ok=True: dict(S=S, ms=ms, err=err, rel=rel, ok=ok)
    cands = [c(8, 1.0, 9e-7, 0.009), c(16, 2.0, 2e-7, 0.002), c(64, 8.0, 4e-9, 5e-5), c(128, 16.0, 2e-9, 3e-5),
             c(4, 0.5, 1e-9, 1e-6, ok=False)]
    best, best1, ok = sel(cands, 2e-9)          # matched gate 6e-9: S = 64 is the fastest passing
    assert ok and best["S"] == 64 and best1["S"] == 8
    best, best1, ok = sel(cands, 1e-10)         # nothing passes: the most accurate converged stands in
    assert not ok and best["S"] == 128 and best1["S"] == 8
    best, best1, ok = sel([c(8, 1.0, 9e-7, 0.02)], 1e-6)
    assert ok and best["S"] == 8 and best1 is None
