"""bench.py on the CPU: the reference arm's one JSON line (the FP64 oracle timed on the host cores, no
device bytes, printed by rank 0 only), the candidate selection, and the repo arm's contract line built
from a stub result (strict JSON, bounded length, null matched value when the gate fails)."""
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
    # e2e: the oracle's time to solution in ms, the unit of the GPU arm's e2e
    assert d["e2e"]["unit"] == "ms" and d["e2e"]["higher_is_better"] is False and d["e2e"]["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["time_to_solution_ms"]
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
    best, best1, ok, conv = sel(cands, 2e-9)    # matched gate 6e-9: S = 64 is the fastest passing
    assert ok and conv and best["S"] == 64 and best1["S"] == 8
    best, best1, ok, conv = sel(cands, 1e-10)   # nothing passes: the most accurate converged stands in
    assert not ok and conv and best["S"] == 128 and best1["S"] == 8
    best, best1, ok, conv = sel([c(8, 1.0, 9e-7, 0.02)], 1e-6)
    assert ok and conv and best["S"] == 8 and best1 is None
    # nothing converged: nothing is chosen (a failed candidate is never timed as a result)
    inf = float("inf")
    best, best1, ok, conv = sel([c(8, 1.0, inf, inf, ok=False), c(16, 2.0, inf, inf, ok=False)], 1e-6)
    assert best is None and best1 is None and not ok and not conv


def _stub_result(matched):
    inf = float("inf")
    cand = dict(S=512, eps=1e-10, nmin=2, ms=90.0, err=1.6e-10, rel=8e-6, ok=True, inner=2048)
    return {
        "candidate": cand, "candidate_1pct": dict(cand, S=8), "t_end": 157286,
        "s_wall_matched": 22.0 if matched else None, "s_wall_timed": 22.0, "s_wall_1pct": 1400.0,
        "matched_gate_passed": matched, "converged": True, "ms_per_step": 90.0, "t_explicit_ms": 1990.0,
        "e_msc": 1.6e-10, "e_explicit": 2.8e-11, "rms_ref": 1.94e-5, "inner_mlups": 2.4e4,
        "inner_iters_per_step": 4.0,
        "e2e": {"t_msc_ms": 93.0, "t_explicit_ms": 1995.0, "s_wall": 21.4, "h2d_bytes_per_step": 25165824,
                "d2h_bytes_per_step": 25165824},
        "roofline": {"bound": "hbm", "achieved": 5300.0, "peak": 6470.2, "unit": "GB/s", "frac": 0.82,
                     "traffic": None, "kernel": "k_sweep2<float>", "n": 4096, "ms_per_launch": 0.38,
                     "peak_source": "measured hbm_gbs", "bytes_per_site": 120},
        "clocks": {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": []}, "launches": 12345,
        # the large and non-finite parts that stay out of the line
        "candidates": [dict(cand, err=inf, rel=inf, ok=False)] * 40, "secondary": [{"x": inf}] * 3,
        "batch": {"per_instance": [{"rel": inf}] * 48}, "fp16": None, "adjoint": None, "offdesign": None,
    }


class _Args:
    n, steps, warmup = 1024, 20, 5


def test_repo_line_is_strict_bounded_json():
    B = _bench()
    cpu = {"value": 44.7, "unit": "x", "cores": 16, "kind": "oracle", "sample": "1 MSC step", "t": float("inf")}
    for matched in (True, False):
        txt = B.contract_line(_stub_result(matched), cpu, _Args(), 1)
        assert "\n" not in txt and len(txt) < 2048, len(txt)
        d = json.loads(txt, parse_constant=lambda s: (_ for _ in ()).throw(ValueError(s)))  # rejects Infinity/NaN
        for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                  "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "roofline", "cpu_baseline", "clocks",
                  "gpu_launches", "matched_gate_passed", "converged", "s_wall_1pct"):
            assert k in d, k
        for k in ("warm_order", "count_multiple", "S", "eps", "dt", "workload"):
            assert k in d["config"], k
        assert d["e2e"]["unit"] == "ms" and d["e2e"]["value"] == 93.0
        assert d["cpu_baseline"]["t"] is None
        for k in ("candidates", "secondary", "batch", "fp16", "adjoint", "offdesign"):
            assert k not in d, k
        if matched:
            assert d["value"] == 22.0 and "value_reason" not in d
        else:
            assert d["value"] is None and d["value_reason"] and d["s_wall_timed"] == 22.0


def test_details_are_strict_json(tmp_path):
    B = _bench()
    path = tmp_path / "details.json"
    B.write_details(_stub_result(False), str(path))
    d = json.loads(path.read_text(), parse_constant=lambda s: (_ for _ in ()).throw(ValueError(s)))
    assert len(d["candidates"]) == 40 and d["candidates"][0]["err"] is None
