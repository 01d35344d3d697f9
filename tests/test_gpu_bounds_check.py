"""The small-lattice parity tests rerun against the bounds-checked debug build (libmsclbm_check.so,
compiled with -DMSC_BOUNDS_CHECK): every index check of the sweep strips, tiles and halos and of the
shared-memory transforms is compiled in, a failing check skips its access and is counted, nothing
traps.  The tests run in a child pytest process (the library variant is chosen when the binding is
first imported) and pass only if the parity tests pass and the library counted no failed check.

The cases cover the smallest lattices, where the 32-column warp strips and the 32 x 8 tiles wrap onto
themselves (n = 8, 16), a ragged last strip (n = 64), both storage precisions, the lift, FP16
storage, the general TRT sweep, the shadow solve, the march, the explicit step and the batch."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    *[f"tests/test_gpu_stages.py::test_sweep_matches_oracle[{d}-{n}-{l}-{p}]"
      for d, n in ((2, 8), (2, 16), (2, 64), (3, 8), (3, 16)) for l in ("nolift", "lift") for p in ("fp64", "fp32")],
    *[f"tests/test_gpu_stages.py::test_shadow_solve_matches_oracle[{d}-{n}-{p}]"
      for d, n in ((2, 8), (2, 16), (2, 64), (3, 8), (3, 16)) for p in ("fp64", "fp32")],
    "tests/test_gpu_stages.py::test_sweep_hpair_matches_oracle[8-True]",
    "tests/test_gpu_stages.py::test_sweep_hpair_matches_oracle[64-False]",
    "tests/test_gpu_stages.py::test_equilibrium_matches_oracle[2-16-fp64]",
    "tests/test_gpu_stages.py::test_equilibrium_matches_oracle[3-8-fp32]",
    "tests/test_gpu_fp16.py::test_fp16_sweep_within_one_ulp_of_the_oracle[8-lift]",
    "tests/test_gpu_fp16.py::test_fp16_sweep_within_one_ulp_of_the_oracle[64-nolift]",
    "tests/test_gpu_trt.py::test_trt_sweep_matches_oracle[0.12-0.25-8-lift-fp64]",
    "tests/test_gpu_trt.py::test_trt_sweep_matches_oracle[0.12-0.25-64-nolift-fp32]",
    "tests/test_gpu_march.py::test_picard_replay_parity_fp64",
    "tests/test_gpu_march.py::test_3d_tgv_fp64_replay_parity",
    "tests/test_gpu_march.py::test_fp32_storage_against_fp64_oracle[2-64-10]",
    "tests/test_gpu_march.py::test_fp32_storage_against_fp64_oracle[3-16-4]",
    "tests/test_gpu_march.py::test_explicit_march_matches_oracle[fp32]",
    "tests/test_gpu_march.py::test_explicit_march_3d",
    "tests/test_gpu_march.py::test_stepwise_march_equals_graph_march[2-64-fp64-None-True-1e-09]",
    "tests/test_gpu_march.py::test_stepwise_march_equals_graph_march[3-16-fp32-4-True-1e-09]",
    "tests/test_gpu_batch.py::test_batch_fp64_replay_matches_oracle",
]


def test_small_lattice_parity_under_the_bounds_checked_build(tmp_path):
    lib = os.path.join(ROOT, "paper_2609_39474_b300", "libmsclbm_check.so")
    assert os.path.exists(lib), "build the checked library first: python -m paper_2609_39474_b300.build --check"
    report = tmp_path / "bounds.json"
    env = dict(os.environ, MSC_LIB_VARIANT="check", MSC_BOUNDS_REPORT=str(report))
    p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *CASES], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert p.returncode == 0, p.stdout[-3000:] + p.stderr[-2000:]
    d = json.loads(report.read_text())
    assert d["lib"].endswith("libmsclbm_check.so") and d["rc"] == 0
    assert d["count"] == 0, f"{d['count']} failed index checks, first: site {d['first'] >> 40}, index {d['first'] & ((1 << 40) - 1)}"
