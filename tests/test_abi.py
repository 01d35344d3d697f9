"""The C-ABI library loads and exports every entry point the header declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2609_39474_b300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "msclbm.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    from paper_2609_39474_b300 import _lib
    return _lib


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(msc_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L.lib, name), name
    assert sorted(L.exported_names()) == names  # the binding covers exactly the header


def test_header_compiles_as_plain_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "msclbm.h"\nint main(void){ msc_lattice_desc d = {2, 64, MSC_FP64, 1, 1};'
                   ' return (int)msc_workspace_bytes(&d) == 0; }\n')
    import subprocess
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-c", str(src), "-I", os.path.dirname(HEADER),
                        "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_workspace_and_scratch_sizes(L):
    ok = L.LatticeDesc(2, 64, L.MSC_FP64, 16, 16)
    n64 = L.lib.msc_workspace_bytes(ctypes.byref(ok))
    # five population arrays of 9 x 64^2 doubles dominate
    assert n64 > 5 * 9 * 64 * 64 * 8
    f32 = L.LatticeDesc(2, 64, L.MSC_FP32, 16, 16)
    assert L.lib.msc_workspace_bytes(ctypes.byref(f32)) < n64
    for bad in [L.LatticeDesc(2, 48, 0, 1, 1), L.LatticeDesc(2, 4, 0, 1, 1), L.LatticeDesc(4, 64, 0, 1, 1),
                L.LatticeDesc(2, 64, 7, 1, 1), L.LatticeDesc(2, 64, 0, 0, 1), L.LatticeDesc(2, 8192, 0, 1, 1),
                L.LatticeDesc(3, 512, 1, 1, 1), L.LatticeDesc(3, 256, 0, 1, 1)]:
        assert L.lib.msc_workspace_bytes(ctypes.byref(bad)) == 0
    assert L.lib.msc_workspace_bytes(ctypes.byref(L.LatticeDesc(3, 128, 1, 1, 1))) > 0
    assert L.lib.msc_stage_scratch_bytes(2, 256, L.MSC_FP32) > 0
    assert L.lib.msc_stage_scratch_bytes(2, 100, L.MSC_FP32) == 0


def test_argument_errors_need_no_device(L):
    ctx = ctypes.c_void_p()
    d = L.LatticeDesc(2, 64, L.MSC_FP64, 16, 16)
    assert L.lib.msc_create(ctypes.byref(ctx), ctypes.byref(d), None, 0, None) == L.MSC_ERR_ARG
    assert L.lib.msc_create(None, ctypes.byref(d), None, 0, None) == L.MSC_ERR_ARG
    assert L.lib.msc_sweep(2, 64, 0, 0.1, None, None, None, None, None, None, None, 0, None) == L.MSC_ERR_ARG
    assert L.lib.msc_shadow_solve(2, 64, 0, 0.1, 1 / 6, None, None, None, 0, None) == L.MSC_ERR_ARG
    assert L.lib.msc_march(None, 1) == L.MSC_ERR_ARG
    assert L.strerror(L.MSC_ERR_NONCONVERGED).startswith("physical step")
    assert L.strerror(99) == "unknown status"


def test_batch_tuning_struct_matches_header(L, tmp_path):
    # the ctypes mirror of msc_batch_tuning has the C layout (size and field offsets)
    src = tmp_path / "t.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "msclbm.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(msc_batch_tuning),'
                   ' offsetof(msc_batch_tuning, sweep_rows), offsetof(msc_batch_tuning, col_lines),'
                   ' offsetof(msc_batch_tuning, sweep_ctas_per_sm), offsetof(msc_batch_tuning, sweep_us),'
                   ' offsetof(msc_batch_tuning, colsolve_us)); return 0; }\n')
    import subprocess
    exe = tmp_path / "t"
    r = subprocess.run(["gcc", "-std=c99", str(src), "-I", os.path.dirname(HEADER), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    T = L.BatchTuning
    assert got == [ctypes.sizeof(T), T.sweep_rows.offset, T.col_lines.offset, T.sweep_ctas_per_sm.offset,
                   T.sweep_us.offset, T.colsolve_us.offset]
    assert L.MSC_BATCH_MAX == 64 and L.MSC_BATCH_CLASSES == 8


def test_batch_rejects_invalid_lists_without_a_device(L):
    # validation happens before any device work: an empty or NULL list sizes to 0 and create refuses it
    assert L.lib.msc_batch_workspace_bytes(None, 0) == 0
    assert L.lib.msc_batch_workspace_bytes(None, 3) == 0
    h = ctypes.c_void_p()
    assert L.lib.msc_batch_create(ctypes.byref(h), None, 0, None, 0, None) == L.MSC_ERR_ARG
    assert L.lib.msc_batch_march(None, None) == L.MSC_ERR_ARG
    assert L.lib.msc_batch_autotune(None, 1, None) == L.MSC_ERR_ARG


def test_adjoint_io_struct_matches_header(L, tmp_path):
    # the ctypes mirror of msc_adjoint_io has the C layout (size and the offsets around the padding)
    src = tmp_path / "t.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "msclbm.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu\\n", sizeof(msc_adjoint_io), offsetof(msc_adjoint_io, m_new),'
                   ' offsetof(msc_adjoint_io, abar_prev), offsetof(msc_adjoint_io, warm)); return 0; }\n')
    import subprocess
    exe = tmp_path / "t"
    r = subprocess.run(["gcc", "-std=c99", str(src), "-I", os.path.dirname(HEADER), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    S = L.AdjointIO
    assert got == [ctypes.sizeof(S), S.m_new.offset, S.abar_prev.offset, S.warm.offset]


def test_new_entry_points_reject_bad_arguments_without_a_device(L):
    fp64, fp32 = L.MSC_FP64, L.MSC_FP32
    # full-symbol scratch: twiddles (n complex) + 9 x (n/2 + 1) x n complex, each 256-byte aligned
    for n, prec, cb in ((64, fp64, 16), (1024, fp32, 8)):
        want = -(-n * cb // 256) * 256 + -(-9 * (n // 2 + 1) * n * cb // 256) * 256
        assert L.lib.msc_full_symbol_scratch_bytes(n, prec) == want
    for n, prec in ((2048, fp32), (100, fp64), (4, fp64), (64, L.MSC_FP16)):
        assert L.lib.msc_full_symbol_scratch_bytes(n, prec) == 0
    buf = ctypes.c_void_p(256)  # never dereferenced: every call below fails its host-side checks
    assert L.lib.msc_full_symbol_correct(2048, fp32, 0.1, 1.0, 1.0, buf, buf, buf, buf, 1 << 40, None) == L.MSC_ERR_ARG
    assert L.lib.msc_full_symbol_correct(64, fp64, 0.1, 2.0, 1.0, buf, buf, buf, buf, 1 << 40, None) == L.MSC_ERR_ARG
    assert L.lib.msc_full_symbol_correct(64, fp64, 0.0, 1.0, 1.0, buf, buf, buf, buf, 1 << 40, None) == L.MSC_ERR_ARG
    assert L.lib.msc_full_symbol_correct(64, fp64, 0.1, 1.0, 1.0, None, buf, buf, buf, 1 << 40, None) == L.MSC_ERR_ARG
    assert L.lib.msc_full_symbol_correct(64, fp64, 0.1, 1.0, 1.0, buf, buf, buf, buf, 16, None) == L.MSC_ERR_ARG
    assert L.lib.msc_full_symbol_correct(64, fp64, 0.1, 1.0, 1.0, buf, buf, buf, ctypes.c_void_p(264), 1 << 40,
                                         None) == L.MSC_ERR_ARG  # scratch not 256-byte aligned
    io = (L.AdjointIO * 1)()
    out = (L.AdjointStats * 1)()
    assert L.lib.msc_adjoint_steps(None, 1, io, buf, 1e-8, 10, out) == L.MSC_ERR_ARG
    assert L.lib.msc_adjoint_step(None, 1, buf, buf, None, buf, buf, None, buf, 1e-8, 10, None) == L.MSC_ERR_ARG
    assert L.lib.msc_copy_fields_async(None, buf) == L.MSC_ERR_ARG
