"""The allocation-free sweep (msc_sweep_d2q9_noalloc) against the allocating one (msc_sweep).

Callers that cannot allocate device memory (frameworks that own the device-memory budget,
bindings that only pass inputs and outputs, loops where an allocation would synchronise the
device) use msc_sweep_d2q9_noalloc, whose reduction scratch is a static device array shared by
all calls.  This file is collected last so that a failure here leaves every other test already
run; it passes both alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle.lattice import D2Q9
from workloads.fields import random_moments, random_populations

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(f=1e-14, pr=1e-13, ss=1e-12), "fp32": dict(f=1e-6, pr=1e-5, ss=1e-5)}


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,lift", [(64, True), (256, False), (1024, True)])
def test_noalloc_sweep_matches_allocating_sweep_twice(n, lift, precision):
    from paper_2609_39474_b300 import _lib as L
    from paper_2609_39474_b300 import lattice as PL
    T = PL.storage_dtype(precision)
    code = PL.precision_code(precision)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row: the shared static scratch must not leak state
        f = torch.as_tensor(random_populations(D2Q9.Q, (n, n), seed=30 + call, scale=1e-3)).to("cuda", T)
        h = torch.as_tensor(random_moments(2, (n, n), seed=40 + call, scale=1e-4)).to("cuda", T)
        dm = torch.as_tensor(random_moments(2, (n, n), seed=50 + call, scale=1e-4)).to("cuda", T) if lift else None
        a = 0.02 + 0.01 * call
        ref_f, ref_pr, ref_ss = PL.sweep(2, n, precision, a, f, h, dm)
        out_f = torch.empty_like(f)
        out_pr = torch.empty_like(ref_pr)
        out_ss = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.lib.msc_sweep_d2q9_noalloc(n, code, a, f.data_ptr(), dm.data_ptr() if lift else None, h.data_ptr(),
                                          out_f.data_ptr(), out_pr.data_ptr(), out_ss.data_ptr(), stream)
        assert rc == L.MSC_OK, L.strerror(rc)
        torch.cuda.synchronize()
        tol = TOL[precision]
        assert _rel(out_f, ref_f) < tol["f"]
        assert _rel(out_pr, ref_pr) < tol["pr"]
        assert abs(out_ss.item() / ref_ss.item() - 1) < tol["ss"]


def test_noalloc_argument_validation():
    # sizes and storage types outside the documented limits are rejected before any launch (the
    # bound of the static scratch itself is a compile-time check in the library)
    from paper_2609_39474_b300 import _lib as L
    p = [ctypes.c_void_p(16), None, ctypes.c_void_p(16), ctypes.c_void_p(32), ctypes.c_void_p(64),
         ctypes.c_void_p(128), None]
    for n, prec in ((8192, L.MSC_FP32), (4096, L.MSC_FP64), (100, L.MSC_FP32), (4, L.MSC_FP64), (64, L.MSC_FP16)):
        assert L.lib.msc_sweep_d2q9_noalloc(n, prec, 0.01, *p) == L.MSC_ERR_ARG, (n, prec)
