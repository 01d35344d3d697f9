"""ctypes binding of libmsclbm.so (argument marshalling only; every step runs in the CUDA library).

The names mirror include/msclbm.h.  Importing this module loads the in-tree shared object and
raises if it is missing: there is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# MSC_LIB_VARIANT=check selects the bounds-checked debug build (libmsclbm_check.so, built by
# build.build(variant="check")); the default is the optimised library
VARIANT = os.environ.get("MSC_LIB_VARIANT", "")
if VARIANT not in ("", "check"):
    raise ValueError(f"unknown MSC_LIB_VARIANT {VARIANT!r} (expected 'check' or unset)")
LIB_PATH = os.path.join(HERE, "libmsclbm_check.so" if VARIANT == "check" else "libmsclbm.so")

MSC_OK = 0
MSC_ERR_ARG = 1
MSC_ERR_NONCONVERGED = 2
MSC_ERR_NONFINITE = 3
MSC_ERR_TIMEOUT = 4
MSC_ERR_CUDA = 5
MSC_ERR_STATE = 6
MSC_FP64 = 0
MSC_FP32 = 1
MSC_FP16 = 2


class LatticeDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_steps", ctypes.c_int), ("hist_cap", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("dt", ctypes.c_double), ("eps", ctypes.c_double),
                ("kmax", ctypes.c_int), ("nmin", ctypes.c_int), ("corrector", ctypes.c_int),
                ("replay", ctypes.c_int), ("warm_order", ctypes.c_int), ("count_multiple", ctypes.c_int),
                ("force", ctypes.c_double * 3), ("omega", ctypes.c_double * 2)]


class Stats(ctypes.Structure):
    _fields_ = [("steps_done", ctypes.c_int64), ("inner_total", ctypes.c_int64),
                ("steps_in_call", ctypes.c_int32), ("last_iters", ctypes.c_int32),
                ("last_q", ctypes.c_int32), ("status", ctypes.c_int32), ("last_R", ctypes.c_double)]


MSC_BATCH_MAX = 64
MSC_BATCH_CLASSES = 8


class BatchTuning(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int), ("n", ctypes.c_int * MSC_BATCH_CLASSES),
                ("sweep_rows", ctypes.c_int * MSC_BATCH_CLASSES), ("fft_rows", ctypes.c_int * MSC_BATCH_CLASSES),
                ("col_lines", ctypes.c_int * MSC_BATCH_CLASSES), ("sweep_ctas_per_sm", ctypes.c_int),
                ("sweep_us", ctypes.c_float), ("rowfft_us", ctypes.c_float), ("colsolve_us", ctypes.c_float)]


class AdjointStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("residual", ctypes.c_double)]


class AdjointIO(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("m_new", ctypes.c_void_p), ("m_cur", ctypes.c_void_p),
                ("m_prev", ctypes.c_void_p), ("abar_new", ctypes.c_void_p), ("abar_cur", ctypes.c_void_p),
                ("abar_prev", ctypes.c_void_p), ("warm", ctypes.c_int)]


class MscError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_39474_b300.build`")
    return ctypes.CDLL(LIB_PATH)


lib = _load()

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_sz = ctypes.c_size_t
_SIG = {
    "msc_workspace_bytes": (_sz, [ctypes.POINTER(LatticeDesc)]),
    "msc_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(LatticeDesc), _vp, _sz, _vp]),
    "msc_destroy": (None, [_vp]),
    "msc_set_params": (_i, [_vp, ctypes.POINTER(Params)]),
    "msc_init_fields": (_i, [_vp, _vp, _vp, _i]),
    "msc_march": (_i, [_vp, _i]),
    "msc_march_stepwise": (_i, [_vp, _i]),
    "msc_explicit_march": (_i, [_vp, _i]),
    "msc_get_stats": (_i, [_vp, ctypes.POINTER(Stats)]),
    "msc_read_fields": (_i, [_vp, _vp, _vp, _i]),
    "msc_copy_fields_async": (_i, [_vp, _vp]),
    "msc_read_populations": (_i, [_vp, _vp, _i]),
    "msc_get_residual_history": (_i, [_vp, _vp, _i, ctypes.POINTER(_i)]),
    "msc_get_step_iters": (_i, [_vp, _vp, _i, ctypes.POINTER(_i)]),
    "msc_set_replay_counts": (_i, [_vp, _vp, _i]),
    "msc_save_state": (_i, [_vp, _vp, ctypes.POINTER(_sz)]),
    "msc_load_state": (_i, [_vp, _vp, _sz]),
    "msc_strerror": (ctypes.c_char_p, [_i]),
    "msc_stage_scratch_bytes": (_sz, [_i, _i, _i]),
    "msc_sweep": (_i, [_i, _i, _i, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "msc_bounds_check_report": (_i, [ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong), _i]),
    "msc_sweep_d3q19_pf": (_i, [_i, _i, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "msc_sweep_hpair": (_i, [_i, _i, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "msc_shadow_solve": (_i, [_i, _i, _i, _d, _d, _vp, _vp, _vp, _sz, _vp]),
    "msc_equilibrium": (_i, [_i, _i, _i, _vp, _vp, _vp, _vp]),
    "msc_sweep_d2q9_noalloc": (_i, [_i, _i, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "msc_sweep_trt": (_i, [_i, _i, _d, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "msc_full_symbol_scratch_bytes": (_sz, [_i, _i]),
    "msc_full_symbol_correct": (_i, [_i, _i, _d, _d, _d, _vp, _vp, _vp, _vp, _sz, _vp]),
    "msc_adjoint_step": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _d, _i, ctypes.POINTER(AdjointStats)]),
    "msc_adjoint_steps": (_i, [_vp, _i, ctypes.POINTER(AdjointIO), _vp, _d, _i, ctypes.POINTER(AdjointStats)]),
    "msc_adjoint_steps_stepwise": (_i, [_vp, _i, ctypes.POINTER(AdjointIO), _vp, _d, _i,
                                        ctypes.POINTER(AdjointStats)]),
    "msc_save_state_device": (_i, [_vp, _vp, ctypes.POINTER(_sz)]),
    "msc_selftest_conversions": (_i, [_i, _i, ctypes.c_ulonglong, ctypes.POINTER(_i)]),
    "msc_load_state_device": (_i, [_vp, _vp, _sz]),
    "msc_batch_workspace_bytes": (_sz, [ctypes.POINTER(_vp), _i]),
    "msc_batch_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _vp, _sz, _vp]),
    "msc_batch_destroy": (None, [_vp]),
    "msc_batch_march": (_i, [_vp, ctypes.POINTER(_i)]),
    "msc_batch_explicit_march": (_i, [_vp, ctypes.POINTER(_i)]),
    "msc_batch_autotune": (_i, [_vp, _i, ctypes.POINTER(BatchTuning)]),
    "msc_batch_get_tuning": (_i, [_vp, ctypes.POINTER(BatchTuning)]),
    "msc_batch_set_tuning": (_i, [_vp, ctypes.POINTER(BatchTuning)]),
    "msc_batch_time_stage": (_i, [_vp, _i, _i, ctypes.POINTER(ctypes.c_float)]),
}
for _name, (_res, _args) in _SIG.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def strerror(code: int) -> str:
    return lib.msc_strerror(int(code)).decode()


def check(code: int, where: str) -> None:
    if code != MSC_OK:
        raise MscError(code, where)


def exported_names():
    return list(_SIG)
