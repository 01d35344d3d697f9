"""Python front end of the MSC-LBM library: torch tensors in, C ABI calls out.

PyTorch provides device memory (the context workspace and field buffers) and the CUDA stream;
every computation runs in libmsclbm.so.  Field layout: p_hat[(z,) y, x], u[alpha, (z,) y, x],
populations f[k, (z,) y, x], float64 on the host side of the API.
"""
import ctypes

import numpy as np
import torch

from . import _lib as L

# precision -> (code, population storage dtype, working-field dtype)
_DT = {"fp64": (L.MSC_FP64, torch.float64, torch.float64), "fp32": (L.MSC_FP32, torch.float32, torch.float32),
       "fp16": (L.MSC_FP16, torch.float16, torch.float32)}


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def precision_code(precision: str) -> int:
    return _DT[precision][0]


def storage_dtype(precision: str) -> torch.dtype:
    """dtype of stored populations (FP16 storage: float16)."""
    return _DT[precision][1]


def field_dtype(precision: str) -> torch.dtype:
    """dtype of the working fields h, P r, dm (float32 for FP16 population storage)."""
    return _DT[precision][2]


class MscLattice:
    """One periodic D2Q9 (dim=2) or D3Q19 (dim=3) lattice with its device-resident march state."""

    def __init__(self, dim: int, n: int, precision: str = "fp64", max_steps: int = 1 << 16,
                 hist_cap: int = 1 << 16, device: str = "cuda", stream=None):
        self.dim, self.n, self.precision = dim, n, precision
        self.Q = 9 if dim == 2 else 19
        self.sites = n ** dim
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.desc = L.LatticeDesc(dim, n, precision_code(precision), max_steps, hist_cap)
        nbytes = L.lib.msc_workspace_bytes(ctypes.byref(self.desc))
        if nbytes == 0:
            raise ValueError(f"unsupported lattice dim={dim} n={n} precision={precision}")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._ctx = ctypes.c_void_p()
        L.check(L.lib.msc_create(ctypes.byref(self._ctx), ctypes.byref(self.desc), _ptr(self.workspace),
                                 nbytes, self.stream.cuda_stream), "msc_create")
        self.max_steps, self.hist_cap = max_steps, hist_cap

    @property
    def grid(self):
        return (self.n,) * self.dim

    def close(self):
        if self._ctx:
            L.lib.msc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, dt: float, eps: float = 1e-8, nu: float = 1.0 / 6.0, kmax: int = 300,
                   nmin=None, corrector: bool = True, replay: bool = False, warm_order: int = 0,
                   count_multiple: int = 0, force=None, omega=None):
        """warm_order: 3 cubic (Section 3.1), 2 linear, 1 none; 0 = 3 for FP64, FP32: 2 (D2Q9) / 1 (D3Q19).
        count_multiple: accepted inner counts are multiples of it (1 = Algorithm 1, 2 = sweeps in pairs);
        0 = 2 for FP32 D2Q9, else 1.  force: uniform body force (d components, default zero).
        omega: (omega+, omega-) of the general TRT collision (D2Q9; default the operating point)."""
        if nmin is None:
            nmin = 2 if self.dim == 2 else 1
        fv = [0.0, 0.0, 0.0]
        if force is not None:
            for al, v in enumerate(force):
                fv[al] = float(v)
        om = [0.0, 0.0] if omega is None else [float(omega[0]), float(omega[1])]
        p = L.Params(nu, dt, eps, kmax, nmin, int(corrector), int(replay), int(warm_order), int(count_multiple),
                     (ctypes.c_double * 3)(*fv), (ctypes.c_double * 2)(*om))
        L.check(L.lib.msc_set_params(self._ctx, ctypes.byref(p)), "msc_set_params")

    def init_fields(self, p_hat, u):
        """f^0 = f_eq(p_hat, u); accepts numpy arrays or torch tensors (host or device), float64."""
        p_t = torch.as_tensor(np.asarray(p_hat) if not torch.is_tensor(p_hat) else p_hat, dtype=torch.float64)
        u_t = torch.as_tensor(np.asarray(u) if not torch.is_tensor(u) else u, dtype=torch.float64)
        if tuple(p_t.shape) != self.grid or tuple(u_t.shape) != (self.dim,) + self.grid:
            raise ValueError("field shapes do not match the lattice")
        on_dev = int(p_t.is_cuda)
        if on_dev != int(u_t.is_cuda):
            raise ValueError("p_hat and u must be on the same side")
        p_t, u_t = p_t.contiguous(), u_t.contiguous()
        self._init_keep = (p_t, u_t)  # keep the sources alive until the async copy has run
        L.check(L.lib.msc_init_fields(self._ctx, _ptr(p_t), _ptr(u_t), on_dev), "msc_init_fields")

    def march(self, n_steps: int):
        L.check(L.lib.msc_march(self._ctx, int(n_steps)), "msc_march")

    def march_stepwise(self, n_steps: int):
        """Host-driven march (same kernels, one launch each); for profiling and debugging."""
        L.check(L.lib.msc_march_stepwise(self._ctx, int(n_steps)), "msc_march_stepwise")

    def explicit_march(self, n_steps: int):
        L.check(L.lib.msc_explicit_march(self._ctx, int(n_steps)), "msc_explicit_march")

    def stats(self) -> dict:
        s = L.Stats()
        L.check(L.lib.msc_get_stats(self._ctx, ctypes.byref(s)), "msc_get_stats")
        return {k: getattr(s, k) for k, _ in L.Stats._fields_}

    def fields(self, on_device: bool = True, out=None):
        """(p_hat, u) of the accepted state m^n, float64.  out: preallocated (p_hat, u) tensors to read
        into (e.g. pinned host buffers, for a fast device-to-host copy); their side decides on_device."""
        if out is not None:
            p, u = out
            if (p.dtype != torch.float64 or u.dtype != torch.float64 or not p.is_contiguous() or
                    not u.is_contiguous() or tuple(p.shape) != self.grid or
                    tuple(u.shape) != (self.dim,) + self.grid or p.is_cuda != u.is_cuda):
                raise ValueError("out must be contiguous float64 (p_hat, u) tensors of the lattice's shape")
            on_device = p.is_cuda
        else:
            dev = self.device if on_device else torch.device("cpu")
            p = torch.empty(self.grid, dtype=torch.float64, device=dev)
            u = torch.empty((self.dim,) + self.grid, dtype=torch.float64, device=dev)
        L.check(L.lib.msc_read_fields(self._ctx, _ptr(p), _ptr(u), int(on_device)), "msc_read_fields")
        return p, u

    def populations(self) -> np.ndarray:
        f = np.empty((self.Q,) + self.grid, dtype=np.float64)
        L.check(L.lib.msc_read_populations(self._ctx, f.ctypes.data, 0), "msc_read_populations")
        return f

    def residual_history(self) -> np.ndarray:
        out = np.empty(self.hist_cap, dtype=np.float64)
        n = ctypes.c_int()
        L.check(L.lib.msc_get_residual_history(self._ctx, out.ctypes.data, self.hist_cap, ctypes.byref(n)),
                "msc_get_residual_history")
        return out[:n.value].copy()

    def step_iters(self) -> np.ndarray:
        out = np.empty(self.max_steps, dtype=np.int32)
        n = ctypes.c_int()
        L.check(L.lib.msc_get_step_iters(self._ctx, out.ctypes.data, self.max_steps, ctypes.byref(n)),
                "msc_get_step_iters")
        return out[:n.value].copy()

    def set_replay_counts(self, counts):
        c = np.ascontiguousarray(np.asarray(counts, dtype=np.int32))
        L.check(L.lib.msc_set_replay_counts(self._ctx, c.ctypes.data, len(c)), "msc_set_replay_counts")

    def save_state(self) -> bytes:
        n = ctypes.c_size_t()
        L.check(L.lib.msc_save_state(self._ctx, None, ctypes.byref(n)), "msc_save_state")
        buf = ctypes.create_string_buffer(n.value)
        L.check(L.lib.msc_save_state(self._ctx, buf, ctypes.byref(n)), "msc_save_state")
        return buf.raw[:n.value]

    def load_state(self, blob: bytes):
        L.check(L.lib.msc_load_state(self._ctx, blob, len(blob)), "msc_load_state")

    def save_state_device(self) -> torch.Tensor:
        """The msc_save_state blob, kept in device memory (uint8 tensor)."""
        n = ctypes.c_size_t()
        L.check(L.lib.msc_save_state_device(self._ctx, None, ctypes.byref(n)), "msc_save_state_device")
        blob = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        L.check(L.lib.msc_save_state_device(self._ctx, _ptr(blob), ctypes.byref(n)), "msc_save_state_device")
        return blob

    def load_state_device(self, blob: torch.Tensor):
        L.check(L.lib.msc_load_state_device(self._ctx, _ptr(blob), blob.numel()), "msc_load_state_device")

    def moments_into(self, out: torch.Tensor):
        """Copy m^n = (p_hat, u) of the last accepted step into a (d+1, n, ...) float64 device tensor."""
        _check_moments(out)
        L.check(L.lib.msc_read_fields(self._ctx, _ptr(out[0]), _ptr(out[1]), 1), "msc_read_fields")

    def copy_fields_async(self, out: torch.Tensor):
        """msc_copy_fields_async: m^n into a (d+1, n, ...) float64 device tensor, stream-ordered, no sync."""
        _check_moments(out)
        L.check(L.lib.msc_copy_fields_async(self._ctx, _ptr(out)), "msc_copy_fields_async")

    def adjoint_step(self, q: int, m_new, m_cur, m_prev, abar_new, abar_cur, abar_prev, dforce,
                     eps: float = 1e-10, kmax: int = 1000) -> dict:
        """msc_adjoint_step: dL/dm^{n+1} -> accumulate into dL/dm^n, dL/dm^{n-1}, dL/dF (device float64)."""
        _check_moments(m_new, m_cur, m_prev, abar_new, abar_cur, abar_prev)
        st = L.AdjointStats()
        rc = L.lib.msc_adjoint_step(self._ctx, int(q), _ptr(m_new), _ptr(m_cur), _dptr(m_prev), _ptr(abar_new),
                                    _ptr(abar_cur), _dptr(abar_prev), _ptr(dforce), float(eps), int(kmax),
                                    ctypes.byref(st))
        L.check(rc, "msc_adjoint_step")
        return {"iters": st.iters, "residual": st.residual}

    def adjoint_steps(self, steps, dforce, eps: float = 1e-10, kmax: int = 1000, stepwise: bool = False) -> list:
        """msc_adjoint_steps: several adjoint steps in list order, one synchronisation per 64 steps.

        `steps` holds tuples (q, m_new, m_cur, m_prev, abar_new, abar_cur, abar_prev[, warm]) as in
        adjoint_step; warm (default False) starts the step's solve from the last converged step.  Returns one dict (iters, residual, status) per step; raises on a failed step.
        stepwise=True: msc_adjoint_steps_stepwise (host-driven, for profiling; identical results)."""
        arr = (L.AdjointIO * max(1, len(steps)))()
        for i, st in enumerate(steps):
            q, m_new, m_cur, m_prev, abar_new, abar_cur, abar_prev = st[:7]
            _check_moments(m_new, m_cur, m_prev, abar_new, abar_cur, abar_prev)
            arr[i] = L.AdjointIO(int(q), _ptr(m_new), _ptr(m_cur), _dptr(m_prev), _ptr(abar_new), _ptr(abar_cur),
                                 _dptr(abar_prev), int(bool(st[7])) if len(st) > 7 else 0)
        _check_moments(dforce)
        out = (L.AdjointStats * max(1, len(steps)))()
        fn = L.lib.msc_adjoint_steps_stepwise if stepwise else L.lib.msc_adjoint_steps
        rc = fn(self._ctx, len(steps), arr, _ptr(dforce), float(eps), int(kmax), out)
        L.check(rc, "msc_adjoint_steps")
        return [{"iters": s.iters, "residual": s.residual, "status": s.status} for s in out[:len(steps)]]


# ---- stage calls ---------------------------------------------------------------------------------

def _dptr(t):
    return None if t is None else t.data_ptr()


def _check_moments(*ts):
    for t in ts:
        if t is not None and (t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous()):
            raise ValueError("moment arrays must be contiguous float64 device tensors of shape (d+1, n, n)")


class MscBatch:
    """Several D2Q9 lattices (one precision, one stream, any mix of n and parameters) marched by one
    CUDA graph; see msc_batch_* in include/msclbm.h.  Per-instance setup and read-back stay on the
    MscLattice objects (set_params, init_fields, stats, fields, step_iters ...)."""

    def __init__(self, lattices):
        self.lattices = list(lattices)
        k = len(self.lattices)
        if k == 0:
            raise ValueError("empty batch")
        self.stream = self.lattices[0].stream
        arr = (ctypes.c_void_p * k)(*[lat._ctx.value for lat in self.lattices])
        nbytes = L.lib.msc_batch_workspace_bytes(arr, k)
        if nbytes == 0:
            raise ValueError("invalid batch: D2Q9 lattices of one precision, at most "
                             f"{L.MSC_BATCH_MAX} of them and {L.MSC_BATCH_CLASSES} distinct n")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.lattices[0].device)
        self._b = ctypes.c_void_p()
        L.check(L.lib.msc_batch_create(ctypes.byref(self._b), arr, k, _ptr(self.workspace), nbytes,
                                       self.stream.cuda_stream), "msc_batch_create")

    def close(self):
        if self._b:
            L.lib.msc_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _counts(self, n_steps):
        if isinstance(n_steps, int):
            n_steps = [n_steps] * len(self.lattices)
        if len(n_steps) != len(self.lattices):
            raise ValueError("one step count per lattice")
        return (ctypes.c_int * len(n_steps))(*[int(v) for v in n_steps])

    def march(self, n_steps):
        """n_steps: one count per lattice (or one int for all)."""
        L.check(L.lib.msc_batch_march(self._b, self._counts(n_steps)), "msc_batch_march")

    def explicit_march(self, n_steps):
        L.check(L.lib.msc_batch_explicit_march(self._b, self._counts(n_steps)), "msc_batch_explicit_march")

    @staticmethod
    def _tuning_dict(t) -> dict:
        k = t.n_classes
        return {"n": list(t.n[:k]), "sweep_rows": list(t.sweep_rows[:k]), "fft_rows": list(t.fft_rows[:k]),
                "col_lines": list(t.col_lines[:k]), "sweep_ctas_per_sm": t.sweep_ctas_per_sm,
                "sweep_us": t.sweep_us, "rowfft_us": t.rowfft_us, "colsolve_us": t.colsolve_us}

    def autotune(self, reps: int = 5) -> dict:
        t = L.BatchTuning()
        L.check(L.lib.msc_batch_autotune(self._b, int(reps), ctypes.byref(t)), "msc_batch_autotune")
        return self._tuning_dict(t)

    @property
    def tuning(self) -> dict:
        t = L.BatchTuning()
        L.check(L.lib.msc_batch_get_tuning(self._b, ctypes.byref(t)), "msc_batch_get_tuning")
        return self._tuning_dict(t)

    def time_stage(self, which: str, reps: int = 10) -> float:
        """Best-of-reps microseconds of one batched kernel family ('sweep', 'rowfft', 'colsolve')."""
        us = ctypes.c_float()
        code = {"sweep": 0, "rowfft": 1, "colsolve": 2}[which]
        L.check(L.lib.msc_batch_time_stage(self._b, code, int(reps), ctypes.byref(us)), "msc_batch_time_stage")
        return us.value

    def set_tuning(self, tun: dict):
        t = L.BatchTuning()
        L.check(L.lib.msc_batch_get_tuning(self._b, ctypes.byref(t)), "msc_batch_get_tuning")
        for key in ("sweep_rows", "fft_rows", "col_lines"):
            for c, v in enumerate(tun[key]):
                getattr(t, key)[c] = int(v)
        t.sweep_ctas_per_sm = int(tun["sweep_ctas_per_sm"])
        L.check(L.lib.msc_batch_set_tuning(self._b, ctypes.byref(t)), "msc_batch_set_tuning")


class StageScratch:
    def __init__(self, dim: int, n: int, precision: str, device="cuda"):
        self.nbytes = L.lib.msc_stage_scratch_bytes(dim, n, precision_code(precision))
        if self.nbytes == 0:
            raise ValueError("unsupported lattice")
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)


def sweep(dim: int, n: int, precision: str, a: float, f_in: torch.Tensor, h: torch.Tensor,
          dm: torch.Tensor = None, scratch: StageScratch = None, stream=None):
    """One fused sweep through msc_sweep: returns (f_out, P r, sum r^2 as a device double)."""
    dt, ft = storage_dtype(precision), field_dtype(precision)
    for t, want in ((f_in, dt), (h, ft)) + (((dm, ft),) if dm is not None else ()):
        if t.dtype != want or not t.is_cuda or not t.is_contiguous():
            raise ValueError("stage inputs must be contiguous device tensors of the storage / field type")
    scratch = scratch or StageScratch(dim, n, precision, f_in.device)
    f_out = torch.empty_like(f_in)
    pr = torch.empty((dim + 1,) + (n,) * dim, dtype=ft, device=f_in.device)
    ssq = torch.empty((), dtype=torch.float64, device=f_in.device)
    L.check(L.lib.msc_sweep(dim, n, precision_code(precision), float(a), _ptr(f_in),
                            _ptr(dm) if dm is not None else None, _ptr(h), _ptr(f_out), _ptr(pr), _ptr(ssq),
                            _ptr(scratch.buf), scratch.nbytes, _stream(stream)), "msc_sweep")
    return f_out, pr, ssq


def _outputs(out, shapes, device):
    """Caller-given output tensors (checked against (shape, dtype) pairs), or new ones."""
    if out is None:
        return [torch.empty(sh, dtype=dt, device=device) for sh, dt in shapes]
    if len(out) != len(shapes) or any(tuple(t.shape) != tuple(sh) or t.dtype != dt or not t.is_cuda or
                                      not t.is_contiguous() for t, (sh, dt) in zip(out, shapes)):
        raise ValueError("out: contiguous device tensors of shapes and dtypes " + str(shapes))
    return list(out)


def sweep_hpair(n: int, precision: str, a: float, f_in: torch.Tensor, h: torch.Tensor, dm: torch.Tensor = None,
                scratch: StageScratch = None, stream=None, out=None):
    """The D2Q9 march's sweep through msc_sweep_hpair: h of shape (2, 3, n, n) (high, low parts) for
    binary32 storage, (3, n, n) for FP64; returns (f_out, P r, sum r^2 as a device double), written
    into `out` = (f_out, P r, sum) when given (repeated calls then allocate nothing)."""
    dt, ft = storage_dtype(precision), field_dtype(precision)
    hshape = (3, n, n) if precision == "fp64" else (2, 3, n, n)
    if tuple(h.shape) != hshape:
        raise ValueError(f"h must have shape {hshape}")
    for t, want in ((f_in, dt), (h, ft)) + (((dm, ft),) if dm is not None else ()):
        if t.dtype != want or not t.is_cuda or not t.is_contiguous():
            raise ValueError("stage inputs must be contiguous device tensors of the storage / field type")
    scratch = scratch or StageScratch(2, n, precision, f_in.device)
    f_out, pr, ssq = _outputs(out, [(f_in.shape, dt), ((3, n, n), ft), ((), torch.float64)], f_in.device)
    L.check(L.lib.msc_sweep_hpair(n, precision_code(precision), float(a), _ptr(f_in),
                                  _ptr(dm) if dm is not None else None, _ptr(h), _ptr(f_out), _ptr(pr), _ptr(ssq),
                                  _ptr(scratch.buf), scratch.nbytes, _stream(stream)), "msc_sweep_hpair")
    return f_out, pr, ssq


def sweep_d3q19_pf(n: int, precision: str, a: float, f_in: torch.Tensor, pf_in: torch.Tensor, h: torch.Tensor,
                   dm: torch.Tensor = None, scratch: StageScratch = None, stream=None, out=None):
    """The march's halo-free D3Q19 sweep through msc_sweep_d3q19_pf (pf_in = P f_in): returns
    (f_out, P f_out, P r, sum r^2 as a device double), written into `out` when given.  h: (4, n, n, n)
    for FP64 storage, the binary32 pair (2, 4, n, n, n) = (high parts, low parts) for FP32 storage."""
    dt = storage_dtype(precision)
    for t in (f_in, pf_in, h) + ((dm,) if dm is not None else ()):
        if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise ValueError("stage inputs must be contiguous device tensors of the storage type")
    if h.numel() != (2 if precision == "fp32" else 1) * 4 * n ** 3:
        raise ValueError("h: 4 n^3 values (FP64) or a binary32 pair of 2 x 4 n^3 values (FP32)")
    scratch = scratch or StageScratch(3, n, precision, f_in.device)
    f_out, pf_out, pr, ssq = _outputs(out, [(f_in.shape, dt), (pf_in.shape, dt), ((4, n, n, n), dt),
                                            ((), torch.float64)], f_in.device)
    L.check(L.lib.msc_sweep_d3q19_pf(n, precision_code(precision), float(a), _ptr(f_in), _ptr(pf_in),
                                     _ptr(dm) if dm is not None else None, _ptr(h), _ptr(f_out), _ptr(pf_out), _ptr(pr),
                                     _ptr(ssq), _ptr(scratch.buf), scratch.nbytes, _stream(stream)),
            "msc_sweep_d3q19_pf")
    return f_out, pf_out, pr, ssq


def sweep_trt(n: int, precision: str, a: float, omega_p: float, omega_m: float, f_in: torch.Tensor, h: torch.Tensor,
              dm: torch.Tensor = None, scratch: StageScratch = None, stream=None):
    """One D2Q9 sweep with the general TRT collision through msc_sweep_trt: (f_out, P r, sum r^2)."""
    dt, ft = storage_dtype(precision), field_dtype(precision)
    for t, want in ((f_in, dt), (h, ft)) + (((dm, ft),) if dm is not None else ()):
        if t.dtype != want or not t.is_cuda or not t.is_contiguous():
            raise ValueError("stage inputs must be contiguous device tensors of the storage / field type")
    scratch = scratch or StageScratch(2, n, precision, f_in.device)
    f_out = torch.empty_like(f_in)
    pr = torch.empty((3, n, n), dtype=ft, device=f_in.device)
    ssq = torch.empty((), dtype=torch.float64, device=f_in.device)
    L.check(L.lib.msc_sweep_trt(n, precision_code(precision), float(a), float(omega_p), float(omega_m), _ptr(f_in),
                                _dptr(dm), _ptr(h), _ptr(f_out), _ptr(pr), _ptr(ssq), _ptr(scratch.buf),
                                scratch.nbytes, _stream(stream)), "msc_sweep_trt")
    return f_out, pr, ssq


def full_symbol_correct(n: int, precision: str, a: float, omega_p: float, omega_m: float, f: torch.Tensor,
                        f_swept: torch.Tensor, out: torch.Tensor = None, scratch: torch.Tensor = None, stream=None):
    """msc_full_symbol_correct: f + F^-1[(I - Z J)^-1 F[f_swept - f]] (D2Q9, FP64 or FP32 storage)."""
    dt = storage_dtype(precision)
    for t in (f, f_swept):
        if t.dtype != dt or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != (9, n, n):
            raise ValueError("populations must be contiguous (9, n, n) device tensors of the storage type")
    need = L.lib.msc_full_symbol_scratch_bytes(n, precision_code(precision))
    if need == 0:
        raise ValueError(f"full-symbol correction: unsupported n = {n} or precision {precision}")
    if scratch is None:
        scratch = torch.empty(need, dtype=torch.uint8, device=f.device)
    out = torch.empty_like(f) if out is None else out
    L.check(L.lib.msc_full_symbol_correct(n, precision_code(precision), float(a), float(omega_p), float(omega_m),
                                          _ptr(f), _ptr(f_swept), _ptr(out), _ptr(scratch), scratch.numel(),
                                          _stream(stream)), "msc_full_symbol_correct")
    return out


def shadow_solve(dim: int, n: int, precision: str, a: float, nu: float, pr: torch.Tensor,
                 scratch: StageScratch = None, stream=None):
    """delta m = F^-1[chi H^-1 F[P r]] through msc_shadow_solve."""
    scratch = scratch or StageScratch(dim, n, precision, pr.device)
    dm = torch.empty_like(pr)
    L.check(L.lib.msc_shadow_solve(dim, n, precision_code(precision), float(a), float(nu), _ptr(pr), _ptr(dm),
                                   _ptr(scratch.buf), scratch.nbytes, _stream(stream)), "msc_shadow_solve")
    return dm


def equilibrium(dim: int, n: int, precision: str, p_hat: torch.Tensor, u: torch.Tensor, stream=None):
    f = torch.empty((9 if dim == 2 else 19,) + (n,) * dim, dtype=storage_dtype(precision), device=p_hat.device)
    L.check(L.lib.msc_equilibrium(dim, n, precision_code(precision), _ptr(p_hat.contiguous()),
                                  _ptr(u.contiguous()), _ptr(f), _stream(stream)), "msc_equilibrium")
    return f
