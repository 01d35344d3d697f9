"""Shared helpers of the GPU parity tests (inputs from workloads/, expected values from oracle/)."""
import numpy as np
import torch

from oracle import kinetics as OK
from oracle import march as OM
from oracle.lattice import lattice_for_dim


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype).contiguous()


def host(t):
    return t.detach().to("cpu", torch.float64).numpy()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def oracle_free_run(dim, p, u, params: OM.MarchParams, steps):
    lat = lattice_for_dim(dim)
    st = OM.init_state(lat, p, u)
    recs = OM.march(st, params, steps)
    return st, recs


def oracle_replay(dim, p, u, params: OM.MarchParams, counts):
    lat = lattice_for_dim(dim)
    st = OM.init_state(lat, p, u)
    recs = OM.march(st, params, len(counts), replay_counts=counts)
    return st, recs


def oracle_moments(dim, f):
    return OK.moments(lattice_for_dim(dim), f)


def state_blob(dim, n, precision, st) -> bytes:
    """msc_load_state blob of an oracle state: header, step count, f^n.. (storage type), m^n, m^{n-1}."""
    import struct
    nav = len(st.f_hist)
    hdr = struct.pack("<6iq", 0x4D53434C, dim, n, 0 if precision == "fp64" else 1, nav, 0, st.steps_done)
    dt = np.float64 if precision == "fp64" else np.float32
    parts = [hdr] + [np.ascontiguousarray(f, dtype=dt).tobytes() for f in st.f_hist]
    parts += [np.ascontiguousarray(st.m_n, dtype=np.float64).tobytes(),
              np.ascontiguousarray(st.m_nm1, dtype=np.float64).tobytes()]
    return b"".join(parts)
