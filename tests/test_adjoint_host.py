"""Host logic of the reverse pass (paper_2609_39474_b300/adjoint.py) on the CPU, with a stand-in
lattice: the order of the adjoint steps, their BDF orders and warm-start flags, the moments each step
receives after checkpoint reloads and replays, the chunking of recorded runs into calls of 64 steps,
and the accumulation of dL/dm^n, dL/dm^{n-1} and dL/dF.  The stand-in's 'adjoint step' is the plain
linear map of the BDF history (dL/dh = dL/dm^{n+1}), so the expected gradient follows from a
recursion written out in the test."""
import numpy as np
import pytest
import torch

from paper_2609_39474_b300 import build as _build

_build.build()  # the binding loads the in-tree library at import (no compute call is made here)
from paper_2609_39474_b300.adjoint import MarchRunner  # noqa: E402

SHAPE = (4, 4)


def moments_of(n):
    """The stand-in march's m^n: a field whose every value encodes n."""
    m = torch.empty((3,) + SHAPE, dtype=torch.float64)
    m[0] = 100.0 + n
    m[1] = 200.0 + n
    m[2] = 300.0 + n
    return m


class FakeLattice:
    dim, Q, precision, device = 2, 9, "fp64", torch.device("cpu")
    grid, sites = SHAPE, SHAPE[0] * SHAPE[1]

    def __init__(self):
        self.n = 0
        self.calls = []      # (n, q, warm) per adjoint step, in call order
        self.batches = []    # steps per adjoint_steps call
        self.params = None

    def set_params(self, **kw):
        self.params = kw

    def init_fields(self, p0, u0):
        self.n = 0

    def march(self, k):
        self.n += k

    march_stepwise = march

    def stats(self):
        return {"status": 0}

    def moments_into(self, m):
        m.copy_(moments_of(self.n))

    def copy_fields_async(self, m):
        m.copy_(moments_of(self.n))

    def save_state_device(self):
        # the msc_save_state layout: header (n_avail = 1 at int32 index 4, steps done at byte 24),
        # one population array, then m^n and m^{n-1}
        hdr = torch.zeros(8, dtype=torch.int32)
        hdr[4] = 1
        hdr[6] = self.n
        pops = torch.zeros(self.Q * self.sites * 8, dtype=torch.uint8)
        mom = torch.cat([moments_of(self.n).flatten(), moments_of(max(self.n - 1, 0)).flatten()])
        return torch.cat([hdr.view(torch.uint8), pops, mom.view(torch.uint8)])

    def load_state_device(self, blob):
        self.n = int(blob[:32].view(torch.int32)[6])

    def adjoint_steps(self, steps, dF, eps, kmax, stepwise=False):
        self.batches.append(len(steps))
        out = []
        for st in steps:
            q, m_new, m_cur, m_prev, abar_new, abar_cur, abar_prev, warm = st
            n = int(round(float(m_cur[0, 0, 0]) - 100.0))
            assert torch.equal(m_new, moments_of(n + 1)) and torch.equal(m_cur, moments_of(n))
            if q == 2:
                assert torch.equal(m_prev, moments_of(n - 1))
            c1, c2 = (1.0, 0.0) if q == 1 else (2.0, 0.5)
            abar_cur += c1 * abar_new
            if q == 2:
                abar_prev -= c2 * abar_new
            dF[:2] += abar_new[1:].sum(dim=(1, 2))
            self.calls.append((n, q, bool(warm)))
            out.append({"iters": n, "residual": 0.0, "status": 0})
        return out


def expected(S, g):
    a = {k: torch.zeros((3,) + SHAPE, dtype=torch.float64) for k in range(-1, S + 1)}
    a[S][1:] = g
    dF = torch.zeros(2, dtype=torch.float64)
    for n in range(S - 1, -1, -1):
        q = 1 if n == 0 else 2
        dF += a[n + 1][1:].sum(dim=(1, 2))
        a[n] += (1.0 if q == 1 else 2.0) * a[n + 1]
        if q == 2:
            a[n - 1] -= 0.5 * a[n + 1]
    return a[0], dF


@pytest.mark.parametrize("S,K,record", [(10, 1, False), (10, 3, False), (10, 8, False), (10, 10, False),
                                        (10, 4, True), (130, 8, False), (130, 8, True)])
def test_reverse_pass_bookkeeping(S, K, record):
    L = FakeLattice()
    R = MarchRunner(L, dt=1.0, steps=S, checkpoint_every=K, record_moments=record)
    uS = R.forward(torch.zeros(SHAPE), torch.zeros((2,) + SHAPE))
    assert torch.equal(uS, moments_of(S)[1:])
    g = torch.as_tensor(np.random.default_rng(1).standard_normal((2,) + SHAPE))
    gp, gu, gF = R.backward(g)
    a0, dF = expected(S, g)
    assert torch.allclose(gp, a0[0], rtol=1e-12, atol=0) and torch.allclose(gu, a0[1:], rtol=1e-12, atol=0)
    assert torch.allclose(gF, dF, rtol=1e-12, atol=0)
    # every step once, last first; BDF1 only for the first physical step; cold start only for the
    # first step of the reverse pass
    assert [c[0] for c in L.calls] == list(range(S - 1, -1, -1))
    assert all((c[1] == 1) == (c[0] == 0) for c in L.calls)
    assert all(c[2] == (c[0] != S - 1) for c in L.calls)
    assert R.adjoint_iters == list(range(S))
    if record:
        assert L.batches == [64] * (S // 64) + ([S % 64] if S % 64 else [])
    else:
        assert L.batches == [min(K, S - s0) for s0 in range(0, S, K)][::-1]
