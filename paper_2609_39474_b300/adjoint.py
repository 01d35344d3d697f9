"""Gradients of a march through its discrete adjoint (msc_adjoint_steps), with checkpoints.

The forward march stores a device-resident state blob every `checkpoint_every` physical steps.
The reverse pass walks the segments last first.  For each it reloads the checkpoint and replays
the segment one step at a time (bit-identical to the forward march), recording each step's
moments m^{n+1} with stream-ordered copies.  Then one msc_adjoint_steps call runs the adjoint of
those steps, last first, with one synchronisation per segment.  The adjoint moment arrays of one
segment (checkpoint interval + 2 of them) are live at a time.  With record_moments=True the
forward march instead keeps every step's moments in device memory (HBM holds thousands of steps
of a 256^2 or 1024^2 lattice) and the reverse pass runs the adjoint alone, 64 steps per call.
Every step runs in the CUDA library; this module only orders the calls and holds the buffers.

``MscMarch.apply(u0, force, runner, p0)`` wraps it as a torch.autograd.Function: the output is the
final velocity u^S (float64, device); backward returns dL/du0 and dL/dforce.
"""
import torch

from .lattice import MscLattice


class MarchRunner:
    """A D2Q9 march of `steps` physical steps with its adjoint."""

    def __init__(self, lattice: MscLattice, dt: float, steps: int, eps: float = 1e-8, checkpoint_every: int = 8,
                 eps_adjoint: float = 1e-10, kmax_adjoint: int = 2000, stepwise: bool = False,
                 record_moments: bool = False, **params):
        # record_moments: keep every step's moments on the device during the forward march ((S + 1) x 3
        # fields of float64; 1.9 GB for N = 256, S = 1229) instead of checkpoints, so the reverse pass
        # replays nothing.  Same gradients.
        # stepwise: every kernel launched from the host (march_stepwise, msc_adjoint_steps_stepwise),
        # same results; for profilers, which do not descend into conditional graph nodes
        if lattice.dim != 2:
            raise ValueError("the adjoint exists for D2Q9 lattices")
        self.L = lattice
        self.dt, self.steps, self.eps = float(dt), int(steps), float(eps)
        self.K = max(1, int(checkpoint_every))
        self.eps_adj, self.kmax_adj = float(eps_adjoint), int(kmax_adjoint)
        self.params = params
        self.stepwise = bool(stepwise)
        self.record = bool(record_moments)
        self.recorded = None
        self.checkpoints = []
        self.adjoint_iters = []

    def _march(self, n):
        if self.stepwise:
            self.L.march_stepwise(n)
        else:
            self.L.march(n)

    def _set_params(self, force):
        self.L.set_params(dt=self.dt, eps=self.eps, force=force, **self.params)

    def forward(self, p0: torch.Tensor, u0: torch.Tensor, force=(0.0, 0.0)) -> torch.Tensor:
        """March from f^0 = f_eq(p0, u0) under the body force; returns u^S (device float64)."""
        self.force = [float(v) for v in force]
        self._set_params(self.force)
        self.L.init_fields(p0, u0)
        self.checkpoints = []
        if self.record:
            return self._forward_recorded()
        for s0 in range(0, self.steps, self.K):
            self.checkpoints.append(self.L.save_state_device())
            self._march(min(self.K, self.steps - s0))
            st = self.L.stats()
            if st["status"] != 0:
                raise RuntimeError(f"forward march stopped with status {st['status']} near step {s0}")
        m = torch.empty((3,) + self.L.grid, dtype=torch.float64, device=self.L.device)
        self.L.moments_into(m)
        return m[1:].clone()

    def _forward_recorded(self):
        shape = (self.steps + 1, 3) + self.L.grid
        if self.recorded is None or self.recorded.shape != shape:
            self.recorded = torch.empty(shape, dtype=torch.float64, device=self.L.device)
        self.L.copy_fields_async(self.recorded[0])
        for n in range(self.steps):  # stream-ordered: one synchronisation for the whole march
            self._march(1)
            self.L.copy_fields_async(self.recorded[n + 1])
        st = self.L.stats()  # an error stops every later step and stays recorded
        if st["status"] != 0:
            raise RuntimeError(f"forward march stopped with status {st['status']}")
        return self.recorded[self.steps][1:].clone()

    def _backward_recorded(self, abar, dF):
        ms, shape, dev = self.recorded, (3,) + self.L.grid, self.L.device
        steps = []
        for n in range(self.steps - 1, -1, -1):
            q = 1 if n == 0 else 2
            for k in (n, n - 1):
                if k >= 0 and k not in abar:
                    abar[k] = torch.zeros(shape, dtype=torch.float64, device=dev)
            steps.append((q, ms[n + 1], ms[n], ms[n - 1] if q == 2 else None, abar[n + 1], abar[n],
                          abar.get(n - 1) if q == 2 else None, n != self.steps - 1))
            if len(steps) == 64 or n == 0:  # one call per 64 steps (one synchronisation)
                rs = self.L.adjoint_steps(steps, dF, self.eps_adj, self.kmax_adj, self.stepwise)
                for k, r in zip(range(n + len(steps) - 1, n - 1, -1), rs):
                    self.adjoint_iters[k] = r["iters"]
                for k in range(n + 1, n + len(steps) + 1):
                    del abar[k]
                steps = []

    def _blob_moments(self, blob: torch.Tensor):
        """(m^n, m^{n-1}) stored in a state blob (layout of msc_save_state)."""
        hdr = blob[:24].cpu().view(torch.int32)
        n_avail = int(hdr[4])
        sites = self.L.sites
        pop_bytes = {"fp64": 8, "fp32": 4, "fp16": 2}[self.L.precision]
        o = 32 + n_avail * self.L.Q * sites * pop_bytes
        nb = 3 * sites * 8
        m_n = blob[o:o + nb].view(torch.float64).view((3,) + self.L.grid)
        m_p = blob[o + nb:o + 2 * nb].view(torch.float64).view((3,) + self.L.grid)
        return m_n, m_p

    def backward(self, grad_u: torch.Tensor):
        """(dL/dp0, dL/du0, dL/dF) for dL/du^S = grad_u."""
        shape = (3,) + self.L.grid
        dev = self.L.device
        abar = {self.steps: torch.zeros(shape, dtype=torch.float64, device=dev)}
        abar[self.steps][1:] = grad_u.to(device=dev, dtype=torch.float64)
        dF = torch.zeros(3, dtype=torch.float64, device=dev)
        self._set_params(self.force)
        self.adjoint_iters = [0] * self.steps
        if self.record:
            self._backward_recorded(abar, dF)
            return abar[0][0].clone(), abar[0][1:].clone(), dF[:2].clone()
        for seg in range(len(self.checkpoints) - 1, -1, -1):
            s0 = seg * self.K
            s1 = min(self.steps, s0 + self.K)
            blob = self.checkpoints[seg]
            m_n, m_p = self._blob_moments(blob)
            ms = {s0: m_n.clone()}
            if s0 >= 1:
                ms[s0 - 1] = m_p.clone()
            self.L.load_state_device(blob)
            for n in range(s0, s1):  # replay the segment, recording each accepted step's moments
                self._march(1)
                m = torch.empty(shape, dtype=torch.float64, device=dev)
                self.L.copy_fields_async(m)  # stream-ordered: no synchronisation inside the replay
                ms[n + 1] = m
            st = self.L.stats()
            if st["status"] != 0:
                raise RuntimeError(f"replay of steps {s0}..{s1} stopped with status {st['status']}")
            steps = []
            for n in range(s1 - 1, s0 - 1, -1):
                q = 1 if n == 0 else 2
                for k in (n, n - 1):
                    if k >= 0 and k not in abar:
                        abar[k] = torch.zeros(shape, dtype=torch.float64, device=dev)
                # every step after the first of the reverse pass starts from its successor's solution
                steps.append((q, ms[n + 1], ms[n], ms.get(n - 1) if q == 2 else None, abar[n + 1], abar[n],
                              abar.get(n - 1) if q == 2 else None, n != self.steps - 1))
            # the segment's adjoint steps, last first, in one call (one synchronisation)
            rs = self.L.adjoint_steps(steps, dF, self.eps_adj, self.kmax_adj, self.stepwise)
            for n, r in zip(range(s1 - 1, s0 - 1, -1), rs):
                self.adjoint_iters[n] = r["iters"]
            for n in range(s0 + 1, s1 + 1):
                del abar[n]
        return abar[0][0].clone(), abar[0][1:].clone(), dF[:2].clone()


class MscMarch(torch.autograd.Function):
    """u^S = march(p0, u0; F); gradients by the discrete adjoint."""

    @staticmethod
    def forward(ctx, u0, force, runner: MarchRunner, p0):
        ctx.runner = runner
        ctx.force_device = force.device
        uS = runner.forward(p0, u0.detach(), [float(v) for v in force.detach().cpu()])
        return uS

    @staticmethod
    def backward(ctx, grad_u):
        _, g_u0, g_F = ctx.runner.backward(grad_u.contiguous())
        return g_u0, g_F.to(ctx.force_device), None, None
