"""Differentiable dam break: a ``torch.autograd.Function`` over the C ABI.

Forward: the SPH_FP64 time loop at fixed dt, with a checkpoint of the full
state every ``checkpoint_every`` steps (``sph_save_state`` into torch-owned
device buffers) and the sensor objective
    J = mean over the last ``window`` states and over the sensors of P_s,
or, with ``front_tau`` set, the front objective
    J = mean over the last ``window`` states of tau log sum_a exp(x_a / tau).
Backward: for each checkpoint segment in reverse, the segment is recomputed
from its checkpoint (storing the start state of every step), then the
hand-written adjoint runs step by step in reverse (``sph_adjoint_step``), adding
the objective's derivative at every recorded state (``sph_sensor_adjoint`` or
``sph_front_adjoint``).
The result is dJ/d(initial fluid velocity) (the initial state has
v^{-1} = v^0, so both adjoint slots count) and dJ/d(alpha).
All arithmetic runs in libsph; torch supplies memory and the stream.
"""
from __future__ import annotations

import copy
import math

import numpy as np
import torch

from . import sph as S


class DamBreakRun:
    """Configuration of one differentiable run (input data, horizon, sensors)."""

    def __init__(self, case, steps, dt, window, sensors=None, checkpoint_every=20, device="cuda",
                 front_tau=None):
        assert 1 <= window <= steps
        assert (sensors is None) != (front_tau is None), "sensors or front_tau, not both"
        self.case = case
        self.steps = int(steps)
        self.dt = float(dt)
        self.window = int(window)
        self.k = max(1, int(checkpoint_every))
        self.device = torch.device(device)
        self.front_tau = None if front_tau is None else float(front_tau)
        if sensors is None:
            self.sensors = torch.zeros((1, 3), dtype=torch.float64, device=self.device)
            self.n_sensors = 0
        else:
            self.sensors = torch.as_tensor(np.ascontiguousarray(sensors, np.float64),
                                           device=self.device).contiguous()
            self.n_sensors = int(self.sensors.shape[0])
        self.sim = None
        self.stats = {}

    def _make_sim(self, vel0, alpha):
        c = self.case
        p = copy.copy(c.params)
        p.alpha = float(alpha)
        p.fixed_dt = self.dt
        dev = self.device
        pos = torch.as_tensor(c.pos, dtype=torch.float64, device=dev).contiguous()
        vel = torch.zeros((c.n, 3), dtype=torch.float64, device=dev)
        vel[:c.n_f] = vel0.to(dev, torch.float64)
        rho = torch.as_tensor(c.rho, dtype=torch.float64, device=dev).contiguous()
        return S.Simulation(p, c.n_f, c.n_b, pos, vel.contiguous(), rho, precision="fp64",
                            device=dev)

    def _recorded(self, n):
        """State n (the state at the start of step n) enters J."""
        return n >= self.steps - self.window + 1

    def forward(self, vel0, alpha):
        sim = self._make_sim(vel0, alpha)
        self.sim = sim
        nb = sim.checkpoint_bytes()
        nseg = math.ceil(self.steps / self.k)
        new = lambda: torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.ckpts = [new() for _ in range(nseg)]
        self.final = new()
        p_buf = torch.zeros(max(self.n_sensors, 1), dtype=torch.float64, device=self.device)
        acc = torch.zeros((), dtype=torch.float64, device=self.device)
        for n in range(self.steps):
            if n % self.k == 0:
                sim.save_state(self.ckpts[n // self.k])
            sim.neighbour_list()
            if self._recorded(n):
                acc = acc + self._measure(sim, p_buf)
            sim.interact()
            sim.update()
        sim.save_state(self.final)
        sim.neighbour_list()
        acc = acc + self._measure(sim, p_buf)
        self.stats["checkpoint_bytes"] = nb * (nseg + 1)
        return acc / (max(self.n_sensors, 1) * self.window)

    def _measure(self, sim, buf):
        """The objective's term of the current state (sum over the sensors, or
        the front position)."""
        if self.front_tau is None:
            S.sph_sensor_pressure(sim.ctx, self.sensors, self.n_sensors, buf)
            return buf.sum()
        S.sph_front_position(sim.ctx, self.front_tau, buf)
        return buf[0].clone()

    def _measure_adjoint(self, sim, dj, dj_dp, lam):
        if self.front_tau is None:
            S.sph_sensor_adjoint(sim.ctx, self.sensors, self.n_sensors, dj_dp, lam)
        else:
            S.sph_front_adjoint(sim.ctx, self.front_tau, dj, lam)

    def backward(self, grad_j):
        sim = self.sim
        c = self.case
        N = c.n
        dev = self.device
        dj = float(grad_j) / (max(self.n_sensors, 1) * self.window)
        dj_dp = torch.full((max(self.n_sensors, 1),), dj, dtype=torch.float64, device=dev)
        lam = torch.zeros(11 * N, dtype=torch.float64, device=dev)
        lam2 = torch.zeros_like(lam)
        dalpha = torch.zeros(1, dtype=torch.float64, device=dev)
        # the final state
        sim.load_state(self.final)
        sim.neighbour_list()
        self._measure_adjoint(sim, dj, dj_dp, lam)
        nb = sim.checkpoint_bytes()
        snaps = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(self.k)]
        nseg = len(self.ckpts)
        for seg in reversed(range(nseg)):
            n0 = seg * self.k
            n1 = min(n0 + self.k, self.steps)
            # recompute the segment, keeping the start state of every step
            sim.load_state(self.ckpts[seg])
            for n in range(n0, n1):
                sim.save_state(snaps[n - n0])
                if n < n1 - 1:
                    sim.step()
            for n in reversed(range(n0, n1)):
                sim.load_state(snaps[n - n0])
                S.sph_adjoint_step(sim.ctx, lam, lam2, dalpha)
                if self._recorded(n):
                    self._measure_adjoint(sim, dj, dj_dp, lam2)
                lam, lam2 = lam2, lam
        self.stats["checkpoint_bytes"] += nb * self.k
        nf = c.n_f
        gv = lam[3 * N:3 * N + 3 * nf] + lam[7 * N:7 * N + 3 * nf]
        return gv.view(nf, 3), dalpha[0]


class DamBreakObjective(torch.autograd.Function):
    """J(vel0, alpha) for a ``DamBreakRun``; backward by the hand-written adjoint."""

    @staticmethod
    def forward(ctx, vel0, alpha, run):
        J = run.forward(vel0.detach(), float(alpha))
        ctx.run = run
        return J

    @staticmethod
    def backward(ctx, grad_j):
        gv, ga = ctx.run.backward(float(grad_j))
        return gv, ga.reshape(()), None


def objective(vel0, alpha, run):
    """Differentiable J(vel0 [n_f, 3] float64 CUDA tensor, alpha 0-d tensor)."""
    return DamBreakObjective.apply(vel0, alpha, run)
