"""Gradient oracle: the fixed-dt SPH step restated with plain PyTorch CPU
float64 operations over an explicit pair list, differentiated by autograd.

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` alone).  The interacting pairs
of every step come from the C oracle's cell lists (``oracle.pairs``) and are
constants of the step, as in the method: the set of pairs changes only where
W and grad W vanish (q = 2).  Every formula follows ``sph_oracle.c`` (Table 1
formulation; see that file for the references).

State (persistent-id order, fluid first): x [N,3], v [N,3] (boundary rows 0),
u = v^{n-1}, rho [N], sig = rho^{n-1}.  Objective: the mean over sensors and
over the recorded states of the Shepard-interpolated pressure, or (front_tau
given) the mean over the recorded states of the front position, the smooth
maximum tau log sum_a exp(x_a / tau) of the fluid x coordinates.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import oracle as O

DT = torch.float64


def _consts(p):
    B = p.c0 * p.c0 * p.rho0 / p.gamma
    aD = 1.0 / (math.pi * p.h ** 3)
    return B, aD


def pressure(p, rho):
    B, _ = _consts(p)
    return B * ((rho / p.rho0) ** p.gamma - 1.0)


def sound(p, rho):
    return p.c0 * (rho / p.rho0) ** (0.5 * (p.gamma - 1.0))


def kernel_w(p, r):
    _, aD = _consts(p)
    q = r / p.h
    return torch.where(q < 1.0, aD * (1.0 - 1.5 * q * q + 0.75 * q ** 3),
                       torch.where(q < 2.0, aD * 0.25 * (2.0 - q) ** 3, torch.zeros_like(q)))


def kernel_f(p, r):
    """grad_a W = F r_ab; F = (dW/dq)/(h r)."""
    _, aD = _consts(p)
    q = r / p.h
    dwdq = torch.where(q < 1.0, aD * (-3.0 * q + 2.25 * q * q), aD * (-0.75 * (2.0 - q) ** 2))
    return dwdq / (p.h * r)


def rates(p, nf, x, v, rho, alpha, pa, pb):
    """PI on a fixed pair list: fluid accelerations [nf,3] (gravity included)
    and density rates [N]."""
    n = x.shape[0]
    r_ab = x[pa] - x[pb]
    v_ab = v[pa] - v[pb]
    r2 = (r_ab * r_ab).sum(1)
    r = torch.sqrt(r2)
    F = kernel_f(p, r)
    vdr = (v_ab * r_ab).sum(1)
    eta2 = p.eta2_coef * p.h * p.h
    mu = p.h * vdr / (r2 + eta2)
    P = pressure(p, rho)
    c = sound(p, rho)
    cbar = 0.5 * (c[pa] + c[pb])
    rhobar = 0.5 * (rho[pa] + rho[pb])
    Pi = torch.where(vdr < 0.0, -alpha * cbar * mu / rhobar, torch.zeros_like(mu))
    fluid_a = pa < nf
    coef = -p.mass * (P[pa] / rho[pa] ** 2 + P[pb] / rho[pb] ** 2 + Pi)
    mom = (coef * F)[:, None] * r_ab
    mom = torch.where(fluid_a[:, None], mom, torch.zeros_like(mom))
    ace = torch.zeros((n, 3), dtype=DT).index_add(0, pa, mom)[:nf]
    ace = ace + torch.tensor(p.g, dtype=DT)
    ar = torch.zeros(n, dtype=DT).index_add(0, pa, p.mass * (vdr * F))
    return ace, ar


def step(p, nf, x, v, u, rho, sig, alpha, step_index, dt):
    """One fixed-dt step (NL -> PI -> SU) on tensors; returns the new state."""
    pa_np, pb_np = O.pairs(p, nf, x.shape[0] - nf, x.detach().numpy())
    pa = torch.from_numpy(pa_np)
    pb = torch.from_numpy(pb_np)
    ace, ar = rates(p, nf, x, v, rho, alpha, pa, pb)
    euler = ((step_index + 1) % p.verlet_euler_every) == 0
    vf, uf = v[:nf], u[:nf]
    if euler:
        v_new = vf + dt * ace
        rho_new = rho + dt * ar
    else:
        v_new = uf + 2.0 * dt * ace
        rho_new = sig + 2.0 * dt * ar
    x_new = torch.cat([x[:nf] + dt * vf + 0.5 * dt * dt * ace, x[nf:]], 0)
    if p.clamp_boundary_rho:
        rho_new = torch.cat([rho_new[:nf], torch.clamp(rho_new[nf:], min=p.rho0)], 0)
    zeros_b = torch.zeros((x.shape[0] - nf, 3), dtype=DT)
    return (x_new, torch.cat([v_new, zeros_b], 0), torch.cat([vf, zeros_b], 0), rho_new, rho)


def sensor_pressure(p, nf, x, rho, spos):
    """Shepard pressure at sensor points from fluid particles within 2h."""
    xs = torch.as_tensor(spos, dtype=DT)
    d = xs[:, None, :] - x[None, :nf, :]
    r = torch.sqrt((d * d).sum(-1))
    inside = r < 2.0 * p.h
    w = torch.where(inside, kernel_w(p, torch.where(inside, r, torch.ones_like(r))) * p.mass
                    / rho[None, :nf], torch.zeros_like(r))
    num = (w * pressure(p, rho)[None, :nf]).sum(1)
    den = w.sum(1)
    return torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)),
                       torch.zeros_like(den))


def front_position(nf, x, tau):
    """Front of the fluid: the smooth maximum tau log sum_a exp(x_a / tau) of the
    fluid x coordinates (it lies between max x and max x + tau log nf)."""
    return tau * torch.logsumexp(x[:nf, 0] / tau, 0)


def objective(case, vel0, alpha, steps, dt, window, spos, front_tau=None):
    """J = mean over sensors and over the states after steps (steps-window, steps]
    of the sensor pressure, or of the front position when front_tau is given.
    vel0: fluid initial velocity [nf,3] tensor; alpha: 0-d tensor."""
    p = case.params
    nf = case.n_f
    x = torch.as_tensor(case.pos, dtype=DT)
    zeros_b = torch.zeros((case.n_b, 3), dtype=DT)
    v = torch.cat([vel0, zeros_b], 0)
    u = v
    rho = torch.as_tensor(case.rho, dtype=DT)
    sig = rho
    acc = torch.zeros((), dtype=DT)
    for n in range(steps):
        x, v, u, rho, sig = step(p, nf, x, v, u, rho, sig, alpha, n, dt)
        if n + 1 > steps - window:
            if front_tau is None:
                acc = acc + sensor_pressure(p, nf, x, rho, spos).sum()
            else:
                acc = acc + front_position(nf, x, front_tau)
    return acc / ((len(spos) if front_tau is None else 1) * window)


def gradient(case, vel0, alpha, steps, dt, window, spos, front_tau=None):
    """(J, dJ/dvel0 [nf,3], dJ/dalpha) by autograd."""
    v0 = torch.as_tensor(vel0, dtype=DT).clone().requires_grad_(True)
    a = torch.tensor(float(alpha), dtype=DT, requires_grad=True)
    J = objective(case, v0, a, steps, dt, window, spos, front_tau)
    gv, ga = torch.autograd.grad(J, (v0, a))
    return float(J.detach()), gv.numpy(), float(ga)


def objective_c(case, vel0, alpha, steps, dt, window, spos, front_tau=None):
    """The same objective evaluated by the C oracle (for finite differences)."""
    import copy
    p = copy.copy(case.params)
    p.alpha = float(alpha)
    p.fixed_dt = dt
    st = O.State(case, params_override=p)
    st.vel[:case.n_f] = vel0
    st.velm1[:] = st.vel
    acc = 0.0
    for n in range(steps):
        st.step()
        if n + 1 > steps - window:
            if front_tau is None:
                acc += O.sensor_pressure(p, case.n_f, st.pos, st.rho, spos).sum()
            else:
                xs = st.pos[:case.n_f, 0] / front_tau
                m = xs.max()
                acc += front_tau * (m + math.log(np.exp(xs - m).sum()))
    return acc / ((len(spos) if front_tau is None else 1) * window)
