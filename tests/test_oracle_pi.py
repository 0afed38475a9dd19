"""Pins of the oracle's particle interaction (PI, Sections 2 and 4.5).

The checks come from properties of the equations rather than a retyped
formula: pairwise antisymmetry of the forces (Section 3.1: f_ba = -f_ab, so a
closed fluid conserves momentum), the rest state (no pressure, no motion),
the SPH approximation of -rho div(v) and of -grad(P)/rho, the dissipative
sign of the artificial viscosity, and the absence of boundary-boundary
interactions (Section 2).
"""
import math

import numpy as np
import pytest

from sphcases import uniform_block, dam_break, random_cloud


def test_momentum_conserved_closed_fluid(oracle_lib):
    """g = 0, no boundaries: sum_a m ace_a = 0 to round-off."""
    c = uniform_block(10, 0.01, seed=3, vel_sigma=0.3, rho_sigma=0.01, jitter=0.2)
    ace, ar, vm, counts, nout = oracle_lib.interact(c.params, c.n_f, 0, c.pos, c.vel, c.rho)
    m = c.params.mass
    tot = (m * ace).sum(0)
    scale = (m * np.abs(ace)).sum()
    assert scale > 0
    assert np.abs(tot).max() <= 1e-13 * scale
    assert vm > 0


def test_rest_state(oracle_lib):
    """Uniform lattice at rho0 with v = 0: P = 0, so ace = g and ar = 0 exactly."""
    c = uniform_block(8, 0.01)
    p = c.params
    p.g = (0.0, 0.0, -9.81)
    ace, ar, vm, counts, nout = oracle_lib.interact(p, c.n_f, 0, c.pos, c.vel, c.rho)
    assert (ace == np.array([0.0, 0.0, -9.81])).all()
    assert (ar == 0.0).all()
    assert vm == 0.0


def test_continuity_linear_velocity_field(oracle_lib):
    """v = A x on the lattice: drho/dt ~ -rho tr(A) away from the edges."""
    c = uniform_block(14, 0.01)
    A = np.array([[0.3, 0.1, -0.2], [0.05, -0.7, 0.4], [0.2, 0.1, 0.15]])
    vel = c.pos @ A.T
    ace, ar, vm, counts, nout = oracle_lib.interact(c.params, c.n_f, 0, c.pos, vel, c.rho)
    ctr = c.pos.mean(0)
    interior = np.all(np.abs(c.pos - ctr) < 0.02, axis=1)
    assert interior.sum() > 20
    expect = -1000.0 * np.trace(A)
    assert np.allclose(ar[interior], expect, rtol=2e-2)


def test_pressure_gradient_balances_gravity(oracle_lib):
    """Hydrostatic column at t = 0: the SPH pressure force cancels g to ~2%
    for fluid particles farther than 2h from walls and the free surface."""
    c = dam_break(0.01)
    p = c.params
    ace, ar, vm, counts, nout = oracle_lib.interact(p, c.n_f, c.n_b, c.pos, c.vel, c.rho)
    f = c.pos[:c.n_f]
    s = p.cell_size
    Lx, Ly, _ = c.tank
    H = c.meta["H"]
    interior = ((f[:, 0] > s) & (f[:, 0] < 0.4 - s) & (f[:, 1] > s) & (f[:, 1] < Ly - s)
                & (f[:, 2] > s) & (f[:, 2] < H - s))
    assert interior.sum() > 1000
    assert np.abs(ace[interior]).max() < 0.03 * 9.81
    assert (ar == 0.0).all()  # nothing moves at t = 0


def test_viscosity_is_dissipative(oracle_lib):
    """Two approaching particles at rho0 (no pressure): the viscous force opposes
    the relative velocity; receding particles feel no viscous force."""
    c = uniform_block(2, 0.01)
    p = c.params
    pos = np.array([[0.05, 0.05, 0.05], [0.05 + 0.012, 0.05, 0.05]])
    rho = np.full(2, 1000.0)
    approach = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    ace, ar, vm, counts, _ = oracle_lib.interact(p, 2, 0, pos, approach, rho)
    rel_v = approach[0] - approach[1]
    rel_a = ace[0] - ace[1]
    assert rel_a @ rel_v < 0
    assert np.allclose(ace[0], -ace[1])
    recede = -approach
    ace2, *_ = oracle_lib.interact(p, 2, 0, pos, recede, rho)
    assert (ace2 == 0.0).all()
    # linear in alpha for approaching pairs
    p2 = uniform_block(2, 0.01).params
    p2.alpha = 2 * p.alpha
    ace3, *_ = oracle_lib.interact(p2, 2, 0, pos, approach, rho)
    assert np.allclose(ace3, 2 * ace, rtol=1e-14)


def test_no_boundary_boundary_interaction(oracle_lib):
    c = random_cloud(400, box=0.05, dp=0.01, n_b=400, seed=1)
    ace, ar, vm, counts, _ = oracle_lib.interact(c.params, 0, c.n_b, c.pos, c.vel, c.rho)
    assert (ar == 0.0).all() and counts[3] == 0


def test_pair_counts_match_pair_list(oracle_lib):
    c = random_cloud(1200, box=0.1, dp=0.01, n_b=300, seed=7)
    pa, pb = oracle_lib.pairs(c.params, c.n_f, c.n_b, c.pos)
    _, _, _, counts, _ = oracle_lib.interact(c.params, c.n_f, c.n_b, c.pos, c.vel, c.rho)
    assert counts[1] + counts[3] == len(pa)
    assert counts[3] == int((pa >= c.n_f).sum())


def _brute_pi(case):
    """Independent all-pairs evaluation of the same sums, vectorised (checks the
    cell-list machinery: which pairs enter and with which types)."""
    p = case.params
    pos, vel, rho = case.pos, case.vel, case.rho
    n, nf = case.n, case.n_f
    B = p.c0 ** 2 * p.rho0 / p.gamma
    P = B * ((rho / p.rho0) ** p.gamma - 1.0)
    cs = p.c0 * (rho / p.rho0) ** ((p.gamma - 1) / 2)
    rab = pos[:, None, :] - pos[None, :, :]
    vab = vel[:, None, :] - vel[None, :, :]
    r2 = (rab ** 2).sum(-1)
    isb = np.arange(n) >= nf
    mask = (r2 < 4 * p.h ** 2) & ~np.eye(n, dtype=bool) & ~(isb[:, None] & isb[None, :])
    r = np.sqrt(np.where(mask, r2, 1.0))
    q = r / p.h
    ad = 1.0 / (math.pi * p.h ** 3)
    dwdq = np.where(q < 1, ad * (-3 * q + 2.25 * q * q), ad * (-0.75 * (2 - q) ** 2))
    F = np.where(mask, dwdq / (p.h * r), 0.0)
    vdr = (vab * rab).sum(-1)
    mu = p.h * vdr / (r2 + p.eta2_coef * p.h ** 2)
    Pi = np.where(vdr < 0, -p.alpha * 0.5 * (cs[:, None] + cs[None, :]) * mu
                  / (0.5 * (rho[:, None] + rho[None, :])), 0.0)
    coef = -p.mass * (P[:, None] / rho[:, None] ** 2 + P[None, :] / rho[None, :] ** 2 + Pi)
    ace = (coef[..., None] * F[..., None] * rab).sum(1)[:nf] + np.asarray(p.g)
    ar = (p.mass * vdr * F).sum(1)
    vm = np.abs(np.where(mask, mu, 0.0)).max()
    return ace, ar, vm


def test_pi_matches_all_pairs_evaluation(oracle_lib):
    c = random_cloud(900, box=0.08, dp=0.01, n_b=250, seed=11)
    ace, ar, vm, _, _ = oracle_lib.interact(c.params, c.n_f, c.n_b, c.pos, c.vel, c.rho)
    ace2, ar2, vm2 = _brute_pi(c)
    assert np.allclose(ace, ace2, rtol=1e-11, atol=1e-9 * np.abs(ace2).max())
    assert np.allclose(ar, ar2, rtol=1e-11, atol=1e-9 * np.abs(ar2).max())
    assert vm == pytest.approx(vm2, rel=1e-14)


def _approaching_pair(v_rel):
    """Two fluid particles on the x axis, 0.012 m apart, with unequal densities
    (1000 and 1100 kg/m^3) and so unequal pressures and sound speeds, moving
    towards each other (v_a = +v_rel/2, v_b = -v_rel/2 along x).  Round
    constants: h = 0.01 m (support and cell 0.02 m), m = 1e-3 kg, rho0 = 1000,
    gamma = 7, c0 = 10 m/s, alpha = 0.1, eta^2 = 0.01 h^2, no gravity."""
    from sphcases.dambreak import RunParams
    p = RunParams(dp=0.01, h=0.01, cell_size=0.02, c0=10.0, mass=1e-3, g=(0.0, 0.0, 0.0),
                  dom_min=(0.0, 0.0, 0.0), dom_max=(0.2, 0.2, 0.2))
    pos = np.array([[0.05, 0.05, 0.05], [0.062, 0.05, 0.05]])
    vel = np.array([[0.5 * v_rel, 0.0, 0.0], [-0.5 * v_rel, 0.0, 0.0]])
    rho = np.array([1000.0, 1100.0])
    return p, pos, vel, rho


def test_viscosity_hand_values_unequal_pair(oracle_lib):
    """Artificial viscosity of Monaghan (1992) (Table 1) on one approaching pair
    with unequal rho and c, every number worked by hand:

      r_ab = x_a - x_b = (-0.012, 0, 0),  r = 0.012,  q = r/h = 1.2
      v_ab = (10, 0, 0),  v_ab . r_ab = -0.12  (approaching, so Pi applies)
      mu_ab = h v.r / (r^2 + eta^2) = 0.01 (-0.12) / (1.44e-4 + 1e-6) = -8.2758620689655
      c_a = c0 = 10,  c_b = c0 (1.1)^3 = 13.31,  cbar = 11.655,  rhobar = 1050
      Pi_ab = -alpha cbar mu / rhobar = 0.1 * 11.655 * 8.2758620689655 / 1050 = 9.1862068965517e-3
      dW/dr (1 <= q < 2) = -0.75 (2 - q)^2 / (pi h^4) = -0.48 / (pi 1e-8),
      so grad_a W = (1.5278874536822e7, 0, 0)
      P_a = 0,  P_b / rho_b^2 = (c0^2 rho0 / 7)(1.1^7 - 1) / 1100^2 = 1.1200910271547e-2
      ace_a = -m (P_b/rho_b^2 + Pi_ab) grad_a W = (-311.49220537886, 0, 0),  ace_b = -ace_a
      viscous share of ace_a = -m Pi_ab grad_a W = -140.35490264170
      ar_a = ar_b = m v_ab . grad_a W = 1.5278874536822e5,  max |mu| = 8.2758620689655

    A mu without its factor h, eta^2 taken as 0.01 instead of 0.01 h^2, c_a or
    c_b in place of cbar, or rho_a or rho_b in place of rhobar each moves
    Pi_ab (and the viscous share) by 5 % or more."""
    p, pos, vel, rho = _approaching_pair(10.0)
    ace, ar, vm, counts, _ = oracle_lib.interact(p, 2, 0, pos, vel, rho)
    assert ace[0, 0] == pytest.approx(-311.49220537886, rel=1e-11)
    assert ace[1, 0] == pytest.approx(311.49220537886, rel=1e-11)
    assert np.abs(ace[:, 1:]).max() == 0.0
    assert ar == pytest.approx([1.5278874536822e5, 1.5278874536822e5], rel=1e-11)
    assert vm == pytest.approx(8.2758620689655, rel=1e-11)
    # receding: no viscosity, the pressure term alone
    ace_r, ar_r, vm_r, _, _ = oracle_lib.interact(p, 2, 0, pos, -vel, rho)
    assert ace[0, 0] - ace_r[0, 0] == pytest.approx(-140.35490264170, rel=1e-10)
    assert ace_r[0, 0] == pytest.approx(-311.49220537886 + 140.35490264170, rel=1e-10)
    assert vm_r == pytest.approx(8.2758620689655, rel=1e-11)   # |mu| enters dt either way
