"""Pins of the oracle's system update (SU): the Verlet scheme with its periodic
Euler step and the variable time step (Table 1, Section 4.1).

Free fall is solved by hand: with a constant acceleration a, fixed dt and
v^{-1} = v^0 = 0 the Verlet recurrence gives v^n = 2 a dt ceil(n/2) up to the
Euler step at n = N_s - 1, and v^n = (n + 1) a dt after it; with an Euler step
every step, v^n = a n dt and x^n = x^0 + a (n dt)^2 / 2 exactly.
"""
import math

import numpy as np
import pytest

from sphcases import uniform_block, still_tank, dam_break

A = -9.81


def _single(dt, every):
    c = uniform_block(1, 0.01)
    p = c.params
    p.g = (0.0, 0.0, A)
    p.fixed_dt = dt
    p.verlet_euler_every = every
    return c, p


def _run(oracle_lib, c, p, steps):
    st = oracle_lib.State(c, params_override=p)
    xs, vs = [st.pos[0, 2]], [st.vel[0, 2]]
    for _ in range(steps):
        st.step()
        xs.append(st.pos[0, 2])
        vs.append(st.vel[0, 2])
    return np.array(xs), np.array(vs)


def test_free_fall_euler_every_step_is_exact(oracle_lib):
    dt = 1e-3
    c, p = _single(dt, 1)
    xs, vs = _run(oracle_lib, c, p, 60)
    n = np.arange(61)
    x0 = c.pos[0, 2]
    assert np.allclose(vs, A * n * dt, rtol=1e-12, atol=1e-15)
    assert np.allclose(xs, x0 + 0.5 * A * (n * dt) ** 2, rtol=1e-12, atol=1e-15)


def test_free_fall_verlet_with_euler_resync(oracle_lib):
    dt = 1e-3
    every = 40
    c, p = _single(dt, every)
    steps = 90
    xs, vs = _run(oracle_lib, c, p, steps)
    n = np.arange(steps + 1)
    # hand-derived closed form of the velocity sequence (two Euler steps: 39, 79)
    v = np.where(n < every, 2 * A * dt * np.ceil(n / 2), A * dt * (n + 1))
    assert np.allclose(vs, v, rtol=1e-12, atol=1e-15)
    # x^{n+1} = x^n + dt v^n + dt^2 a / 2, summed over the closed-form velocities
    x0 = c.pos[0, 2]
    x = x0 + np.concatenate([[0.0], np.cumsum(dt * v[:-1] + 0.5 * dt * dt * A)])
    assert np.allclose(xs, x, rtol=1e-12, atol=1e-15)
    # before the resync, x^{2K} = x0 + a dt^2 (2K^2 + K)  (exact motion + a t dt / 2)
    K = np.arange(0, 20)
    assert np.allclose(xs[2 * K], x0 + A * dt * dt * (2 * K * K + K), rtol=1e-12, atol=1e-15)


def test_time_step_at_rest(oracle_lib):
    """Still lattice at rho0: no viscous term and ace = g, so
    dt = CFL min(sqrt(h/|g|), h/c0)."""
    c = uniform_block(6, 0.01)
    p = c.params
    p.g = (0.0, 0.0, -9.81)
    ace, ar, vm, counts, _ = oracle_lib.interact(p, c.n_f, 0, c.pos, c.vel, c.rho)
    dt = oracle_lib.time_step(p, c.n_f, 0, c.pos, ace, c.rho, vm)
    assert dt == pytest.approx(0.2 * min(math.sqrt(p.h / 9.81), p.h / p.c0), rel=1e-15)
    # at rest in a tank: the sound-speed limit binds
    assert dt == pytest.approx(0.2 * p.h / p.c0, rel=1e-15)


def test_time_step_force_limit(oracle_lib):
    """A large acceleration makes the force limit bind: dt = CFL sqrt(h/|f|)."""
    c = uniform_block(4, 0.01)
    p = c.params
    p.g = (0.0, 0.0, -9.81e4)
    ace, ar, vm, counts, _ = oracle_lib.interact(p, c.n_f, 0, c.pos, c.vel, c.rho)
    dt = oracle_lib.time_step(p, c.n_f, 0, c.pos, ace, c.rho, vm)
    assert dt == pytest.approx(0.2 * math.sqrt(p.h / 9.81e4), rel=1e-14)


def test_boundary_density_clamped_and_fixed(oracle_lib):
    """Boundary particles never move; their density never drops below rho0."""
    c = dam_break(0.02)
    st = oracle_lib.State(c)
    b0 = st.pos[c.n_f:].copy()
    for _ in range(30):
        st.step()
    assert (st.pos[c.n_f:] == b0).all()
    assert (st.vel[c.n_f:] == 0).all()
    assert (st.rho[c.n_f:] >= 1000.0).all()


@pytest.mark.slow
def test_still_tank_stays_hydrostatic(oracle_lib):
    """A tank filled to 0.1 m over its whole floor: averaged over steps 400-800
    and over depth bins, the Tait pressure of the fluid stays within 5% of
    rho0 g depth (instantaneous values carry acoustic and dynamic-boundary
    noise, a known effect of weak compressibility)."""
    c = still_tank(0.01, depth=0.1, width=(0.15, 0.15))
    st = oracle_lib.State(c)
    st.run(400, nthreads=8)
    H = c.meta["H"]
    bins = (0.03, 0.05, 0.07)
    acc = {lo: [] for lo in bins}
    for k in range(40):
        st.run(10, nthreads=8)
        f = st.pos[:c.n_f]
        P = np.array([oracle_lib.pressure(c.params, r) for r in st.rho[:c.n_f]])
        depth = H - f[:, 2]
        inner = (f[:, 0] > 0.03) & (f[:, 0] < 0.12) & (f[:, 1] > 0.03) & (f[:, 1] < 0.12)
        for lo in bins:
            sel = inner & (depth >= lo) & (depth < lo + 0.02)
            assert sel.sum() > 20
            acc[lo].append((P[sel].mean(), 1000.0 * 9.81 * depth[sel].mean()))
    assert st.n_out == 0
    for lo in bins:
        got, expect = np.mean(acc[lo], axis=0)
        assert abs(got - expect) < 0.05 * expect
    # and the particles are still almost at rest
    assert np.abs(st.vel[:c.n_f]).max() < 0.1


def test_time_step_viscous_limit_hand_value(oracle_lib):
    """dt = CFL min(sqrt(h / max|f|), h / (max c + max|mu|)) (Monaghan & Kos
    1999, Table 1) where the viscous term binds and matters.  The pair of
    tests/test_oracle_pi.py (h = 0.01, rho 1000 and 1100, closing at 10 m/s,
    no gravity) has max c = 13.31, max |mu| = 8.2758620689655 and
    |f| = 311.49220537886, so by hand
      force limit:        0.2 sqrt(0.01 / 311.49) = 1.1332e-3
      sound + viscosity:  0.2 * 0.01 / (13.31 + 8.2758620689655) = 9.2653237272161e-5
    and dt is the second.  Without the viscous term it would be
    0.2 * 0.01 / 13.31 = 1.5026e-4."""
    from tests.test_oracle_pi import _approaching_pair
    p, pos, vel, rho = _approaching_pair(10.0)
    ace, ar, vm, counts, _ = oracle_lib.interact(p, 2, 0, pos, vel, rho)
    dt = oracle_lib.time_step(p, 2, 0, pos, ace, rho, vm)
    assert dt == pytest.approx(9.2653237272161e-5, rel=1e-11)
    # the same closing speed ten times lower: |mu| = 0.82758620689655 still adds
    # 6 % to the sound speed, 0.2 * 0.01 / (13.31 + 0.82758620689655) = 1.4146630e-4
    ace, ar, vm, counts, _ = oracle_lib.interact(p, 2, 0, pos, 0.1 * vel, rho)
    dt = oracle_lib.time_step(p, 2, 0, pos, ace, rho, vm)
    assert dt == pytest.approx(0.2 * 0.01 / (13.31 + 0.82758620689655), rel=1e-11)
