"""Pins of the gradient oracle (oracle/grad.py).

Its forward must equal the C oracle's fixed-dt run, and its gradient must
agree with central finite differences of the C oracle itself: tightly on a
smooth case (no viscosity switch, no boundary clamp) and to the FD noise of
the C0 viscosity switch on the dam break.
"""
import copy
import math

import numpy as np
import pytest
import torch

from sphcases import small_dam, uniform_block, wall_sensors

DT = 2e-4


@pytest.fixture(scope="module")
def G():
    from oracle import grad
    return grad


def _blob():
    c = uniform_block(5, 0.02, seed=4, vel_sigma=0.05, rho_sigma=0.002, jitter=0.1)
    c.params.alpha = 0.0
    spos = np.array([[0.05, 0.05, 0.05], [0.03, 0.06, 0.07]])
    return c, spos


def test_torch_forward_equals_c_oracle(oracle_lib, G):
    c = small_dam(0.02)
    spos = wall_sensors(c, wall="back", n_y=2, n_z=2, z_top=0.12)
    v0 = torch.as_tensor(c.vel[:c.n_f])
    J = G.objective(c, v0, torch.tensor(0.1, dtype=torch.float64), 20, DT, 6, spos)
    Jc = G.objective_c(c, c.vel[:c.n_f], 0.1, 20, DT, 6, spos)
    assert float(J) == pytest.approx(Jc, rel=1e-12)


def test_gradient_smooth_case_matches_finite_differences(oracle_lib, G):
    """alpha = 0 and no boundaries: the objective is smooth, so central FD of
    the C oracle converge and must match to 1e-6."""
    c, spos = _blob()
    steps, window = 15, 5
    v0 = c.vel[:c.n_f].copy()
    J, gv, ga = G.gradient(c, v0, 0.0, steps, DT, window, spos)
    rng = np.random.default_rng(2)
    for _ in range(3):
        d = rng.normal(size=v0.shape)
        eps = 1e-4
        jp = G.objective_c(c, v0 + eps * d, 0.0, steps, DT, window, spos)
        jm = G.objective_c(c, v0 - eps * d, 0.0, steps, DT, window, spos)
        fd = (jp - jm) / (2 * eps)
        an = float((gv * d).sum())
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-9
    # dJ/dalpha at alpha = 0: the one-sided switch makes FD one-sided too;
    # compare with a forward difference
    eps = 1e-6
    fd_a = (G.objective_c(c, v0, eps, steps, DT, window, spos) - J) / eps
    assert fd_a == pytest.approx(ga, rel=1e-3, abs=1e-6)


def test_gradient_dam_break_matches_finite_differences(oracle_lib, G):
    """Small dam break with viscosity and dynamic boundaries: 3 random
    directions of v0 and alpha.  The viscosity switch is only C0 (Pi jumps in
    slope where v_ab.r_ab = 0), so central FD carry an O(eps) kink error; with
    eps = 1e-7 they agree to 1e-6 (at eps = 1e-4 the spread is about 1e-3)."""
    c = small_dam(0.02)
    spos = wall_sensors(c, wall="back", n_y=2, n_z=2, z_top=0.12)
    steps, window = 30, 10
    v0 = c.vel[:c.n_f].copy()
    J, gv, ga = G.gradient(c, v0, 0.1, steps, DT, window, spos)
    rng = np.random.default_rng(1)
    for _ in range(3):
        d = rng.normal(size=v0.shape)
        eps = 1e-7
        jp = G.objective_c(c, v0 + eps * d, 0.1, steps, DT, window, spos)
        jm = G.objective_c(c, v0 - eps * d, 0.1, steps, DT, window, spos)
        fd = (jp - jm) / (2 * eps)
        an = float((gv * d).sum())
        assert abs(fd - an) <= 1e-6 * abs(an)
    eps = 1e-6
    fd_a = (G.objective_c(c, v0, 0.1 + eps, steps, DT, window, spos)
            - G.objective_c(c, v0, 0.1 - eps, steps, DT, window, spos)) / (2 * eps)
    assert fd_a == pytest.approx(ga, rel=1e-6)


def test_front_position_closed_forms(oracle_lib, G):
    """The smooth maximum lies in [max x, max x + tau log n]; n equal values give
    exactly x + tau log n; for tau far below the spacing it is the maximum."""
    rng = np.random.default_rng(4)
    x = torch.as_tensor(rng.uniform(0.0, 0.4, size=(500, 3)))
    for tau in (1e-3, 1e-2, 0.1):
        J = float(G.front_position(400, x, tau))
        m = float(x[:400, 0].max())
        assert m <= J <= m + tau * math.log(400)
    same = torch.full((37, 3), 0.25, dtype=torch.float64)
    assert float(G.front_position(37, same, 0.01)) == pytest.approx(0.25 + 0.01 * math.log(37),
                                                                    rel=1e-14)
    assert float(G.front_position(400, x, 1e-6)) == pytest.approx(float(x[:400, 0].max()),
                                                                  abs=1e-12)


def test_front_objective_forward_and_gradient(oracle_lib, G):
    """Front-position objective (mean over the last states of the smooth maximum
    of the fluid x, tau = dp): the autograd forward equals the C oracle's, and
    its gradient matches central differences of the C oracle (eps = 1e-7, the
    viscosity switch being only C0)."""
    c = small_dam(0.02)
    tau = c.params.dp
    steps, window = 30, 10
    v0 = c.vel[:c.n_f].copy()
    J, gv, ga = G.gradient(c, v0, 0.1, steps, DT, window, None, front_tau=tau)
    Jc = G.objective_c(c, v0, 0.1, steps, DT, window, None, front_tau=tau)
    assert J == pytest.approx(Jc, rel=1e-12)
    rng = np.random.default_rng(3)
    for _ in range(2):
        d = rng.normal(size=v0.shape)
        eps = 1e-7
        jp = G.objective_c(c, v0 + eps * d, 0.1, steps, DT, window, None, front_tau=tau)
        jm = G.objective_c(c, v0 - eps * d, 0.1, steps, DT, window, None, front_tau=tau)
        fd = (jp - jm) / (2 * eps)
        an = float((gv * d).sum())
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_gradient_general_gamma_matches_finite_differences(oracle_lib, G):
    """Tait exponent 5 (the general sound speed c0 (rho/rho0)^2 and the
    c_bar / rho_bar viscosity, not the gamma = 7 form): the gradient oracle's
    forward equals the C oracle's and its gradient matches central differences
    of the C oracle run with the same exponent."""
    c = small_dam(0.02)
    c.params = copy.copy(c.params)
    c.params.gamma = 5.0
    spos = wall_sensors(c, wall="back", n_y=2, n_z=2, z_top=0.12)
    steps, window = 25, 8
    v0 = c.vel[:c.n_f].copy()
    J, gv, ga = G.gradient(c, v0, 0.1, steps, DT, window, spos)
    assert J == pytest.approx(G.objective_c(c, v0, 0.1, steps, DT, window, spos), rel=1e-12)
    rng = np.random.default_rng(5)
    for _ in range(2):
        d = rng.normal(size=v0.shape)
        eps = 1e-7
        jp = G.objective_c(c, v0 + eps * d, 0.1, steps, DT, window, spos)
        jm = G.objective_c(c, v0 - eps * d, 0.1, steps, DT, window, spos)
        fd = (jp - jm) / (2 * eps)
        an = float((gv * d).sum())
        assert abs(fd - an) <= 1e-6 * abs(an)
    eps = 1e-6
    fd_a = (G.objective_c(c, v0, 0.1 + eps, steps, DT, window, spos)
            - G.objective_c(c, v0, 0.1 - eps, steps, DT, window, spos)) / (2 * eps)
    assert fd_a == pytest.approx(ga, rel=1e-6)
