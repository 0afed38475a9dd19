"""Pins of the oracle's cubic spline kernel and Tait equation of state (Table 1).

Each check compares the oracle with something other than its own formula: a
quadrature, a finite difference, a lattice moment, or the hydrostatic state the
input recipe builds.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from sphcases import dam_break, uniform_block

H = 0.015


def test_kernel_normalised(oracle_lib):
    """4 pi int_0^{2h} W(r) r^2 dr = 1 (unit normalisation of the 3D kernel)."""
    O = oracle_lib
    val, err = integrate.quad(lambda r: 4 * math.pi * r * r * O.kernel_w(H, r), 0.0, 2 * H,
                              points=[H], epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-10


def test_kernel_compact_support(oracle_lib):
    O = oracle_lib
    assert O.kernel_w(H, 2 * H) == 0.0
    assert O.kernel_f(H, 2 * H) == 0.0
    assert O.kernel_w(H, 3 * H) == 0.0
    # W and grad W go to zero continuously at q = 2
    assert O.kernel_w(H, 2 * H * (1 - 1e-6)) < 1e-15 / H ** 3
    assert abs(O.kernel_f(H, 2 * H * (1 - 1e-6))) * H ** 5 < 1e-10
    assert O.kernel_w(H, 0.0) == pytest.approx(1.0 / (math.pi * H ** 3), rel=1e-15)


@pytest.mark.parametrize("q", [0.05, 0.3, 0.77, 0.999, 1.001, 1.4, 1.9])
def test_gradient_factor_is_dw_dr_over_r(oracle_lib, q):
    """grad_a W = F r_ab  <=>  F r = dW/dr (central difference of W)."""
    O = oracle_lib
    r = q * H
    eps = 1e-6 * H
    dwdr = (O.kernel_w(H, r + eps) - O.kernel_w(H, r - eps)) / (2 * eps)
    assert O.kernel_f(H, r) * r == pytest.approx(dwdr, rel=2e-7, abs=1e-9 / H ** 4)


def test_kernel_c2_at_q1(oracle_lib):
    """W, dW/dr and d2W/dr2 are continuous at q = 1 (cubic spline is C2)."""
    O = oracle_lib
    e = 1e-7 * H
    w = lambda r: O.kernel_w(H, r)
    d1 = lambda r: O.kernel_f(H, r) * r
    assert w(H - e) == pytest.approx(w(H + e), rel=1e-6)
    assert d1(H - e) == pytest.approx(d1(H + e), rel=1e-6)
    k = 1e-4 * H
    d2m = (d1(H - k) - d1(H - 2 * k)) / k
    d2p = (d1(H + 2 * k) - d1(H + k)) / k
    assert d2m == pytest.approx(d2p, rel=2e-3)


def _lattice_offsets(dp, h):
    n = int(math.ceil(2 * h / dp)) + 1
    g = np.arange(-n, n + 1) * dp
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    off = np.stack([X.ravel(), Y.ravel(), Z.ravel()], -1)
    r = np.linalg.norm(off, axis=1)
    return off[r < 2 * h], r[r < 2 * h]


def test_lattice_partition_of_unity(oracle_lib):
    """sum_b W_ab dp^3 ~ 1 for an interior particle of the cubic lattice."""
    O = oracle_lib
    dp = 0.01
    h = 0.866 * math.sqrt(3) * dp
    off, r = _lattice_offsets(dp, h)
    s = sum(O.kernel_w(h, ri) for ri in r) * dp ** 3
    assert abs(s - 1.0) < 1e-2


def test_lattice_gradient_moment(oracle_lib):
    """sum_b (m/rho) r_ab (x) grad_a W_ab ~ -I on the lattice (integration by parts
    of int r (x) grad W dV = -I): pins the sign and scale of F against W."""
    O = oracle_lib
    dp = 0.01
    h = 0.866 * math.sqrt(3) * dp
    off, r = _lattice_offsets(dp, h)
    M = np.zeros((3, 3))
    for o, ri in zip(off, r):
        if ri == 0:
            continue
        # r_ab = x_a - x_b = -o for neighbour at offset o
        rab = -o
        M += dp ** 3 * np.outer(rab, O.kernel_f(h, ri) * rab)
    assert np.allclose(M, -np.eye(3), atol=2e-2)


def test_eos_zero_at_rest_density(oracle_lib):
    c = dam_break(0.02)
    assert oracle_lib.pressure(c.params, 1000.0) == 0.0
    assert oracle_lib.sound(c.params, 1000.0) == pytest.approx(c.params.c0, rel=1e-15)


@pytest.mark.parametrize("rho", [990.0, 1000.0, 1003.0, 1030.0])
def test_sound_speed_is_sqrt_dp_drho(oracle_lib, rho):
    """c(rho)^2 = dP/drho (central difference of the oracle's Tait pressure)."""
    O = oracle_lib
    p = dam_break(0.02).params
    e = 1e-4
    dpdrho = (O.pressure(p, rho + e) - O.pressure(p, rho - e)) / (2 * e)
    assert O.sound(p, rho) ** 2 == pytest.approx(dpdrho, rel=1e-7)


def test_initial_state_is_hydrostatic(oracle_lib):
    """Tait pressure of the initial density equals rho0 g depth (the recipe's
    hydrostatic column) to round-off."""
    O = oracle_lib
    c = dam_break(0.02)
    H = c.meta["H"]
    idx = np.arange(0, c.n, 97)
    for i in idx:
        depth = max(0.0, H - c.pos[i, 2])
        P = O.pressure(c.params, c.rho[i])
        assert P == pytest.approx(1000.0 * 9.81 * depth, rel=1e-11, abs=1e-9)
