"""Golden spline values and pins of the oracle's sensor interpolation."""
import math
import os

import numpy as np
import pytest

from sphcases import dam_break, uniform_block, wall_sensors

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cubic_spline_values.txt")


def test_spline_matches_published_values(oracle_lib):
    rows = np.loadtxt(GOLDEN)
    h = 0.02
    for q, w, dw in rows:
        r = q * h
        assert math.pi * h ** 3 * oracle_lib.kernel_w(h, r) == pytest.approx(w, abs=1e-15)
        if 0 < q < 2:
            # dW/dq = h dW/dr = h F r
            got = math.pi * h ** 3 * h * oracle_lib.kernel_f(h, r) * r
            assert got == pytest.approx(dw, rel=1e-13)


def test_sensor_reproduces_uniform_pressure(oracle_lib):
    """Shepard normalisation: a uniform density gives its own pressure exactly."""
    c = uniform_block(10, 0.01)
    rho = np.full(c.n, 1004.0)
    P0 = oracle_lib.pressure(c.params, 1004.0)
    spos = np.array([[0.05, 0.05, 0.05], [0.031, 0.047, 0.062], [0.01, 0.02, 0.09]])
    out = oracle_lib.sensor_pressure(c.params, c.n_f, c.pos, rho, spos)
    assert np.allclose(out, P0, rtol=1e-13)


def test_sensor_hydrostatic_wall(oracle_lib):
    """Sensors in the hydrostatic column read ~rho0 g depth; above it, 0."""
    c = dam_break(0.01)
    spos = wall_sensors(c, wall="back")
    out = oracle_lib.sensor_pressure(c.params, c.n_f, c.pos, c.rho, spos)
    depth = c.meta["H"] - spos[:, 2]
    inside = depth > 2 * c.params.h
    assert np.allclose(out[inside], 1000 * 9.81 * depth[inside], rtol=2e-2)
    far = wall_sensors(c, wall="far")
    assert (oracle_lib.sensor_pressure(c.params, c.n_f, c.pos, c.rho, far) == 0).all()
