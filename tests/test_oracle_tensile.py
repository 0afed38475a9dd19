"""Pins of the oracle's tensile correction (Monaghan 2000; the "tensil" array of
Table 3), a variant that is off in the dam-break configurations."""
import copy

import numpy as np
import pytest

from sphcases import uniform_block


def _pair_case(distance, rho):
    c = uniform_block(2, 0.01)
    pos = np.array([[0.05, 0.05, 0.05], [0.05 + distance, 0.05, 0.05]])
    return c.params, pos, np.zeros((2, 3)), np.full(2, rho)


def _with(p, **kw):
    q = copy.copy(p)
    for k, v in kw.items():
        setattr(q, k, v)
    return q


def test_tensile_off_by_default(oracle_lib):
    p, pos, vel, rho = _pair_case(0.012, 995.0)
    a0, *_ = oracle_lib.interact(p, 2, 0, pos, vel, rho)
    a1, *_ = oracle_lib.interact(_with(p, tensile_eps=0.0, tensile_pos=0.0), 2, 0, pos, vel, rho)
    assert np.array_equal(a0, a1)


def test_tensile_repels_under_negative_pressure(oracle_lib):
    """P < 0 pulls two particles together; the correction adds a repulsion that
    is linear in eps and scales like (W(r)/W(dp))^n F(r) r with distance."""
    O = oracle_lib
    p = _pair_case(0.012, 995.0)[0]
    extra = {}
    for d in (0.012, 0.016):
        _, pos, vel, rho = _pair_case(d, 995.0)
        off, *_ = O.interact(p, 2, 0, pos, vel, rho)
        on1, *_ = O.interact(_with(p, tensile_eps=0.2), 2, 0, pos, vel, rho)
        on2, *_ = O.interact(_with(p, tensile_eps=0.4), 2, 0, pos, vel, rho)
        e1, e2 = on1 - off, on2 - off
        assert off[0, 0] > 0          # particle 0 is pulled towards +x (attraction)
        assert e1[0, 0] < 0           # the correction pushes it back
        assert np.allclose(e1[0], -e1[1])
        assert np.allclose(e2, 2 * e1, rtol=1e-12, atol=0)
        extra[d] = e1[0, 0]
    h = p.h
    wr = lambda r: O.kernel_w(h, r) / O.kernel_w(h, p.dp)
    fr = lambda r: O.kernel_f(h, r) * r
    expect = (wr(0.012) ** 4 * fr(0.012)) / (wr(0.016) ** 4 * fr(0.016))
    assert extra[0.012] / extra[0.016] == pytest.approx(expect, rel=1e-12)


def test_tensile_positive_pressures_and_momentum(oracle_lib):
    """With both pressures positive the correction is tensile_pos times the
    pressure terms; a closed fluid with mixed signs still conserves momentum."""
    O = oracle_lib
    p, pos, vel, rho = _pair_case(0.012, 1004.0)
    off, *_ = O.interact(p, 2, 0, pos, vel, rho)
    on, *_ = O.interact(_with(p, tensile_pos=0.01), 2, 0, pos, vel, rho)
    prr = 2 * O.pressure(p, 1004.0) / 1004.0 ** 2
    wr = O.kernel_w(p.h, 0.012) / O.kernel_w(p.h, p.dp)
    assert np.allclose(on - off, off * (0.01 * prr * wr ** 4) / prr, rtol=1e-10)
    c = uniform_block(8, 0.01, seed=5, vel_sigma=0.2, rho_sigma=0.01, jitter=0.2)
    q = _with(c.params, tensile_eps=0.2, tensile_pos=0.01)
    ace, *_ = O.interact(q, c.n_f, 0, c.pos, c.vel, c.rho)
    tot = (q.mass * ace).sum(0)
    assert np.abs(tot).max() <= 1e-13 * (q.mass * np.abs(ace)).sum()
