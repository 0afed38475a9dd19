"""Parity at the benchmark sizes, in the configuration bench.py times.

dp = 0.005 dam break (875,927 particles) and dp = 0.0025 (6,073,129):
the neighbour list bit-exact against the oracle's lists; PI against the
oracle on every particle (1M) or on a uniform sample of targets the oracle
evaluates one by one (5M); a short FP32-split run against the oracle run.
"""
import numpy as np
import pytest

from sphcases import dam_break
from tests.gpu_common import need_gpu, make_sim

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def torch_mod():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.lib()
    return oracle


def _perturbed(case, seed):
    rng = np.random.default_rng(seed)
    vel = case.vel.copy()
    vel[:case.n_f] = rng.normal(0, 0.3, size=(case.n_f, 3))
    rho = case.rho * (1 + rng.normal(0, 1e-3, size=case.n))
    return type(case)(**{**case.__dict__, "vel": vel, "rho": rho})


def _nl_bit_exact(O, sim, case):
    ids, cell, start = sim.neighbour_list_arrays()
    p = case.params
    ocell = O.cells(p, case.pos[:case.n_f])
    order, ostart = O.cell_list(p, ocell)
    assert np.array_equal(ids.astype(np.int64), order)
    assert np.array_equal(cell.astype(np.int64), ocell[order])
    assert np.array_equal(start.astype(np.int64), ostart)


@pytest.mark.parametrize("dp", [0.005, 0.0025])
def test_neighbour_list_bit_exact_full_size(torch_mod, O, dp):
    c = dam_break(dp)
    sim = make_sim(c, "fp32")
    sim.neighbour_list()
    _nl_bit_exact(O, sim, c)
    got = sim.count_work()
    if dp == 0.005:
        _, _, _, counts, _ = O.interact(c.params, c.n_f, c.n_b, c.pos, c.vel, c.rho)
        assert np.array_equal(got, counts)


@pytest.mark.parametrize("pi_kernel", ["warp", "warp_sym"])
def test_pi_fp32_all_particles_1m(torch_mod, O, pi_kernel):
    c = _perturbed(dam_break(0.005), 1)
    sim = make_sim(c, "fp32", pi_kernel=pi_kernel)
    sim.neighbour_list()
    sim.interact()
    ace, ar, mx = sim.forces()
    oace, oar, ovm, _, _ = O.interact(c.params, c.n_f, c.n_b, c.pos, c.vel, c.rho)
    assert np.abs(ace - oace).max() / (9.81 + np.abs(oace).max()) < 2e-5
    assert np.abs(ar - oar).max() / np.abs(oar).max() < 2e-5
    assert mx[2] == pytest.approx(ovm, rel=1e-5)


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp64", 1e-12)])
def test_pi_sampled_targets_5m(torch_mod, O, precision, tol):
    c = _perturbed(dam_break(0.0025), 2)
    sim = make_sim(c, precision)
    sim.neighbour_list()
    sim.interact()
    ace, ar, _ = sim.forces()
    stride = 61
    oace, oar, _, _, _, _ = O.interact_sampled(c.params, c.n_f, c.n_b, c.pos, c.vel, c.rho, stride)
    idx = np.arange(0, c.n, stride)
    fi = idx[idx < c.n_f]
    sa = 9.81 + np.abs(oace[fi]).max() if precision == "fp32" else np.abs(oace[fi]).max()
    assert np.abs(ace[fi] - oace[fi]).max() <= tol * sa
    assert np.abs(ar[idx] - oar[idx]).max() <= tol * np.abs(oar[idx]).max()
