"""Time-loop parity at the benchmark sizes and on a collapsed column (gpu, slow).

* dp = 0.0025 dam break (6,073,129 particles), 200 steps: the FP32 split form
  and the FP64 form against the FP64 oracle run over the same 200 steps on all
  host cores (the 5M-particle target).  Split form: position within 1e-4 dp,
  velocity within 1e-3 (max|v| + g t), density within 1e-5 relative; FP64
  form: 1e-9 in each.
* dp = 0.005 dam break (875,927 particles), 200 FP32-split steps against the
  oracle, same bars.
* A collapsed column: the oracle runs the dp = 0.02 dam break for 2000 steps
  (0.52 s of flow: the column has fallen to half its height and the surge
  runs along the floor past x = 1.2 m), then PI of both forms on that state
  and 100 steps of both forms from it.  Neighbourhoods there are sparse and
  uneven, unlike the resting lattice of the first steps.

The errors of each field are also what tests/report_split_precision.py
prints.
"""
import os

import numpy as np
import pytest

from sphcases import dam_break
from tests.gpu_common import need_gpu, make_sim

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

G = 9.81
BARS = {"fp32": {"x": 1e-4, "v": 1e-3, "rho": 1e-5},
        "fp64": {"x": 1e-9, "v": 1e-9, "rho": 1e-9}}


@pytest.fixture(scope="module")
def torch_mod():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.lib()
    return oracle


def field_errors(case, st, pos, vel, rho, t_run):
    """Max and RMS error of position (units of dp), velocity (relative to
    max|v| + g t_run, t_run the flow time of the compared run) and density
    (relative) against oracle state st."""
    vscale = np.abs(st.vel).max() + G * t_run
    ex = np.abs(pos - st.pos) / case.params.dp
    ev = np.abs(vel - st.vel) / vscale
    er = np.abs(rho / st.rho - 1.0)
    return {"x_max_dp": float(ex.max()), "x_rms_dp": float(np.sqrt((ex ** 2).mean())),
            "v_max_rel": float(ev.max()), "v_rms_rel": float(np.sqrt((ev ** 2).mean())),
            "rho_max_rel": float(er.max()), "rho_rms_rel": float(np.sqrt((er ** 2).mean()))}


def run_forms(case, st, steps, forms, start=None):
    """Run each GPU form for `steps` steps from the case (or from `start`, an
    oracle state whose previous levels the GPU takes over) and return the
    field errors against oracle state st."""
    t_run = st.time - (start.time if start is not None else 0.0)
    out = {}
    for prec in forms:
        sim = make_sim(case, prec)
        if start is not None:
            sim.set_state(start.pos, start.vel, start.rho, start.velm1, start.rhom1)
        sim.run(steps)
        pos, vel, rho = sim.get_state()
        out[prec] = field_errors(case, st, pos, vel, rho, t_run)
        out[prec]["status"] = sim.status()
        sim.close()
    return out


def split_precision_errors(dp, steps, forms=("fp32", "fp64")):
    """The dam break at dp for `steps` steps: oracle on all host cores, then
    each GPU form from the same initial state."""
    from oracle import oracle
    c = dam_break(dp)
    st = oracle.State(c)
    st.run(steps, nthreads=os.cpu_count() or 1)
    out = {"dp": dp, "particles": c.n, "steps": steps, "sim_time_s": st.time,
           "out_of_grid": st.n_out}
    out.update(run_forms(c, st, steps, forms))
    return out


def _assert_bars(res, forms):
    for prec in forms:
        b = BARS[prec]
        assert res[prec]["status"] == 0, (prec, res[prec])
        assert res[prec]["x_max_dp"] <= b["x"], (prec, res[prec])
        assert res[prec]["v_max_rel"] <= b["v"], (prec, res[prec])
        assert res[prec]["rho_max_rel"] <= b["rho"], (prec, res[prec])


def test_split_precision_5m_200_steps(torch_mod, O):
    """The 5M-particle target: 200 steps of both forms against the oracle."""
    res = split_precision_errors(0.0025, 200)
    assert res["particles"] == 6073129 and res["out_of_grid"] == 0
    _assert_bars(res, ("fp32", "fp64"))


def test_fp32_split_run_1m_200_steps(torch_mod, O):
    res = split_precision_errors(0.005, 200, forms=("fp32",))
    _assert_bars(res, ("fp32",))


@pytest.fixture(scope="module")
def collapsed(O):
    """The dp = 0.02 dam break after 2000 oracle steps (a multiple of the
    Euler period 40, so both sides take their Euler steps together)."""
    c = dam_break(0.02)
    st = O.State(c)
    st.run(2000, nthreads=os.cpu_count() or 1)
    late = type(c)(**{**c.__dict__, "pos": st.pos.copy(), "vel": st.vel.copy(),
                      "rho": st.rho.copy()})
    return c, late, st


def test_collapsed_column_is_collapsed(O, collapsed):
    """The state differs from the resting lattice: the column has fallen, the
    surge has run out along the floor, and fluid cells are sparser."""
    c, late, st = collapsed
    f = late.pos[:c.n_f]
    assert st.time > 0.5 and st.n_out == 0
    assert f[:, 0].max() > 1.2          # initial front at x = 0.4
    assert f[:, 2].max() < 0.2          # initial top at z = 0.3
    _, cnt = np.unique(O.cells(c.params, f), return_counts=True)
    _, cnt0 = np.unique(O.cells(c.params, c.pos[:c.n_f]), return_counts=True)
    assert cnt.mean() < 0.8 * cnt0.mean()
    assert (cnt < 10).mean() > 0.15


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp64", 1e-12)])
def test_pi_collapsed_column(torch_mod, O, collapsed, precision, tol):
    c, late, st = collapsed
    sim = make_sim(late, precision)
    sim.neighbour_list()
    sim.interact()
    ace, ar, mx = sim.forces()
    oace, oar, ovm, ocounts, nout = O.interact(c.params, c.n_f, c.n_b, late.pos, late.vel,
                                                late.rho)
    assert np.array_equal(sim.count_work(), ocounts)
    sa = G + np.abs(oace).max() if precision == "fp32" else np.abs(oace).max()
    assert np.abs(ace - oace).max() <= tol * sa
    assert np.abs(ar - oar).max() <= tol * np.abs(oar).max()
    assert mx[2] == pytest.approx(ovm, rel=10 * tol)
    sim.close()


def test_time_loop_from_collapsed_column(torch_mod, O, collapsed):
    c, late, st = collapsed
    ref = st.copy()
    ref.run(100, nthreads=os.cpu_count() or 1)
    res = run_forms(late, ref, 100, ("fp32", "fp64"), start=st)
    _assert_bars(res, ("fp32", "fp64"))
