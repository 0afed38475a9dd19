"""Cells finer than the support (the paper's finer cells, Section 4.6, optimisation F):
with cell edge h, or any edge in [h, 2h), a particle's support 2h spans two
cells on each side, so the search visits 125 cells as 25 x-runs of 5 cells.

The neighbour list is checked bit for bit against the oracle's list on the
same fine grid.  PI, the exact pair counts, the time loop, the sensor
pressures and the adjoint are checked against the oracle on its own 2h cells:
the set of interacting pairs, and so every result, does not depend on the cell
size.  The candidate counts are checked against the 125-cell sums of the
oracle's fine-grid cell histogram.
"""
import dataclasses

import numpy as np
import pytest

from sphcases import dam_break, random_cloud, small_dam, wall_sensors
from tests.gpu_common import need_gpu, make_sim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    return need_gpu()


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.lib()
    return oracle


def fine(case, factor=0.5):
    """The same case on cells of edge factor * 2h."""
    p = dataclasses.replace(case.params, cell_size=case.params.cell_size * factor)
    return type(case)(**{**case.__dict__, "params": p})


def _perturbed(case, seed):
    rng = np.random.default_rng(seed)
    vel = case.vel.copy()
    vel[:case.n_f] = rng.normal(0, 0.3, size=(case.n_f, 3))
    rho = case.rho * (1 + rng.normal(0, 2e-3, size=case.n))
    return type(case)(**{**case.__dict__, "vel": vel, "rho": rho})


def _block_sums(O, p, pos_targets, H, R):
    """For every target, the sum of histogram H (z, y, x) over the cells within
    R of its own cell (clipped to the grid); -1 for targets outside the grid."""
    nx, ny, nz = (int(v) for v in O.grid(p))
    c = O.cells(p, pos_targets)
    nc = nx * ny * nz
    ok = c < nc
    cx, cy, cz = c % nx, (c // nx) % ny, c // (nx * ny)
    S = np.zeros((nz + 1, ny + 1, nx + 1), np.int64)
    S[1:, 1:, 1:] = H.cumsum(0).cumsum(1).cumsum(2)
    x0, x1 = np.clip(cx - R, 0, nx), np.clip(cx + R + 1, 0, nx)
    y0, y1 = np.clip(cy - R, 0, ny), np.clip(cy + R + 1, 0, ny)
    z0, z1 = np.clip(cz - R, 0, nz), np.clip(cz + R + 1, 0, nz)
    tot = (S[z1, y1, x1] - S[z0, y1, x1] - S[z1, y0, x1] - S[z1, y1, x0]
           + S[z0, y0, x1] + S[z0, y1, x0] + S[z1, y0, x0] - S[z0, y0, x0])
    return np.where(ok, tot, -1)


def _hist(O, p, pos):
    nx, ny, nz = (int(v) for v in O.grid(p))
    c = O.cells(p, pos)
    c = c[c < nx * ny * nz]
    return np.bincount(c, minlength=nx * ny * nz).reshape(nz, ny, nx)


@pytest.mark.parametrize("factor", [0.5, 0.75])
def test_fine_cells_nl_bit_exact(torch_mod, O, factor):
    for c in (dam_break(0.02), random_cloud(5000, box=0.2, dp=0.01, n_b=300, seed=3)):
        cf = fine(c, factor)
        sim = make_sim(cf, "fp64")
        sim.neighbour_list()
        ids, cell, start = sim.neighbour_list_arrays()
        ocell = O.cells(cf.params, cf.pos[:cf.n_f])
        order, ostart = O.cell_list(cf.params, ocell)
        assert np.array_equal(ids.astype(np.int64), order)
        assert np.array_equal(cell.astype(np.int64), ocell[order])
        assert np.array_equal(start.astype(np.int64), ostart)


def test_fine_cells_work_counts_exact(torch_mod, O):
    c = dam_break(0.02)
    cf = fine(c)
    sim = make_sim(cf, "fp64")
    sim.neighbour_list()
    got = sim.count_work()
    _, _, _, counts, _ = O.interact(c.params, c.n_f, c.n_b, c.pos, c.vel, c.rho)
    assert got[1] == counts[1] and got[3] == counts[3]
    p = cf.params
    Hf, Hb = _hist(O, p, c.pos[:c.n_f]), _hist(O, p, c.pos[c.n_f:])
    bf_f = _block_sums(O, p, c.pos[:c.n_f], Hf, 2)
    bb_f = _block_sums(O, p, c.pos[:c.n_f], Hb, 2)
    bf_b = _block_sums(O, p, c.pos[c.n_f:], Hf, 2)
    assert got[0] == int(((bf_f - 1) + bb_f)[bf_f >= 0].sum())
    assert got[2] == int(bf_b[bf_b >= 0].sum())
    # the finer search tests fewer candidates than the 27 cells of edge 2h
    assert got[0] < 0.7 * counts[0]


@pytest.mark.parametrize("precision,kernel,tol", [("fp64", "warp", 1e-12),
                                                  ("fp32", "thread", 2e-5)])
@pytest.mark.parametrize("factor", [0.5, 0.75])
def test_fine_cells_pi_matches_oracle(torch_mod, O, precision, kernel, tol, factor):
    c = _perturbed(dam_break(0.02), 4)
    sim = make_sim(fine(c, factor), precision, pi_kernel=kernel)
    sim.neighbour_list()
    sim.interact()
    ace, ar, mx = sim.forces()
    oace, oar, ovm, _, _ = O.interact(c.params, c.n_f, c.n_b, c.pos, c.vel, c.rho)
    scale = np.abs(oace).max() if precision == "fp64" else 9.81 + np.abs(oace).max()
    assert np.abs(ace - oace).max() <= tol * scale
    assert np.abs(ar - oar).max() <= tol * np.abs(oar).max()
    assert mx[2] == pytest.approx(ovm, rel=max(tol, 1e-13))


def test_fine_cells_fp64_time_loop(torch_mod, O):
    """60 steps (an Euler step included) on cells of edge h against the oracle."""
    c = dam_break(0.02)
    sim = make_sim(fine(c), "fp64")
    st = O.State(c)
    for _ in range(60):
        sim.step()
        st.step(nthreads=8)
    pos, vel, rho = sim.get_state()
    vscale = np.abs(st.vel).max() + 9.81 * st.time
    assert np.abs(pos - st.pos).max() <= 1e-9 * c.params.dp
    assert np.abs(vel - st.vel).max() <= 1e-9 * vscale
    assert np.abs(rho / st.rho - 1).max() <= 1e-9


def test_fine_cells_fp32_thread_time_loop(torch_mod, O):
    c = dam_break(0.02)
    sim = make_sim(fine(c), "fp32", pi_kernel="thread")
    st = O.State(c)
    for _ in range(60):
        sim.step()
        st.step(nthreads=8)
    pos, vel, rho = sim.get_state()
    vscale = np.abs(st.vel).max() + 9.81 * st.time
    assert np.abs(pos - st.pos).max() <= 1e-4 * c.params.dp
    assert np.abs(vel - st.vel).max() <= 1e-3 * vscale
    assert np.abs(rho / st.rho - 1).max() <= 1e-5


def test_fine_cells_rejected_by_warp_and_fastcells(torch_mod):
    from paper_1110_3711_gb300 import sph
    cf = fine(dam_break(0.02))
    for kernel in ("warp", "thread_fastcells"):
        with pytest.raises(sph.SphError):
            make_sim(cf, "fp32", pi_kernel=kernel)


def test_fine_cells_adjoint_matches_oracle_gradient(torch_mod):
    """The adjoint's pair walks and the sensor search on cells of edge h give
    the gradient of the oracle (on its 2h cells)."""
    from oracle import grad as G
    from paper_1110_3711_gb300.autograd import DamBreakRun, objective
    torch = torch_mod
    steps, dt, window = 20, 2e-4, 5
    c = small_dam(0.02)
    spos = wall_sensors(c, wall="back", n_y=2, n_z=2, z_top=0.12)
    Jo, gvo, gao = G.gradient(c, c.vel[:c.n_f], 0.1, steps, dt, window, spos)
    run = DamBreakRun(fine(c), steps, dt, window, spos, checkpoint_every=6)
    v0 = torch.tensor(c.vel[:c.n_f], dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(0.1, dtype=torch.float64, device="cuda", requires_grad=True)
    J = objective(v0, a, run)
    J.backward()
    assert float(J.detach()) == pytest.approx(Jo, rel=1e-12)
    g = v0.grad.cpu().numpy()
    assert np.abs(g - gvo).max() <= 1e-8 * np.abs(gvo).max()
    assert float(a.grad) == pytest.approx(gao, rel=1e-8)
