"""Pins of the oracle's neighbour list (cell-linked list, Sections 2 and 4.1).

Brute force O(N^2) on small inputs, the definition of the cell of a point,
the (cell, id) order, the CellBeginEnd semantics of Fig. 8 (empty cells have
begin == end) and the equivalence of the 27 cells with 9 x-runs (Section 4.4).
"""
import numpy as np
import pytest

from sphcases import random_cloud, dam_break


def _brute_pairs(case):
    """All ordered (a, b), a != b, r < 2h, not boundary-boundary, by brute force."""
    p = case.params
    pos = case.pos
    d = pos[:, None, :] - pos[None, :, :]
    r2 = np.einsum("ijk,ijk->ij", d, d)
    mask = r2 < 4.0 * p.h * p.h
    np.fill_diagonal(mask, False)
    isb = np.arange(case.n) >= case.n_f
    mask &= ~(isb[:, None] & isb[None, :])
    a, b = np.nonzero(mask)
    return set(zip(a.tolist(), b.tolist()))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pairs_match_brute_force(oracle_lib, seed):
    c = random_cloud(1500, box=0.12, dp=0.01, n_b=300, seed=seed)
    pa, pb = oracle_lib.pairs(c.params, c.n_f, c.n_b, c.pos)
    got = set(zip(pa.tolist(), pb.tolist()))
    assert len(got) == len(pa)
    assert got == _brute_pairs(c)


def test_cell_contains_point(oracle_lib):
    c = random_cloud(3000, box=0.2, dp=0.013, seed=4)
    p = c.params
    dims = oracle_lib.grid(p)
    cell = oracle_lib.cells(p, c.pos)
    nc = int(dims.prod())
    assert (cell < nc).all()
    cx = cell % dims[0]
    cy = (cell // dims[0]) % dims[1]
    cz = cell // (dims[0] * dims[1])
    ci = np.stack([cx, cy, cz], 1)
    lo = np.asarray(p.dom_min) + ci * p.cell_size
    hi = lo + p.cell_size
    tol = 1e-12
    assert (c.pos >= lo - tol).all() and (c.pos < hi + tol).all()


def test_out_of_grid_gets_sentinel(oracle_lib):
    c = random_cloud(200, box=0.1, dp=0.01, seed=5)
    p = c.params
    pos = c.pos.copy()
    pos[3] = [-1.0, 0.05, 0.05]
    pos[7] = [0.05, 0.05, 5.0]
    pos[9] = [np.nan, 0.0, 0.0]
    dims = oracle_lib.grid(p)
    cell = oracle_lib.cells(p, pos)
    nc = int(dims.prod())
    assert cell[3] == nc and cell[7] == nc and cell[9] == nc
    assert (np.delete(cell, [3, 7, 9]) < nc).all()


def test_list_order_and_ranges(oracle_lib):
    c = dam_break(0.02)
    p = c.params
    dims = oracle_lib.grid(p)
    nc = int(dims.prod())
    cell = oracle_lib.cells(p, c.pos[:c.n_f])
    order, start = oracle_lib.cell_list(p, cell)
    # a bijection sorted by (cell, id)
    assert np.array_equal(np.sort(order), np.arange(c.n_f))
    key = cell[order] * (c.n_f + 1) + order
    assert (np.diff(key) > 0).all()
    # CellBeginEnd: start is the exclusive prefix of the cell histogram
    hist = np.bincount(cell, minlength=nc + 1)
    assert np.array_equal(np.diff(start), hist[:nc + 1])
    assert start[0] == 0 and start[-1] == c.n_f
    for k in range(0, nc, 7):
        members = order[start[k]:start[k + 1]]
        assert (cell[members] == k).all()
        if hist[k] == 0:
            assert start[k] == start[k + 1]
    assert (hist == 0).sum() > 0  # the test exercises empty cells


def test_nine_x_runs_equal_27_cells(oracle_lib):
    """Cells x-1, x, x+1 of one (y, z) row are contiguous in the sorted order, so
    the 27 cells are 9 index ranges (Section 4.4, Fig. 10)."""
    c = dam_break(0.02)
    p = c.params
    dims = oracle_lib.grid(p)
    cell = oracle_lib.cells(p, c.pos[:c.n_f])
    order, start = oracle_lib.cell_list(p, cell)
    nx, ny, nz = (int(v) for v in dims)
    occupied = np.unique(cell)
    for cc in occupied[::5]:
        cx, cy, cz = cc % nx, (cc // nx) % ny, cc // (nx * ny)
        via27, via9 = [], []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                y, z = cy + dy, cz + dz
                if not (0 <= y < ny and 0 <= z < nz):
                    continue
                x0, x1 = max(cx - 1, 0), min(cx + 1, nx - 1)
                for x in range(x0, x1 + 1):
                    k = x + nx * (y + ny * z)
                    via27.extend(order[start[k]:start[k + 1]].tolist())
                k0 = x0 + nx * (y + ny * z)
                k1 = x1 + nx * (y + ny * z)
                via9.extend(order[start[k0]:start[k1 + 1]].tolist())
        assert via27 == via9


def test_search_refuses_cells_below_support(oracle_lib):
    """The oracle visits the 27 cells around a particle, which hold its support
    only for cells of edge >= 2h; a finer grid is refused rather than searched
    incompletely (its cell lists stay available)."""
    import dataclasses
    c = random_cloud(200, box=0.1, dp=0.01, n_b=20, seed=4)
    p = dataclasses.replace(c.params, cell_size=c.params.h)
    with pytest.raises(ValueError):
        oracle_lib.pairs(p, c.n_f, c.n_b, c.pos)
    with pytest.raises(ValueError):
        oracle_lib.interact(p, c.n_f, c.n_b, c.pos, c.vel, c.rho)
    cell = oracle_lib.cells(p, c.pos)
    order, start = oracle_lib.cell_list(p, cell)
    assert np.array_equal(np.sort(order), np.arange(c.n))
