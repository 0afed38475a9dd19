"""The neighbour-list call that allocates nothing (sph_neighbour_list_static).

It serves callers that cannot call cudaMalloc -- a solver embedded in a host
program whose allocator owns all device memory, or a loop that must not stall
on an allocation -- by keeping its scratch in a fixed device array inside the
library.  Its outputs must equal those of the context-based neighbour list
(sph_neighbour_list) bit for bit, on consecutive calls that reuse the shared
scratch.  This file is collected last so that a failure here does not hide the
other tests in a run that stops at the first failure.
"""
import numpy as np
import pytest

from sphcases import dam_break, random_cloud
from tests.gpu_common import need_gpu, make_sim

pytestmark = pytest.mark.gpu


def _context_nl(case):
    sim = make_sim(case, "fp32")
    sim.neighbour_list()
    ids, cell, start = sim.neighbour_list_arrays()
    sim.close()
    return ids, cell, start


def _static_nl(torch, case):
    from paper_1110_3711_gb300 import sph
    p = sph.make_params(case.params, "fp32")
    n = case.n_f
    ncells = int(np.prod(_grid(case)))
    pos = torch.from_numpy(np.ascontiguousarray(case.pos[:n])).to("cuda")
    # outputs start as garbage so that every entry must be written
    ids = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    cell = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    start = torch.full((ncells + 2,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    sph.sph_neighbour_list_static(p, n, pos, ids, cell, start, stream)
    torch.cuda.synchronize()
    return (ids.cpu().numpy().view(np.uint32), cell.cpu().numpy().view(np.uint32),
            start.cpu().numpy())


def _grid(case):
    p = case.params
    return [int(np.ceil((p.dom_max[d] - p.dom_min[d]) / p.cell_size)) for d in range(3)]


def test_static_neighbour_list_matches_context_list_on_consecutive_calls():
    torch = need_gpu()
    a = dam_break(0.02)
    b = random_cloud(40000, box=0.25, dp=0.008, n_b=0, seed=3)
    ref_a = _context_nl(a)
    ref_b = _context_nl(b)
    # a, then b (different size and grid), then a again: the scratch left by
    # the previous call must not leak into the next one
    for case, ref in ((a, ref_a), (b, ref_b), (a, ref_a)):
        got = _static_nl(torch, case)
        for g, r in zip(got, ref):
            assert np.array_equal(g.astype(np.int64), r.astype(np.int64))


def _oracle_nl(case, n):
    from oracle import oracle as O
    cell = O.cells(case.params, case.pos[:n])
    order, start = O.cell_list(case.params, cell)
    return order, cell[order], start


def _wide_grid_case(n, dom_max, seed):
    """n random points on a grid of cells of 0.02 m over [0, dom_max]^3, about
    one in ten of them outside the grid (sentinel cell)."""
    from sphcases.dambreak import RunParams, Case
    rng = np.random.default_rng(seed)
    hi = max(dom_max)
    pos = rng.uniform(-0.1, hi + 0.1, size=(n, 3))
    p = RunParams(dp=0.01, h=0.01, cell_size=0.02, mass=1e-3, dom_min=(0.0, 0.0, 0.0),
                  dom_max=tuple(dom_max))
    return Case(params=p, n_f=n, n_b=0, pos=pos, vel=np.zeros_like(pos),
                rho=np.full(n, 1000.0))


def test_static_neighbour_list_at_the_cell_limit():
    """A 256 x 256 x 256 grid (exactly SPH_STATIC_MAX_CELLS cells) with 5,000
    points, some outside it: ids, cells and CellBeginEnd equal the oracle's
    lists, on two calls in a row."""
    torch = need_gpu()
    from paper_1110_3711_gb300 import sph
    c = _wide_grid_case(5000, (5.11, 5.11, 5.11), seed=5)
    assert int(np.prod(_grid(c))) == sph.STATIC_MAX_CELLS
    from oracle import oracle as O
    assert (O.cells(c.params, c.pos) == sph.STATIC_MAX_CELLS).sum() > 100
    ref = _oracle_nl(c, c.n_f)
    for _ in range(2):
        got = _static_nl(torch, c)
        for g, r in zip(got, ref):
            assert np.array_equal(g.astype(np.int64), r.astype(np.int64))


def test_static_neighbour_list_at_the_point_limit():
    """SPH_STATIC_MAX_POINTS random points (radix-sort tiles and scan partials
    at their largest) against the oracle's lists."""
    torch = need_gpu()
    from paper_1110_3711_gb300 import sph
    c = random_cloud(sph.STATIC_MAX_POINTS, box=0.6, dp=0.008, n_b=0, seed=9)
    got = _static_nl(torch, c)
    ref = _oracle_nl(c, c.n_f)
    for g, r in zip(got, ref):
        assert np.array_equal(g.astype(np.int64), r.astype(np.int64))


def _real_size_buffers(torch, p, n):
    from paper_1110_3711_gb300 import sph
    nc = sph.static_grid_cells(p)
    return (torch.zeros((n, 3), dtype=torch.float64, device="cuda"),
            torch.zeros(n, dtype=torch.int32, device="cuda"),
            torch.zeros(n, dtype=torch.int32, device="cuda"),
            torch.zeros(nc + 2, dtype=torch.int32, device="cuda"))


def test_static_neighbour_list_rejects_oversized_input():
    """Beyond either limit the call returns SPH_ERR_TOO_LARGE (-5).  The
    buffers have the full sizes the call would use, so that no order of the
    library's checks could make it touch memory the test does not own."""
    torch = need_gpu()
    from paper_1110_3711_gb300 import sph
    stream = torch.cuda.current_stream().cuda_stream
    c = dam_break(0.02)
    p = sph.make_params(c.params, "fp32")
    n = sph.STATIC_MAX_POINTS + 1
    with pytest.raises(sph.SphError) as e:
        sph.sph_neighbour_list_static(p, n, *_real_size_buffers(torch, p, n), stream)
    assert e.value.code == -5
    w = _wide_grid_case(100, (5.13, 5.11, 5.11), seed=1)
    pw = sph.make_params(w.params, "fp32")
    assert sph.static_grid_cells(pw) > sph.STATIC_MAX_CELLS
    with pytest.raises(sph.SphError) as e:
        sph.sph_neighbour_list_static(pw, 100, *_real_size_buffers(torch, pw, 100), stream)
    assert e.value.code == -5
    torch.cuda.synchronize()


def test_static_neighbour_list_checks_buffers():
    """The binding refuses buffers of the wrong size, type or device before the
    call."""
    torch = need_gpu()
    from paper_1110_3711_gb300 import sph
    c = dam_break(0.02)
    p = sph.make_params(c.params, "fp32")
    n = 100
    pos, ids, cell, start = _real_size_buffers(torch, p, n)
    with pytest.raises(ValueError):
        sph.sph_neighbour_list_static(p, n, pos, ids, cell, start[:-1])
    with pytest.raises(ValueError):
        sph.sph_neighbour_list_static(p, n + 1, pos, ids, cell, start)
    with pytest.raises(TypeError):
        sph.sph_neighbour_list_static(p, n, pos.float(), ids, cell, start)
    with pytest.raises(TypeError):
        sph.sph_neighbour_list_static(p, n, pos.cpu(), ids, cell, start)
