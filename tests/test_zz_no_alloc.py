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


def test_static_neighbour_list_rejects_oversized_input():
    torch = need_gpu()
    from paper_1110_3711_gb300 import sph
    c = dam_break(0.02)
    p = sph.make_params(c.params, "fp32")
    dummy = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(sph.SphError) as e:
        sph.sph_neighbour_list_static(p, sph.STATIC_MAX_POINTS + 1, dummy, dummy, dummy, dummy,
                                      torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -5
