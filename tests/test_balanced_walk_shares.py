"""Host check of the share arithmetic of the balanced hit walk of the float64
work-item kernels (warp_items.cuh, for_each_hit_balanced).

The hits of a tested set are taken in target order (target t = lane t, c_t
hits) and dealt to the 32 lanes in consecutive shares of sh = ceil(T / 32);
lane L walks global hits [L sh, min((L + 1) sh, T)), writing one partial sum
per target it touches to slot L + t, and target t adds the slots of lanes
first_t / sh .. last_t / sh.  The claims the kernel relies on: every hit is
walked once, the slots written in one set are distinct (so no partial sum
overwrites another) and lie in [0, 63), and each target's combine range is
exactly the set of lanes that wrote a partial sum for it."""
import numpy as np


def shares(counts):
    counts = np.asarray(counts)
    incl = np.cumsum(counts)
    T = int(incl[-1])
    if T == 0:
        return {}, {}
    sh = (T + 31) // 32
    written = {}     # slot -> (lane, target)
    walked = np.zeros(T, int)
    for L in range(32):
        g0, g1 = min(L * sh, T), min(L * sh + sh, T)
        for g in range(g0, g1):
            t = int(np.searchsorted(incl, g, side="right"))   # smallest t with incl[t] > g
            walked[g] += 1
            slot = L + t
            assert written.get(slot, (L, t)) == (L, t), "slot shared by two partial sums"
            written[slot] = (L, t)
    assert np.all(walked == 1)
    combine = {}
    for t, c in enumerate(counts):
        if c > 0:
            first, last = int(incl[t] - c), int(incl[t] - 1)
            combine[t] = list(range(first // sh, last // sh + 1))
    return written, combine


def test_shares_cover_every_hit_once_with_distinct_slots():
    rng = np.random.default_rng(3)
    cases = [rng.poisson(60, size=32), np.r_[rng.poisson(100, 27), np.zeros(5, int)],
             np.r_[np.zeros(31, int), [7]], np.ones(32, int), np.r_[[1000], np.zeros(31, int)],
             rng.integers(0, 3, size=32)]
    for _ in range(200):
        cases.append(rng.integers(0, 200, size=32) * (rng.random(32) < 0.8))
    for counts in cases:
        written, combine = shares(counts)
        assert all(0 <= s < 63 for s in written)
        for t, lanes in combine.items():
            got = sorted(L for (L, tt) in written.values() if tt == t)
            assert got == lanes
