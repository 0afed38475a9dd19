"""The bounding-box filter of the warp PI kernels keeps every candidate the
lockstep test can report as a hit.

The kernels (float32, units of h, item frame) keep a candidate b when
    d2 = fma(dx, dx, fma(dy, dy, dz * dz)) < 4.0004,
    dx = max(|b_x - c_x| - e_x, 0)   (same for y, z),
with the box's centre c_x = (box_x0 + box_x1) / 2 and half extent
e_x = (box_x1 - box_x0) / 2, each rounded to float32,
and the lockstep test reports a hit of target a when
    fma(-2 a_x, b_x, fma(-2 a_y, b_y, fma(-2 a_z, b_z, |b|^2))) - (4 - |a|^2) < 0.
A target lies inside the box, so |a - b| >= distance(b, box); the test below
evaluates both expressions with float32 rounding of every operation (a fused
multiply-add rounded once) on random and on adversarial inputs (candidates at
distance 2 +- a few ulp from a target) and checks that no hit is dropped.
Host arithmetic only: it pins the margin argument, not the kernel code."""
import numpy as np

F = np.float32


def fma32(a, b, c):
    # a*b is exact in float64 for float32 a, b; the float64 sum then one
    # rounding to float32 (a second rounding can only matter at a tie, far
    # inside the 4e-4 margin)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def hits(ax, ay, az, bx, by, bz):
    thr = F(4.0) - fma32(ax, ax, fma32(ay, ay, az * az))
    w = fma32(bx, bx, fma32(by, by, bz * bz))
    t = fma32(F(-2.0) * ax, bx, fma32(F(-2.0) * ay, by, fma32(F(-2.0) * az, bz, w)))
    return (t - thr) < 0


def kept(box, bx, by, bz, thr=F(4.0004)):
    d = []
    for k, b in enumerate((bx, by, bz)):
        lo, hi = F(box[2 * k]), F(box[2 * k + 1])
        c = F(0.5) * (lo + hi)
        e = F(0.5) * (hi - lo)
        d.append(np.maximum(np.abs(b - c) - e, F(0.0)))
    dx, dy, dz = d
    return fma32(dx, dx, fma32(dy, dy, dz * dz)) < thr


def _check(targets, cands, thr=F(4.0004)):
    ax, ay, az = (targets[:, k][:, None] for k in range(3))
    bx, by, bz = (cands[:, k][None, :] for k in range(3))
    box = [targets[:, 0].min(), targets[:, 0].max(), targets[:, 1].min(),
           targets[:, 1].max(), targets[:, 2].min(), targets[:, 2].max()]
    h = hits(ax, ay, az, bx, by, bz)
    k = kept(box, cands[:, 0], cands[:, 1], cands[:, 2], thr)
    assert not np.any(h & ~k[None, :]), "a hit was dropped by the box filter"
    return int(h.sum()), int(k.sum())


def test_random_items_lose_no_hit():
    rng = np.random.default_rng(0)
    for _ in range(40):
        nt = int(rng.integers(1, 33))
        # targets in the cell [0, 2)^3 (cells of 2h), candidates in the 27 cells
        targets = rng.uniform(0.0, 2.0, size=(nt, 3)).astype(F)
        cands = rng.uniform(-2.0, 4.0, size=(2000, 3)).astype(F)
        nh, nk = _check(targets, cands)
        assert nk < len(cands)   # the filter drops something


def test_candidates_on_the_support_sphere_lose_no_hit():
    rng = np.random.default_rng(1)
    for _ in range(20):
        nt = int(rng.integers(1, 33))
        targets = rng.uniform(0.0, 2.0, size=(nt, 3)).astype(F)
        # candidates at distance 2 (+- a few ulp) from random targets
        a = targets[rng.integers(0, nt, size=4000)].astype(np.float64)
        u = rng.normal(size=(4000, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        r = 2.0 * (1.0 + rng.uniform(-4e-7, 4e-7, size=(4000, 1)))
        cands = (a + r * u).astype(F)
        nh, _ = _check(targets, cands)
        assert nh > 0


def test_margin_is_needed():
    # a threshold below the support radius drops hits of candidates on the
    # support sphere, so the check above can fail
    rng = np.random.default_rng(2)
    targets = rng.uniform(0.0, 2.0, size=(1, 3)).astype(F)
    u = rng.normal(size=(4000, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    cands = (targets[0].astype(np.float64) + 1.99999 * u).astype(F)
    try:
        _check(targets, cands, thr=F(3.9999))
    except AssertionError:
        return
    raise AssertionError("a threshold of 3.9999 kept every hit")
