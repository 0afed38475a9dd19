"""The bounding-box filter of the warp PI kernels keeps every candidate the
lockstep test can report as a hit.

The kernels (float32, units of h, item frame) keep a candidate b when
    d2 = fma(dx, dx, fma(dy, dy, dz * dz)) < 4.0004,
    dx = max(box_x0 - b_x, b_x - box_x1, 0)   (same for y, z),
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


def kept(box, bx, by, bz):
    dx = np.maximum(np.maximum(box[0] - bx, bx - box[1]), F(0.0))
    dy = np.maximum(np.maximum(box[2] - by, by - box[3]), F(0.0))
    dz = np.maximum(np.maximum(box[4] - bz, bz - box[5]), F(0.0))
    return fma32(dx, dx, fma32(dy, dy, dz * dz)) < F(4.0004)


def _check(targets, cands):
    ax, ay, az = (targets[:, k][:, None] for k in range(3))
    bx, by, bz = (cands[:, k][None, :] for k in range(3))
    box = [targets[:, 0].min(), targets[:, 0].max(), targets[:, 1].min(),
           targets[:, 1].max(), targets[:, 2].min(), targets[:, 2].max()]
    h = hits(ax, ay, az, bx, by, bz)
    k = kept(box, cands[:, 0], cands[:, 1], cands[:, 2])
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
