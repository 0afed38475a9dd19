"""The float32 pair terms evaluate the artificial-viscosity factor of Monaghan's
Pi_ab (Table 1, ref. [28]) without a reciprocal.

Pi_ab = -alpha c_bar mu_ab / rho_bar with c_bar = (c_a + c_b)/2 and
rho_bar = (rho_a + rho_b)/2.  With the Tait sound speed of gamma = 7,
c = c0 (rho/rho0)^3, and a^3 + b^3 = (a + b)(a^2 - a b + b^2):

    -alpha (c_a + c_b) / (rho_a + rho_b) = kcf (rho_a^2 - rho_a rho_b + rho_b^2),
    kcf = -alpha c0 / rho0^3,

which the kernels (csrc/pair32.cuh) evaluate as kcf * fma(rho_b, rho_b - rho_a,
rho_a^2) in float32.  These checks pin the identity against the literal form of
the oracle in float64 and bound the float32 evaluation's error over the density
range of a dam break (and beyond), so that a wrong sign, a missing term or a
swapped density fails here.  Host arithmetic only."""
import numpy as np

F = np.float32
ALPHA, C0, RHO0, GAMMA = 0.1, 10.0 * np.sqrt(9.81 * 0.3), 1000.0, 7.0


def literal(ra, rb):
    ca = C0 * (ra / RHO0) ** ((GAMMA - 1.0) / 2.0)
    cb = C0 * (rb / RHO0) ** ((GAMMA - 1.0) / 2.0)
    cbar, rbar = 0.5 * (ca + cb), 0.5 * (ra + rb)
    return -ALPHA * cbar / rbar


def kernel32(ra, rb):
    kcf = F(-ALPHA * C0 / RHO0 ** 3)
    ra, rb = ra.astype(F), rb.astype(F)
    ra2 = ra * ra
    d = rb - ra                                   # exact for densities within a factor 2
    # fma(rb, d, ra2) rounded once: the float64 product of two float32 values is exact
    t = (rb.astype(np.float64) * d.astype(np.float64) + ra2.astype(np.float64)).astype(F)
    return kcf * t


def test_identity_in_float64():
    rng = np.random.default_rng(0)
    ra = rng.uniform(500.0, 2000.0, 10000)
    rb = rng.uniform(500.0, 2000.0, 10000)
    kcf = -ALPHA * C0 / RHO0 ** 3
    poly = kcf * (ra * ra - ra * rb + rb * rb)
    np.testing.assert_allclose(poly, literal(ra, rb), rtol=1e-13)


def test_float32_evaluation_error():
    rng = np.random.default_rng(1)
    # densities of a dam break stay within a few per cent of rho0; test a wide band
    ra = rng.uniform(900.0, 1100.0, 20000)
    rb = ra * rng.uniform(0.95, 1.05, 20000)
    ref = literal(ra, rb)
    got = kernel32(ra, rb).astype(np.float64)
    rel = np.abs(got / ref - 1.0)
    assert rel.max() < 4e-7, rel.max()


def test_float32_equal_densities():
    # rho_a = rho_b: the factor is -alpha c(rho) / rho
    r = np.linspace(950.0, 1050.0, 101)
    got = kernel32(r, r).astype(np.float64)
    ref = -ALPHA * C0 * (r / RHO0) ** 3 / r
    np.testing.assert_allclose(got, ref, rtol=4e-7)


def test_mistakes_are_caught():
    rng = np.random.default_rng(2)
    ra = rng.uniform(950.0, 1050.0, 1000)
    rb = rng.uniform(950.0, 1050.0, 1000)
    ref = literal(ra, rb)
    kcf = -ALPHA * C0 / RHO0 ** 3
    wrong = {
        "plus middle term": kcf * (ra * ra + ra * rb + rb * rb),
        "no middle term": kcf * (ra * ra + rb * rb),
        "cubes not divided": kcf * (ra ** 3 + rb ** 3),
        "c of a only": -ALPHA * C0 * (ra / RHO0) ** 3 / (0.5 * (ra + rb)),
    }
    for name, w in wrong.items():
        assert np.abs(w / ref - 1.0).max() > 1e-4, name
