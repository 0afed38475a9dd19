"""The hand-written adjoint (sph_adjoint_step, sph_sensor_adjoint) behind the
torch.autograd.Function, against the gradient oracle and finite differences.

Case: the small dam break (180 fluid + 1,304 boundary particles, dp = 0.02 m),
fixed dt = 2e-4 s, 45 steps (so the Euler step at step 39 is included),
objective = mean pressure of 4 sensors on the wall behind the column over the
last 10 states, seeded N(0, 0.05 m/s) initial velocity.  Bars: J within
1e-12, gradients within 1e-8 of the oracle (both float64; the remaining
difference is summation order); checkpoint interval changes nothing; central
differences of the GPU forward within 5e-6: a small eps is needed because the
viscosity switch is C0 (see the oracle's tests), and at eps = 1e-7 the FD
quotient's round-off floor is about 1e-16 * J / (2 eps |dJ/dd|) ~ 1.3e-6.
"""
import numpy as np
import pytest

from sphcases import small_dam, wall_sensors, dam_break
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu

STEPS, DT, WINDOW = 45, 2e-4, 10


@pytest.fixture(scope="module")
def torch_mod():
    return need_gpu()


def _case():
    c = small_dam(0.02)
    return c, wall_sensors(c, wall="back", n_y=2, n_z=2, z_top=0.12)


def _gpu_grad(torch, case, spos, k, vel0=None, alpha=0.1, steps=STEPS, window=WINDOW, dt=DT):
    from paper_1110_3711_gb300.autograd import DamBreakRun, objective
    run = DamBreakRun(case, steps, dt, window, spos, checkpoint_every=k)
    v = case.vel[:case.n_f] if vel0 is None else vel0
    v0 = torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(alpha, dtype=torch.float64, device="cuda", requires_grad=True)
    J = objective(v0, a, run)
    J.backward()
    return float(J.detach()), v0.grad.cpu().numpy(), float(a.grad), run


def _gpu_j(torch, case, spos, vel0, alpha, steps=STEPS, window=WINDOW, dt=DT):
    from paper_1110_3711_gb300.autograd import DamBreakRun
    run = DamBreakRun(case, steps, dt, window, spos, checkpoint_every=steps)
    return float(run.forward(torch.tensor(vel0, dtype=torch.float64, device="cuda"), alpha))


def test_adjoint_matches_oracle_gradient(torch_mod):
    from oracle import grad as G
    c, spos = _case()
    Jo, gvo, gao = G.gradient(c, c.vel[:c.n_f], 0.1, STEPS, DT, WINDOW, spos)
    Jg, gvg, gag, _ = _gpu_grad(torch_mod, c, spos, k=7)
    assert Jg == pytest.approx(Jo, rel=1e-12)
    assert np.abs(gvg - gvo).max() <= 1e-8 * np.abs(gvo).max()
    assert gag == pytest.approx(gao, rel=1e-8)


def test_adjoint_general_gamma_matches_oracle(torch_mod):
    """The adjoint with a Tait exponent other than 7 (general sound speed and
    the c_bar / rho_bar form in the pair derivative, not the polynomial of
    gamma = 7) against the gradient oracle."""
    import copy
    from oracle import grad as G
    c, spos = _case()
    p = copy.copy(c.params)
    p.gamma = 5.0
    c = type(c)(**{**c.__dict__, "params": p})
    Jo, gvo, gao = G.gradient(c, c.vel[:c.n_f], 0.1, STEPS, DT, WINDOW, spos)
    Jg, gvg, gag, _ = _gpu_grad(torch_mod, c, spos, k=7)
    assert Jg == pytest.approx(Jo, rel=1e-12)
    assert np.abs(gvg - gvo).max() <= 1e-8 * np.abs(gvo).max()
    assert gag == pytest.approx(gao, rel=1e-8)


def test_checkpoint_interval_does_not_change_gradient(torch_mod):
    c, spos = _case()
    ref = _gpu_grad(torch_mod, c, spos, k=1)
    for k in (4, STEPS):
        got = _gpu_grad(torch_mod, c, spos, k=k)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1])
        assert got[2] == ref[2]


def test_adjoint_matches_gpu_finite_differences(torch_mod):
    c, spos = _case()
    _, gv, ga, _ = _gpu_grad(torch_mod, c, spos, k=10)
    v0 = c.vel[:c.n_f].copy()
    rng = np.random.default_rng(5)
    for _ in range(2):
        d = rng.normal(size=v0.shape)
        eps = 1e-7
        fd = (_gpu_j(torch_mod, c, spos, v0 + eps * d, 0.1)
              - _gpu_j(torch_mod, c, spos, v0 - eps * d, 0.1)) / (2 * eps)
        an = float((gv * d).sum())
        assert abs(fd - an) <= 5e-6 * abs(an)
    eps = 1e-6
    fd_a = (_gpu_j(torch_mod, c, spos, v0, 0.1 + eps) - _gpu_j(torch_mod, c, spos, v0, 0.1 - eps)) / (2 * eps)
    assert fd_a == pytest.approx(ga, rel=5e-6)


def _front_run(torch, case, k, vel0=None, alpha=0.1):
    from paper_1110_3711_gb300.autograd import DamBreakRun, objective
    run = DamBreakRun(case, STEPS, DT, WINDOW, None, checkpoint_every=k,
                      front_tau=case.params.dp)
    v = case.vel[:case.n_f] if vel0 is None else vel0
    v0 = torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(alpha, dtype=torch.float64, device="cuda", requires_grad=True)
    J = objective(v0, a, run)
    J.backward()
    return float(J.detach()), v0.grad.cpu().numpy(), float(a.grad)


def test_front_position_value(torch_mod):
    """sph_front_position is the smooth maximum of the fluid x of the state."""
    torch = torch_mod
    from paper_1110_3711_gb300 import sph
    c = dam_break(0.02)
    for prec in ("fp64", "fp32"):
        sim = sph.Simulation.from_case(c, precision=prec)
        for _ in range(5):
            sim.step()
        pos, _, _ = sim.get_state()
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        tau = c.params.dp
        sph.sph_front_position(sim.ctx, tau, out)
        xs = pos[:c.n_f, 0] / tau
        want = tau * (xs.max() + np.log(np.exp(xs - xs.max()).sum()))
        assert float(out.cpu()) == pytest.approx(want, rel=1e-13)


def test_front_objective_matches_oracle_gradient(torch_mod):
    """Front-position objective (tau = dp) through the adjoint: J and the
    gradients equal the gradient oracle's; the checkpoint interval changes
    nothing."""
    from oracle import grad as G
    c, _ = _case()
    Jo, gvo, gao = G.gradient(c, c.vel[:c.n_f], 0.1, STEPS, DT, WINDOW, None,
                              front_tau=c.params.dp)
    Jg, gvg, gag = _front_run(torch_mod, c, k=7)
    assert Jg == pytest.approx(Jo, rel=1e-12)
    assert np.abs(gvg - gvo).max() <= 1e-8 * np.abs(gvo).max()
    assert gag == pytest.approx(gao, rel=1e-8, abs=1e-12 * np.abs(gvo).max())
    J1, gv1, ga1 = _front_run(torch_mod, c, k=STEPS)
    assert J1 == Jg and np.array_equal(gv1, gvg) and ga1 == gag


def test_adjoint_step_needs_fixed_dt_fp64(torch_mod):
    torch = torch_mod
    from paper_1110_3711_gb300 import sph
    c = dam_break(0.02)
    lam = torch.zeros(11 * c.n, dtype=torch.float64, device="cuda")
    lam2 = torch.zeros_like(lam)
    da = torch.zeros(1, dtype=torch.float64, device="cuda")
    for prec in ("fp64", "fp32"):
        sim = sph.Simulation.from_case(c, precision=prec)   # variable dt
        with pytest.raises(sph.SphError):
            sph.sph_adjoint_step(sim.ctx, lam, lam2, da)


CONF4 = dict(steps=400, window=100, dt=1e-4)


def _fd_checks(j_of, v0, alpha, gv, ga, alpha_eps, alpha_rel):
    """Central differences of the forward map j_of(v, alpha) against the
    adjoint gradient (gv, ga) on the differentiable configuration:
      * the normalised gradient direction, eps = 1e-3, to 1e-4 relative;
      * 8 seeded random unit directions d of the initial velocities (N(0, 1)
        per component, normalised), eps = 1e-3: |FD - g.d| within 1e-4 |g|
        (|g| bounds |g.d| over unit directions; a random direction's g.d is
        about |g| / sqrt(n), so the error is stated against the gradient's
        scale rather than against the cancellation of 241,200 terms);
      * the 16 components of largest |g|, eps = 1e-5, to 1e-4 relative each
        (at eps = 1e-3 single components of the wall-pressure objective carry
        the O(eps) error of pairs crossing the viscosity switch, which is
        only C0);
      * alpha at alpha_eps to alpha_rel."""
    gn = float(np.linalg.norm(gv))
    d = gv / gn
    eps = 1e-3
    fd = (j_of(v0 + eps * d, alpha) - j_of(v0 - eps * d, alpha)) / (2 * eps)
    assert fd == pytest.approx(gn, rel=1e-4)
    for s in range(8):
        d = np.random.default_rng(1000 + s).normal(size=v0.shape)
        d /= np.linalg.norm(d)
        fd = (j_of(v0 + eps * d, alpha) - j_of(v0 - eps * d, alpha)) / (2 * eps)
        assert abs(fd - float((gv * d).sum())) <= 1e-4 * gn, s
    eps = 1e-5
    for k in np.argsort(-np.abs(gv).ravel())[:16]:
        d = np.zeros(v0.size)
        d[k] = 1.0
        d = d.reshape(v0.shape)
        fd = (j_of(v0 + eps * d, alpha) - j_of(v0 - eps * d, alpha)) / (2 * eps)
        assert fd == pytest.approx(float(gv.ravel()[k]), rel=1e-4), int(k)
    fd_a = (j_of(v0, alpha + alpha_eps) - j_of(v0, alpha - alpha_eps)) / (2 * alpha_eps)
    assert fd_a == pytest.approx(ga, rel=alpha_rel)


@pytest.mark.slow
def test_adjoint_differentiable_configuration(torch_mod):
    """dp = 0.01 dam break (80,400 fluid + 58,606 boundary), fixed dt = 1e-4 s,
    400 steps, checkpoints every 20 steps, 64 sensors on the wall behind the
    column, mean over the last 100 states; the checks of _fd_checks.  In
    alpha the sensor objective is rougher: the viscosity switch (Pi = 0 for
    v.r >= 0) is only C0 and a change of alpha moves many pairs across it,
    each adding an O(eps) error; at eps = 1e-5 the central difference agrees
    to 1e-3 (measured 3e-4, 2.5e-3 at eps = 1e-3)."""
    torch = torch_mod
    c = dam_break(0.01, vel_sigma=0.05, seed=0, fixed_dt=1e-4)
    spos = wall_sensors(c, wall="back")
    J, gv, ga, run = _gpu_grad(torch, c, spos, k=20, **CONF4)
    assert run.stats["checkpoint_bytes"] < 1e9
    _fd_checks(lambda v, al: _gpu_j(torch, c, spos, v, al, **CONF4), c.vel[:c.n_f].copy(), 0.1,
               gv, ga, alpha_eps=1e-5, alpha_rel=1e-3)


@pytest.mark.slow
def test_front_objective_differentiable_configuration(torch_mod):
    """The same configuration with the front-position objective (tau = dp, mean
    over the last 100 states): the checks of _fd_checks, alpha at eps = 1e-3
    to 1e-4 (measured 2.3e-6)."""
    torch = torch_mod
    from paper_1110_3711_gb300.autograd import DamBreakRun, objective
    c = dam_break(0.01, vel_sigma=0.05, seed=0, fixed_dt=1e-4)
    tau = c.params.dp

    def run_j(v, al):
        r = DamBreakRun(c, 400, 1e-4, 100, checkpoint_every=400, front_tau=tau)
        return float(r.forward(torch.tensor(v, dtype=torch.float64, device="cuda"), al))

    run = DamBreakRun(c, 400, 1e-4, 100, checkpoint_every=20, front_tau=tau)
    v0t = torch.tensor(c.vel[:c.n_f], dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(0.1, dtype=torch.float64, device="cuda", requires_grad=True)
    objective(v0t, a, run).backward()
    gv, ga = v0t.grad.cpu().numpy(), float(a.grad)
    _fd_checks(run_j, c.vel[:c.n_f].copy(), 0.1, gv, ga, alpha_eps=1e-3, alpha_rel=1e-4)
