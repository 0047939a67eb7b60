"""Pins of the oracle's dimensionally split variant (§3.1: directional updates built without the transverse
flow, each acting on the state the previous one left, with the order of the directions alternated from step
to step), pinned against what the mathematics fixes:

* a uniform flow is a fixed point, bit for bit, in either order;
* on a problem that varies along x only, the y sweep is an exact identity, so x-first and y-first steps agree
  bit for bit, and both equal the unsplit step (whose transverse terms then vanish) to rounding;
* transposing the state and swapping the order of the sweeps transposes the answer, bit for bit, on a grid
  with dx != dy and mixed boundaries;
* periodic runs conserve mass, momentum and energy to rounding;
* Sod's problem matches the exact solution; the smooth density pulse converges at second order;
* gravity (half-step on every traced v, sources in the y sweep): exact free fall, a second-order difference
  from the unsplit step on a problem along x, mirror symmetry and near-balance of the Rayleigh-Taylor column,
  walls equal to the mirrored periodic box.
"""
import numpy as np
import pytest

import exact_riemann as er
import hydro_problems as hp
import oracle

NG = 4


def _params(pr, **kw):
    xmin, xmax, ymin, ymax = pr.domain
    return oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl, xmin=xmin, xmax=xmax, ymin=ymin,
                         ymax=ymax, **kw)


def _interior(U):
    return U[:, NG:-NG, NG:-NG]


@pytest.mark.parametrize("bc", ["outflow", "periodic"])
@pytest.mark.parametrize("vel", [(0.0, 0.0), (0.37, -1.3)])
def test_uniform_flow_is_a_fixed_point(bc, vel):
    g, rho, pres, nx, ny = 1.4, 0.8, 1.9, 12, 10
    U = np.zeros((4, ny + 2 * NG, nx + 2 * NG))
    U[0], U[1], U[2] = rho, rho * vel[0], rho * vel[1]
    U[3] = pres / (g - 1) + 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2)
    p = oracle.params(nx, ny, bc=(bc,) * 4)
    U0 = U.copy()
    for n in range(4):
        oracle.fill_ghost(p, U)
        oracle.step_split(p, U, oracle.cfl_dt(p, U), n % 2)
    np.testing.assert_array_equal(_interior(U), _interior(U0))


@pytest.mark.parametrize("maker", [lambda: hp.sod(128, 6), lambda: hp.pulse(64, 64, v0=0.0)])
def test_a_problem_along_x_sees_no_y_sweep_and_equals_the_unsplit_step(maker):
    pr = maker()
    if pr.name == "pulse":  # make it one-dimensional: density pulse along x only, constant in y
        U0 = pr.U.copy()
        U0[:, :, :] = U0[:, NG + pr.ny // 2:NG + pr.ny // 2 + 1, :]
        pr.U[:] = U0
    p = _params(pr)
    oracle.advance(p, pr.U, nsteps=8)  # start from a flow with compression, where the viscosity acts
    a, b, c = pr.U.copy(), pr.U.copy(), pr.U.copy()
    for U in (a, b, c):
        oracle.fill_ghost(p, U)
    dt = oracle.cfl_dt(p, a)
    oracle.step_split(p, a, dt, 0)
    oracle.step_split(p, b, dt, 1)
    oracle.step(p, c, dt)
    np.testing.assert_array_equal(_interior(a), _interior(b))
    # the unsplit step converts its face states to conserved variables and back for the (zero) transverse
    # correction: equal to rounding
    scale = np.abs(_interior(c)).reshape(4, -1).max(axis=1)
    err = np.abs(_interior(a) - _interior(c)).reshape(4, -1).max(axis=1) / np.maximum(scale, 1e-300)
    assert np.all(err <= 1e-13), err
    # the one-dimensional step moved something
    assert np.abs(_interior(a) - _interior(pr.U)).max() > 1e-3


@pytest.mark.parametrize("maker", [lambda: hp.quad(23, 17, seed=7), lambda: hp.kh(20, 28, seed=2),
                                   lambda: hp.sod(40, 9)])
def test_transposed_problem_with_swapped_sweeps_gives_the_transposed_answer_bitwise(maker):
    pr = maker()
    p = _params(pr)
    xmin, xmax, ymin, ymax = pr.domain
    pT = oracle.params(pr.ny, pr.nx, bc=(pr.bc[2], pr.bc[3], pr.bc[0], pr.bc[1]), gamma=pr.gamma, cfl=pr.cfl,
                       xmin=ymin, xmax=ymax, ymin=xmin, ymax=xmax)
    U, UT = pr.U.copy(), hp.transpose(pr.U)
    for n in range(4):
        oracle.fill_ghost(p, U)
        oracle.fill_ghost(pT, UT)
        dt = oracle.cfl_dt(p, U)
        assert oracle.cfl_dt(pT, UT) == dt
        oracle.step_split(p, U, dt, n % 2)
        oracle.step_split(pT, UT, dt, 1 - n % 2)
    np.testing.assert_array_equal(_interior(hp.transpose(U)), _interior(UT))


def test_periodic_run_conserves_mass_momentum_energy():
    pr = hp.kh(48, 40, seed=3)
    p = _params(pr)
    U = pr.U.copy()
    t0 = oracle.conserved_totals(p, U)
    scale = np.abs(_interior(U)).sum(axis=(1, 2)) / (48 * 40)
    oracle.advance(p, U, nsteps=30, split=True)
    t1 = oracle.conserved_totals(p, U)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale


def test_sod_matches_the_exact_solution():
    pr = hp.sod(128, 4)
    p = _params(pr)
    U = pr.U.copy()
    t, _ = oracle.advance(p, U, tmax=0.2, split=True)
    assert t == pytest.approx(0.2, rel=1e-14)
    rho = U[0, NG, NG:-NG]
    n = rho.size
    exact = np.array(er.cell_averaged_density(np.linspace(0.0, 1.0, n + 1), 0.2, 0.5, (1.0, 0.0, 1.0),
                                              (0.125, 0.0, 0.1)))
    assert np.abs(rho - exact).sum() / n < 4e-3


def test_smooth_pulse_converges_at_second_order():
    errs = []
    for n in (32, 64, 128):
        pr = hp.pulse(n, n)
        U = pr.U.copy()
        t, _ = oracle.advance(_params(pr), U, tmax=0.25, split=True)
        xc = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(xc, xc)
        exact = 1.0 + sum(np.exp(-60.0 * ((X - 0.5 - t + a) ** 2 + (Y - 0.5 - t + b) ** 2))
                          for a in (-1, 0, 1) for b in (-1, 0, 1))
        errs.append(np.abs(U[0, NG:-NG, NG:-NG] - exact).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] >= 1.8, (errs, orders)


def _box(nx, ny, bc, grav, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.5 * rng.random((ny, nx))
    u = rng.uniform(-0.5, 0.5, (ny, nx))
    v = rng.uniform(-0.5, 0.5, (ny, nx))
    p = 1.0 + rng.random((ny, nx))
    return hp.Problem("box", nx, ny, hp._pack(rho, u, v, p, 1.4), bc, grav=grav)


def test_gravity_free_fall_of_a_uniform_state():
    # gravity acts in the y sweep with the unsplit step's time-centred sources: a uniform state falls as
    # v = g t exactly, density and pressure unchanged
    n, g = 12, -2.0
    one = np.ones((n, n))
    pr = hp.Problem("fall", n, n, hp._pack(one, 0 * one, 0 * one, one, 1.4), ("periodic",) * 4, grav=g)
    U = pr.U.copy()
    t, _ = oracle.advance(_params(pr, grav=g), U, nsteps=9, split=True)
    I = _interior(U)
    np.testing.assert_array_equal(I[0], 1.0)
    np.testing.assert_allclose(I[2] / I[0], g * t, rtol=1e-13)
    pres = 0.4 * (I[3] - 0.5 * (I[1] ** 2 + I[2] ** 2) / I[0])
    np.testing.assert_allclose(pres, 1.0, rtol=1e-13)


def test_gravity_on_a_problem_along_x_differs_from_the_unsplit_step_at_second_order():
    # a state uniform in y with periodic y: without gravity the split step equals the unsplit one to
    # rounding; with gravity the sources of the y sweep see the state the x sweep left, so the two differ by
    # O(dt^2 g): halving dt divides the difference by about 4
    pr = hp.sod(64, 6)
    pr.bc = ("outflow", "outflow", "periodic", "periodic")
    p = _params(pr, grav=-0.8)
    oracle.advance(p, pr.U, nsteps=6)
    oracle.fill_ghost(p, pr.U)
    dt = oracle.cfl_dt(p, pr.U)
    diffs = []
    for h in (dt, 0.5 * dt):
        a, c = pr.U.copy(), pr.U.copy()
        oracle.step_split(p, a, h, 0)
        oracle.step(p, c, h)
        diffs.append(np.abs(_interior(a) - _interior(c)).max())
    assert diffs[0] > 1e-12 and diffs[0] / diffs[1] > 3.0, diffs
    p0 = _params(pr)
    a, c = pr.U.copy(), pr.U.copy()
    oracle.step_split(p0, a, dt, 0)
    oracle.step(p0, c, dt)
    assert np.abs(_interior(a) - _interior(c)).max() <= 1e-13 * np.abs(_interior(c)).max()


def test_rayleigh_taylor_split_stays_mirror_symmetric_and_near_balance():
    pr = hp.rt(16, 48)
    U = pr.U.copy()
    oracle.advance(_params(pr, grav=pr.grav), U, nsteps=20, split=True)
    I = _interior(U)
    M = I[:, :, ::-1].copy()
    M[1] *= -1.0
    np.testing.assert_allclose(I, M, rtol=1e-12, atol=1e-13)
    flat = hp.rt(16, 48, amp=0.0)
    V = flat.U.copy()
    t, _ = oracle.advance(_params(flat, grav=flat.grav), V, nsteps=40, split=True)
    vmax = np.abs(_interior(V)[2] / _interior(V)[0]).max()
    assert vmax < 0.005 * abs(flat.grav) * t, (vmax, t)
    assert np.abs(_interior(V)[0] - _interior(flat.U)[0]).max() < 0.01


def test_reflecting_x_walls_with_gravity_equal_the_mirrored_periodic_box():
    # walls normal to x, gravity along y: the mirrored periodic box of twice the width evolves the same
    nx, ny = 10, 12
    walls = _box(nx, ny, ("reflect", "reflect", "periodic", "periodic"), -1.0, 5)
    I = _interior(walls.U)
    Mi = I[:, :, ::-1].copy()
    Mi[1] *= -1.0
    D = np.zeros((4, ny + 2 * NG, 2 * nx + 2 * NG))
    D[:, NG:-NG, NG:NG + nx] = I
    D[:, NG:-NG, NG + nx:-NG] = Mi
    box = hp.Problem("box", 2 * nx, ny, D, ("periodic",) * 4, domain=(0.0, 2.0, 0.0, 1.0), grav=-1.0)
    Uw, Ub = walls.U.copy(), box.U.copy()
    oracle.advance(_params(walls, grav=-1.0), Uw, nsteps=6, split=True)
    oracle.advance(_params(box, grav=-1.0), Ub, nsteps=6, split=True)
    np.testing.assert_allclose(_interior(Uw), _interior(Ub)[:, :, :nx], rtol=1e-12, atol=1e-12)
