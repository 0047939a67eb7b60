"""Pins of the oracle's HLLC solver, the alternative Riemann solver the paper names (§3.2, after Toro 1997),
against what the conservation laws and the solver's construction fix:

* consistency: equal states give the Euler flux of the state;
* an isolated contact (equal pressure and normal velocity) is resolved exactly: the flux is the upwind
  side's Euler flux, (0, p, 0, 0) when the contact is at rest;
* an isolated shock built from the Rankine-Hugoniot relations, with its exact speed given as the outer wave
  speed, is resolved exactly: the contact speed is the post-shock velocity and the flux is the post-shock
  Euler flux (F_R - F_L = S (U_R - U_L)), for left- and right-facing shocks with the face between the
  shock and the contact, where the star state's formula alone decides the flux;
* supersonic states give the upwind Euler flux; a symmetric collision carries no mass and no energy;
* mirror symmetry (x -> -x); the wave-speed estimates bound both sides' sound waves and reduce to u -/+ c for
  weak waves;
* whole steps with HLLC: uniform flow is a fixed point, periodic runs conserve, the transposed problem gives
  the transposed answer bit for bit, Sod matches the exact solution, the smooth pulse converges at second
  order.
"""
import numpy as np
import pytest

import exact_riemann as er
import hydro_problems as hp
import oracle

G = 1.4
NG = 4
P = oracle.params(8, 8, riemann_solver="hllc")


def _euler_flux(q):
    return oracle.euler_flux(P, q)


def _close(a, b, tol=1e-13):
    a, b = np.asarray(a, float), np.asarray(b, float)
    scale = max(np.abs(b).max(), 1.0)
    assert np.all(np.abs(a - b) <= tol * scale), (a, b)


@pytest.mark.parametrize("q", [(1.0, 0.3, -0.2, 1.0), (0.2, -2.0, 0.5, 0.03), (3.0, 5.0, 1.0, 0.5),
                               (1.0, 0.0, 0.0, 1e-6)])
def test_equal_states_give_the_euler_flux(q):
    F, (SL, Ss, SR) = oracle.hllc(P, q, q)
    _close(F, _euler_flux(q))
    assert SL < Ss < SR
    assert Ss == pytest.approx(q[1], rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("u", [0.7, -0.4, 0.0])
def test_an_isolated_contact_is_resolved_exactly(u):
    qL = (1.0, u, 0.3, 2.0)
    qR = (0.25, u, -0.6, 2.0)
    F, (SL, Ss, SR) = oracle.hllc(P, qL, qR)
    assert Ss == pytest.approx(u, abs=1e-15)
    if u > 0:
        _close(F, _euler_flux(qL))
    elif u < 0:
        _close(F, _euler_flux(qR))
    else:
        np.testing.assert_array_equal(F, [0.0, 2.0, 0.0, 0.0])


def _shock(M, rho0=1.0, p0=1.0, v0=0.4):
    """Left-facing shock of Mach number M running into gas at rest on its left: (pre, post, speed)."""
    c0 = np.sqrt(G * p0 / rho0)
    rho1 = rho0 * (G + 1) * M * M / ((G - 1) * M * M + 2)
    p1 = p0 * (2 * G * M * M - (G - 1)) / (G + 1)
    S = -M * c0
    u1 = S + M * c0 * rho0 / rho1
    return (rho0, 0.0, v0, p0), (rho1, u1, v0, p1), S


def _shift(q, w):
    return (q[0], q[1] + w, q[2], q[3])


@pytest.mark.parametrize("M", [1.1, 2.0, 5.0])
def test_an_isolated_shock_with_its_exact_speed_is_resolved_exactly(M):
    pre, post, S = _shock(M)
    # the post-shock velocity is -M c0 (1 - rho0/rho1) < 0; shift the frame so that the face lies between the
    # shock (moving left) and the contact (moving right): the flux is then F_L + S_L (U*_L - U_L)
    c0 = np.sqrt(G)
    w = M * c0 * (1.0 - 0.5 * pre[0] / post[0])
    qL, qR, SL = _shift(pre, w), _shift(post, w), S + w
    assert SL < 0.0 < post[1] + w
    F, Ss = oracle.hllc_core(P, qL, qR, SL, qR[1] + 10.0)
    assert Ss == pytest.approx(post[1] + w, rel=1e-13)
    # Rankine-Hugoniot: the flux through the face is the post-shock state's Euler flux
    _close(F, _euler_flux(qR))
    # mirror image: a right-facing shock, the face between the contact and the shock
    mL, mR = (qR[0], -qR[1], qR[2], qR[3]), (qL[0], -qL[1], qL[2], qL[3])
    Fm, Ssm = oracle.hllc_core(P, mL, mR, mL[1] - 10.0, -SL)
    assert Ssm == pytest.approx(-(post[1] + w), rel=1e-13)
    _close(Fm, _euler_flux(mL))


def test_supersonic_states_give_the_upwind_flux():
    qL, qR = (1.0, 4.0, 0.2, 1.0), (0.5, 3.5, -0.1, 0.8)
    F, (SL, _, _) = oracle.hllc(P, qL, qR)
    assert SL > 0
    np.testing.assert_array_equal(F, _euler_flux(qL))
    F, (_, _, SR) = oracle.hllc(P, (qR[0], -qR[1], qR[2], qR[3]), (qL[0], -qL[1], qL[2], qL[3]))
    assert SR < 0
    np.testing.assert_array_equal(F, _euler_flux((qL[0], -qL[1], qL[2], qL[3])))


@pytest.mark.parametrize("U", [0.5, 3.0])
def test_a_symmetric_collision_carries_no_mass_or_energy(U):
    q = (1.3, U, 0.0, 0.7)
    F, (SL, Ss, SR) = oracle.hllc(P, q, (1.3, -U, 0.0, 0.7))
    assert Ss == 0.0 and SL == -SR
    assert SL < 0.0  # also for a collision far faster than sound, whose shocks still move outwards
    assert abs(F[0]) <= 1e-14 and abs(F[3]) <= 1e-14 * (1 + U ** 3)
    assert F[1] > 0.7  # the collision raises the pressure at the face


@pytest.mark.parametrize("seed", range(6))
def test_mirror_symmetry(seed):
    rng = np.random.default_rng(seed)
    qL = (rng.uniform(0.1, 2), rng.uniform(-2, 2), rng.uniform(-1, 1), rng.uniform(0.05, 3))
    qR = (rng.uniform(0.1, 2), rng.uniform(-2, 2), rng.uniform(-1, 1), rng.uniform(0.05, 3))
    F, _ = oracle.hllc(P, qL, qR)
    Fm, _ = oracle.hllc(P, (qR[0], -qR[1], qR[2], qR[3]), (qL[0], -qL[1], qL[2], qL[3]))
    _close(Fm, (-F[0], F[1], -F[2], -F[3]), 1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_outer_speeds_bound_both_sides_sound_waves(seed):
    rng = np.random.default_rng(100 + seed)
    qL = (rng.uniform(0.1, 2), rng.uniform(-2, 2), 0.0, rng.uniform(0.05, 3))
    qR = (rng.uniform(0.1, 2), rng.uniform(-2, 2), 0.0, rng.uniform(0.05, 3))
    _, (SL, Ss, SR) = oracle.hllc(P, qL, qR)
    for q in (qL, qR):
        c = np.sqrt(G * q[3] / q[0])
        assert SL <= q[1] - c and SR >= q[1] + c
    assert SL <= Ss <= SR


def test_weak_waves_travel_at_the_sound_speed():
    q = np.array([1.0, 0.2, 0.0, 1.0])
    c = np.sqrt(G)
    for eps in (1e-3, 1e-5):
        _, (SL, _, SR) = oracle.hllc(P, q * (1 + eps), q)
        assert abs(SL - (0.2 - c)) < 10 * eps and abs(SR - (0.2 + c)) < 10 * eps


# ---------------------------------------------------------------- whole steps with HLLC
def _params(pr, **kw):
    xmin, xmax, ymin, ymax = pr.domain
    return oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl, xmin=xmin, xmax=xmax, ymin=ymin,
                         ymax=ymax, riemann_solver="hllc", **kw)


def _interior(U):
    return U[:, NG:-NG, NG:-NG]


@pytest.mark.parametrize("split", [False, True])
def test_uniform_flow_is_a_fixed_point(split):
    rho, pres, vel = 0.8, 1.9, (0.37, -1.3)
    U = np.zeros((4, 18, 20))
    U[0], U[1], U[2] = rho, rho * vel[0], rho * vel[1]
    U[3] = pres / (G - 1) + 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2)
    p = oracle.params(12, 10, bc=("periodic",) * 4, riemann_solver="hllc")
    U0 = U.copy()
    oracle.advance(p, U, nsteps=3, split=split)
    np.testing.assert_allclose(_interior(U), _interior(U0), rtol=1e-14, atol=1e-14)


def test_periodic_run_conserves_and_transposes():
    pr = hp.kh(40, 32, seed=3)
    p = _params(pr)
    U, UT = pr.U.copy(), hp.transpose(pr.U)
    t0 = oracle.conserved_totals(p, U)
    oracle.advance(p, U, nsteps=20)
    t1 = oracle.conserved_totals(p, U)
    scale = np.abs(_interior(pr.U)).sum(axis=(1, 2)) / (40 * 32)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale)
    pT = oracle.params(32, 40, bc=("periodic",) * 4, riemann_solver="hllc")
    oracle.advance(pT, UT, nsteps=20)
    np.testing.assert_array_equal(_interior(hp.transpose(U)), _interior(UT))


@pytest.mark.parametrize("split", [False, True])
def test_sod_matches_the_exact_solution(split):
    pr = hp.sod(128, 4)
    U = pr.U.copy()
    t, _ = oracle.advance(_params(pr), U, tmax=0.2, split=split)
    rho = U[0, NG, NG:-NG]
    exact = np.array(er.cell_averaged_density(np.linspace(0.0, 1.0, 129), 0.2, 0.5, (1.0, 0.0, 1.0),
                                              (0.125, 0.0, 0.1)))
    assert np.abs(rho - exact).mean() < 4e-3


def test_smooth_pulse_converges_at_second_order():
    errs = []
    for n in (32, 64, 128):
        pr = hp.pulse(n, n)
        U = pr.U.copy()
        t, _ = oracle.advance(_params(pr), U, tmax=0.25)
        xc = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(xc, xc)
        exact = 1.0 + sum(np.exp(-60.0 * ((X - 0.5 - t + a) ** 2 + (Y - 0.5 - t + b) ** 2))
                          for a in (-1, 0, 1) for b in (-1, 0, 1))
        errs.append(np.abs(U[0, NG:-NG, NG:-NG] - exact).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] >= 1.8, (errs, orders)
