"""Pins of the oracle's two-shock Riemann solver (paper §3.2, solver of almgren:2010) against the exact
solution, closed forms, an independent root bracketing and symmetries."""
import math

import numpy as np
import pytest

import exact_riemann as er
import oracle

G = 1.4
P = oracle.params(8, 8, gamma=G, riemann_tol=1e-14, riemann_maxiter=64)


def _two_shock_residual(p, L, R, g=G):
    # u*_R(p) - u*_L(p) with the Hugoniot written in Toro's (A, B) form, not the oracle's W form
    out = 0.0
    for (rho, u, pk), sgn in ((L, -1.0), (R, 1.0)):
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        out += (p - pk) * math.sqrt(A / (p + B))
    return out + (R[1] - L[1])


def _rand_state(rng):
    return (float(np.exp(rng.uniform(np.log(0.05), np.log(5.0)))), float(rng.uniform(-2, 2)), 0.0,
            float(np.exp(rng.uniform(np.log(0.01), np.log(10.0)))))


@pytest.mark.parametrize("rho,p,U", [(1.0, 1.0, 0.5), (0.3, 2.0, 3.0), (2.0, 0.01, 10.0)])
def test_symmetric_collision_closed_form(rho, p, U):
    A = 2.0 / ((G + 1.0) * rho)
    B = (G - 1.0) / (G + 1.0) * p
    k = U * U / A
    expect = p + 0.5 * (k + math.sqrt(k * k + 4.0 * k * (p + B)))
    r = oracle.riemann(P, [rho, U, 0.0, p], [rho, -U, 0.0, p])
    assert r["converged"]
    assert r["pstar"] == pytest.approx(expect, rel=1e-13)
    assert abs(r["ustar"]) <= 1e-13 * U


def test_equals_exact_solution_when_both_waves_are_shocks():
    # two-shock iteration is exact when p* exceeds both pL and pR: p*, u* and the sampled face state
    rng = np.random.default_rng(11)
    n = 0
    while n < 300:
        L = _rand_state(rng)
        R = _rand_state(rng)
        try:
            ps, us = er.star_state(L[0], L[1], L[3], R[0], R[1], R[3], G)
        except ValueError:
            continue
        if not (ps > 1.001 * max(L[3], R[3])):
            continue
        n += 1
        r = oracle.riemann(P, L, R)
        assert r["converged"]
        assert r["pstar"] == pytest.approx(ps, rel=2e-13)
        assert r["ustar"] == pytest.approx(us, rel=1e-12, abs=1e-13 * (abs(L[1]) + abs(R[1]) + 1))
        if abs(us) > 1e-6:
            rho, u, p = er.sample(0.0, L[0], L[1], L[3], R[0], R[1], R[3], G, (ps, us))
            assert r["face"][0] == pytest.approx(rho, rel=1e-11)
            assert r["face"][1] == pytest.approx(u, rel=1e-11, abs=1e-12)
            assert r["face"][3] == pytest.approx(p, rel=1e-11)


def test_root_matches_bisection_for_general_states():
    rng = np.random.default_rng(12)
    for _ in range(400):
        L = _rand_state(rng)
        R = _rand_state(rng)
        f_lo = _two_shock_residual(1e-20, (L[0], L[1], L[3]), (R[0], R[1], R[3]))
        if f_lo >= 0.0:  # the two-shock curves meet below the pressure floor; floored root
            continue
        lo, hi = 1e-20, max(L[3], R[3])
        while _two_shock_residual(hi, (L[0], L[1], L[3]), (R[0], R[1], R[3])) < 0:
            hi *= 2
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if _two_shock_residual(mid, (L[0], L[1], L[3]), (R[0], R[1], R[3])) < 0:
                lo = mid
            else:
                hi = mid
        r = oracle.riemann(P, L, R)
        assert r["converged"]
        assert r["pstar"] == pytest.approx(0.5 * (lo + hi), rel=1e-12)


def test_mirror_symmetry_is_exact():
    rng = np.random.default_rng(13)
    for _ in range(200):
        L = list(_rand_state(rng))
        R = list(_rand_state(rng))
        L[2], R[2] = rng.uniform(-1, 1), rng.uniform(-1, 1)
        a = oracle.riemann(P, L, R)
        mL = [R[0], -R[1], R[2], R[3]]
        mR = [L[0], -L[1], L[2], L[3]]
        b = oracle.riemann(P, mL, mR)
        assert b["pstar"] == a["pstar"]
        assert b["ustar"] == -a["ustar"]
        np.testing.assert_array_equal(b["flux"], [-a["flux"][0], a["flux"][1], -a["flux"][2], -a["flux"][3]])


def test_trivial_problem_returns_the_state_and_its_flux():
    rng = np.random.default_rng(14)
    for _ in range(50):
        q = [float(np.exp(rng.uniform(-2, 2))), rng.uniform(-3, 3), rng.uniform(-3, 3), float(np.exp(rng.uniform(-3, 3)))]
        r = oracle.riemann(P, q, q)
        assert r["converged"]
        assert r["pstar"] == pytest.approx(q[3], rel=1e-15)
        assert r["ustar"] == pytest.approx(q[1], rel=1e-15, abs=1e-15)
        rho, un, ut, p = q
        E = p / (G - 1) + 0.5 * rho * (un * un + ut * ut)
        expect = [rho * un, rho * un * un + p, rho * un * ut, un * (E + p)]
        np.testing.assert_allclose(r["flux"], expect, rtol=1e-14, atol=1e-14)


def test_flux_satisfies_rankine_hugoniot_across_an_exact_shock():
    # oracle flux + conversions are consistent with the conservation law: F(q2) - F(q1) = S (U2 - U1)
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us = er.star_state(L[0], L[1], L[2], R[0], R[1], R[2], G)
    cr = math.sqrt(G * R[2] / R[0])
    S = R[1] + cr * math.sqrt((G + 1) / (2 * G) * ps / R[2] + (G - 1) / (2 * G))
    r2, u2, p2 = er.sample(S - 1e-9, L[0], L[1], L[2], R[0], R[1], R[2], G)
    q1, q2 = [R[0], R[1], 0.3, R[2]], [r2, u2, 0.3, p2]
    F1, F2 = oracle.euler_flux(P, q1), oracle.euler_flux(P, q2)
    U1, U2 = oracle.prim_to_cons(P, q1), oracle.prim_to_cons(P, q2)
    # face frame (mass, normal, transverse, energy) vs conserved (rho, rho u, rho v, rho E)
    np.testing.assert_allclose(F2 - F1, S * (U2 - U1), rtol=1e-11)


def test_supersonic_flow_takes_the_upwind_state():
    q = [1.0, 5.0, 0.2, 1.0]   # |u| > c on both sides: the face sees the left state
    q2 = [0.9, 5.1, -0.1, 1.1]
    r = oracle.riemann(P, q, q2)
    np.testing.assert_array_equal(r["face"], q)


def test_strong_expansions_converge_and_match_bisection():
    # p* << rho u^2: rounding bounds |dp| near the root by ~eps rho u c, so the velocity-scale stopping
    # rule is what ends these iterations; the root still agrees with an independent bisection
    rng = np.random.default_rng(22)
    for _ in range(500):
        rho, c_over_u = float(np.exp(rng.uniform(-1, 1))), 10 ** rng.uniform(-2.5, -0.5)
        u = rng.uniform(0.5, 3.0)
        p = rho * (c_over_u * u) ** 2 / G
        L, R = [rho, -0.3 * u, 0.0, p], [rho * 1.3, 0.2 * u, 0.0, 0.7 * p]
        r = oracle.riemann(P, L, R)
        assert r["converged"] and r["iters"] <= 12
        f = lambda x: _two_shock_residual(x, (L[0], L[1], L[3]), (R[0], R[1], R[3]))
        if f(1e-20) >= 0:
            assert r["pstar"] == 1e-20
            continue
        lo, hi = 1e-20, max(L[3], R[3])
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
        assert r["pstar"] == pytest.approx(0.5 * (lo + hi), rel=1e-9)


def test_nonconvergence_is_reported():
    p1 = oracle.params(8, 8, riemann_maxiter=1, riemann_tol=1e-14)
    r = oracle.riemann(p1, [1.0, 0.0, 0.0, 1.0], [0.125, 0.0, 0.0, 0.1])
    assert not r["converged"] and r["iters"] == 1


def test_weak_waves_converge_from_the_acoustic_guess_at_once():
    # the linearised (acoustic) start is exact to second order in the wave strength, so a Newton
    # iteration on a weak problem meets the 1e-14 tolerance within two iterations
    rng = np.random.default_rng(15)
    for _ in range(50):
        rho, u, p = float(np.exp(rng.uniform(-1, 1))), rng.uniform(-1, 1), float(np.exp(rng.uniform(-1, 1)))
        eps = 1e-4 * rng.uniform(-1, 1, size=3)
        L = [rho, u, 0.0, p]
        R = [rho * (1 + eps[0]), u + eps[1] * np.sqrt(p / rho), 0.0, p * (1 + eps[2])]
        r = oracle.riemann(P, L, R)
        assert r["converged"] and r["iters"] <= 2, r["iters"]


def test_transonic_rarefaction_face_state_is_continuous():
    # shift a double-rarefaction problem through the face: the sampled pressure and normal velocity vary
    # continuously (fan head -> unperturbed state, fan tail -> star state); the density jumps only where
    # the contact crosses the face (u* changes sign)
    L0, R0 = [1.0, -0.5, 0.1, 1.0], [0.5, 0.6, -0.2, 0.4]
    shifts = np.linspace(-2.0, 2.0, 4001)
    faces, ust = [], []
    for d in shifts:
        L = [L0[0], L0[1] + d, L0[2], L0[3]]
        R = [R0[0], R0[1] + d, R0[2], R0[3]]
        r = oracle.riemann(P, L, R)
        faces.append(r["face"])
        ust.append(r["ustar"])
    faces, ust = np.array(faces), np.array(ust)
    step = shifts[1] - shifts[0]
    dpu = np.abs(np.diff(faces[:, [1, 3]], axis=0)).max(axis=0)
    assert np.all(dpu < 5 * step), dpu
    contact = np.diff(np.sign(ust)) != 0
    assert contact.sum() == 1
    drho = np.abs(np.diff(faces[:, 0]))[~contact]
    assert drho.max() < 5 * step, drho.max()
    # the face crosses both fans: some samples lie strictly inside a fan
    inside = (np.abs(faces[:, 3] - L0[3]) > 1e-9) & (np.abs(faces[:, 3] - R0[3]) > 1e-9)
    assert inside.sum() > 10
