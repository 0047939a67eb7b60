"""Pins of the test-side exact Riemann solver (Toro 1997) against closed forms."""
import math

import numpy as np
import pytest

import exact_riemann as er

G = 1.4


@pytest.mark.parametrize("rho,p,U", [(1.0, 1.0, 0.5), (0.3, 2.0, 3.0), (2.0, 0.01, 10.0)])
def test_symmetric_collision_closed_form(rho, p, U):
    # (rho, p, +U) | (rho, p, -U): two equal shocks, (p*-p) sqrt(A/(p*+B)) = U -> quadratic in p*-p
    A = 2.0 / ((G + 1.0) * rho)
    B = (G - 1.0) / (G + 1.0) * p
    k = U * U / A
    x = 0.5 * (k + math.sqrt(k * k + 4.0 * k * (p + B)))
    ps, us = er.star_state(rho, U, p, rho, -U, p, G)
    assert ps == pytest.approx(p + x, rel=1e-13)
    assert abs(us) < 1e-13 * U


@pytest.mark.parametrize("rho,p,U", [(1.0, 1.0, 0.5), (0.3, 2.0, 1.0), (2.0, 0.5, 0.2)])
def test_symmetric_expansion_closed_form(rho, p, U):
    # (rho, p, -U) | (rho, p, +U): two equal rarefactions, p* = p (1 - (g-1) U / (2c))^(2g/(g-1))
    c = math.sqrt(G * p / rho)
    expect = p * (1.0 - (G - 1.0) * U / (2.0 * c)) ** (2.0 * G / (G - 1.0))
    ps, us = er.star_state(rho, -U, p, rho, U, p, G)
    assert ps == pytest.approx(expect, rel=1e-12)
    assert abs(us) < 1e-13


def test_rankine_hugoniot_across_exact_shock():
    # mass and momentum fluxes balance across the exact right shock: F(q*) - F(qR) = S (U* - UR)
    rl, ul, pl, rr, ur, pr = 1.0, 0.0, 1.0, 0.125, 0.0, 0.1
    ps, us = er.star_state(rl, ul, pl, rr, ur, pr, G)
    eps = 1e-9
    cr = math.sqrt(G * pr / rr)
    S = ur + cr * math.sqrt((G + 1) / (2 * G) * ps / pr + (G - 1) / (2 * G))
    r2, u2, p2 = er.sample(S - eps, rl, ul, pl, rr, ur, pr, G)
    r1, u1, p1 = er.sample(S + eps, rl, ul, pl, rr, ur, pr, G)
    assert (r1, u1, p1) == (rr, ur, pr)
    assert r2 * u2 - r1 * u1 == pytest.approx(S * (r2 - r1), rel=1e-12)
    assert (r2 * u2 * u2 + p2) - (r1 * u1 * u1 + p1) == pytest.approx(S * (r2 * u2 - r1 * u1), rel=1e-12)
    E2 = p2 / (G - 1) + 0.5 * r2 * u2 * u2
    E1 = p1 / (G - 1) + 0.5 * r1 * u1 * u1
    assert u2 * (E2 + p2) - u1 * (E1 + p1) == pytest.approx(S * (E2 - E1), rel=1e-12)


def test_rarefaction_is_isentropic_and_continuous():
    rl, ul, pl, rr, ur, pr = 1.0, 0.0, 1.0, 0.125, 0.0, 0.1
    ps, us = er.star_state(rl, ul, pl, rr, ur, pr, G)
    cl = math.sqrt(G * pl / rl)
    cs = cl * (ps / pl) ** ((G - 1) / (2 * G))
    for xi in np.linspace(-cl, us - cs, 7):
        r, u, p = er.sample(xi, rl, ul, pl, rr, ur, pr, G)
        assert p / r ** G == pytest.approx(pl / rl ** G, rel=1e-12)
        # inside the fan the left-facing characteristic through the origin: u - c = xi
        assert u - math.sqrt(G * p / r) == pytest.approx(xi, abs=1e-12)
