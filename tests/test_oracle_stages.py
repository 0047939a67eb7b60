"""Pins of the oracle's per-cell stages: EOS conversions (Eqs. 11-12), limited slopes (§3.1), flattening
(§3.2) and characteristic tracing (§3.2, Eq. 13)."""
import numpy as np
import pytest

import oracle

G = 1.4
P = oracle.params(8, 8, gamma=G)


# ---------------------------------------------------------------- EOS
def test_conversions_hand_values():
    # rho = 2, u = 3, v = 4, p = 5: e = p/((g-1) rho) = 6.25, E = e + 25/2 = 18.75, rho E = 37.5
    U = oracle.prim_to_cons(P, [2.0, 3.0, 4.0, 5.0])
    np.testing.assert_allclose(U, [2.0, 6.0, 8.0, 37.5], rtol=1e-15)
    np.testing.assert_allclose(oracle.cons_to_prim(P, U), [2.0, 3.0, 4.0, 5.0], rtol=1e-14)


def test_floors_apply_to_copies():
    q = oracle.cons_to_prim(P, [0.0, 0.0, 0.0, -1.0])
    assert q[0] == 1e-10 and q[3] == 1e-20


# ---------------------------------------------------------------- slopes
@pytest.mark.parametrize("limiter", [1, 2])
def test_linear_data_gives_exact_slope(limiter):
    for b in (0.7, -2.5):
        q = [3.0 + b * i for i in range(-2, 3)]
        assert oracle.slope(limiter, *q) == pytest.approx(b, rel=1e-14)


def test_fourth_order_slope_is_the_five_point_derivative():
    # for a smooth monotone cubic the unlimited fourth-order slope equals f'(0) (exact for degree <= 4)
    f = lambda i: 1.0 + 0.8 * i + 0.03 * i * i + 0.004 * i ** 3
    assert oracle.slope(2, *[f(i) for i in range(-2, 3)]) == pytest.approx(0.8, rel=1e-14)
    # while the MC slope is the centred difference (f(1) - f(-1))/2 = 0.8 + 0.004
    assert oracle.slope(1, *[f(i) for i in range(-2, 3)]) == pytest.approx(0.804, rel=1e-14)


@pytest.mark.parametrize("limiter", [1, 2])
def test_extrema_are_flattened_and_profiles_stay_monotone(limiter):
    assert oracle.slope(limiter, 0.0, 1.0, 2.0, 1.5, 0.0) == 0.0
    assert oracle.slope(limiter, 0.0, 1.0, 1.0, 2.0, 3.0) == 0.0
    rng = np.random.default_rng(3)
    for _ in range(2000):
        q = rng.normal(size=5)
        s = oracle.slope(limiter, *q)
        lo, hi = min(q[1], q[3]), max(q[1], q[3])
        # the reconstructed face values q0 +- s/2 stay within the neighbours
        if q[2] >= lo and q[2] <= hi:
            assert lo - 1e-12 <= q[2] + 0.5 * s <= hi + 1e-12
            assert lo - 1e-12 <= q[2] - 0.5 * s <= hi + 1e-12
        else:
            assert s == 0.0


def test_piecewise_constant_option():
    assert oracle.slope(0, 0.0, 1.0, 2.0, 3.0, 4.0) == 0.0


# ---------------------------------------------------------------- flattening
def test_flattening_special_values():
    # a linear pressure ramp (z = 1/2) is never flattened
    assert oracle.flatten_chi(1.0, 2.0, 4.0, 5.0, 1.0, 0.0) == 1.0
    # a compressive step (z = 1) is fully flattened
    assert oracle.flatten_chi(1.0, 1.0, 10.0, 10.0, 1.0, 0.0) == 0.0
    # the same step in an expansion is left alone
    assert oracle.flatten_chi(1.0, 1.0, 10.0, 10.0, 0.0, 1.0) == 1.0
    # a jump below 0.33 of the smaller pressure is left alone
    assert oracle.flatten_chi(1.0, 1.0, 1.3, 1.3, 1.0, 0.0) == 1.0
    # z = 0.8 sits in the middle of the ramp between 0.75 and 0.85
    assert oracle.flatten_chi(0.0, 1.0, 9.0, 10.0, 1.0, 0.0) == pytest.approx(0.5, rel=1e-12)
    assert oracle.flatten_chi(0.0, 1.0, 8.5, 10.0, 1.0, 0.0) == 1.0  # z = 0.75


# ---------------------------------------------------------------- tracing
def _jacobian(q, g=G):
    # primitive-variable Euler system q_t + A q_x = 0 in (rho, un, ut, p)
    rho, u, _, p = q
    c2 = g * p / rho
    return np.array([[u, rho, 0, 0], [0, u, 0, 1 / rho], [0, 0, u, 0], [0, rho * c2, 0, u]], dtype=float)


def _right_eigvecs(q, g=G):
    rho, u, _, p = q
    c = np.sqrt(g * p / rho)
    lam = np.array([u - c, u, u, u + c])
    R = np.array([[1, -c / rho, 0, c * c], [1, 0, 0, 0], [0, 0, 1, 0], [1, c / rho, 0, c * c]], dtype=float)
    return lam, R


@pytest.mark.parametrize("u", [0.3, -0.4, 2.0, -2.0, 0.0])
def test_traced_states_follow_the_characteristics(u):
    q = np.array([1.3, u, 0.2, 0.9])
    lam, R = _right_eigvecs(q)
    A = _jacobian(q)
    for nu in range(4):  # the test's eigenvectors really are eigenvectors of the primitive system
        np.testing.assert_allclose(A @ R[nu], lam[nu] * R[nu], rtol=1e-13, atol=1e-13)
    rng = np.random.default_rng(5)
    sigma = 0.37
    for _ in range(20):
        b = rng.normal(size=4) * 1e-3
        dq = b @ R  # slope written in wave coordinates
        ql, qr = oracle.trace(P, sigma, q, dq)
        # left state at i+1/2: waves with lam >= 0 extrapolate by (1 - sigma lam)/2, the others carry the
        # reference factor (1 - sigma lam_max)/2; mirror image for the right state at i-1/2
        el = q + sum(0.5 * (1 - sigma * (lam[n] if lam[n] >= 0 else lam[3])) * b[n] * R[n] for n in range(4))
        er_ = q - sum(0.5 * (1 + sigma * (lam[n] if lam[n] <= 0 else lam[0])) * b[n] * R[n] for n in range(4))
        np.testing.assert_allclose(ql, el, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(qr, er_, rtol=1e-13, atol=1e-15)


def test_entropy_wave_reduces_to_the_advection_hat_state():
    # a density jump carried at u > 0 traces exactly like Eq. 4: a + (1 - dt u/dx) da / 2
    q = np.array([1.0, 0.6, -0.3, 2.0])
    dq = np.array([0.05, 0.0, 0.0, 0.0])
    sigma = 0.4
    ql, _ = oracle.trace(P, sigma, q, dq)
    np.testing.assert_allclose(ql, [1.0 + 0.5 * (1 - sigma * 0.6) * 0.05, 0.6, -0.3, 2.0], rtol=1e-14)


def test_zero_time_step_gives_half_slope_extrapolation():
    q = np.array([1.0, 0.5, 0.1, 1.0])
    dq = np.array([0.1, -0.05, 0.02, 0.3])
    ql, qr = oracle.trace(P, 0.0, q, dq)
    np.testing.assert_allclose(ql, q + 0.5 * dq, rtol=1e-15)
    np.testing.assert_allclose(qr, q - 0.5 * dq, rtol=1e-15)
