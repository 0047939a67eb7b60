"""Pins of the FP64 reference MLP of the learned star-pressure proposal: backpropagation against central
finite differences, the scaling symmetry of the features, and invariance of the target."""
import numpy as np
import pytest

import oracle
from oracle import mlp


def test_parameter_count():
    assert mlp.NPARAM == 64 * 6 + 64 + 64 * 64 + 64 + 64 + 1 == 4673


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init(1) + 0.01 * rng.normal(size=mlp.NPARAM)  # non-zero biases
    x = rng.normal(size=(40, 6))
    t = rng.normal(size=40)
    g = mlp.gradient(theta, x, t)
    idx = rng.choice(mlp.NPARAM, size=200, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.NPARAM)
        e[k] = h
        fd = (mlp.loss(theta + e, x, t) - mlp.loss(theta - e, x, t)) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-9)


def test_features_are_scale_and_galilean_invariant():
    rng = np.random.default_rng(1)
    s = [rng.uniform(0.1, 2, 50) for _ in range(6)]
    x0, pref0 = mlp.features(*s)
    a, b, w = 3.7, 0.02, 1.3   # rho -> a rho, p -> b p, u -> sqrt(b/a) u + w
    k = np.sqrt(b / a)
    x1, pref1 = mlp.features(a * s[0], k * s[1] + w, b * s[2], a * s[3], k * s[4] + w, b * s[5])
    np.testing.assert_allclose(x1, x0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pref1, b * pref0, rtol=1e-14)


def test_target_is_invariant_under_the_same_transformation():
    # ln(p*/p_ref) of the two-shock solver does not change under the scaling symmetry
    P = oracle.params(8, 8)
    L, R = [0.7, 0.3, 0.0, 2.0], [0.2, -0.4, 0.0, 0.05]
    r0 = oracle.riemann(P, L, R)
    a, b = 5.0, 0.1
    k = np.sqrt(b / a)
    r1 = oracle.riemann(P, [a * L[0], k * L[1] + 0.5, 0.0, b * L[3]], [a * R[0], k * R[1] + 0.5, 0.0, b * R[3]])
    _, pref0 = mlp.features(L[0], L[1], L[3], R[0], R[1], R[3])
    _, pref1 = mlp.features(a * L[0], k * L[1] + 0.5, b * L[3], a * R[0], k * R[1] + 0.5, b * R[3])
    assert np.log(r1["pstar"] / pref1) == pytest.approx(np.log(r0["pstar"] / pref0), abs=1e-12)
