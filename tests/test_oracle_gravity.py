"""Pins of the oracle's gravity source and reflecting / hydrostatic boundaries (paper §3.2: the rho g and
rho U.g sources of the Euler equations, and the hydrostatic boundary of the Rayleigh-Taylor problem).

* free fall: a uniform state in a periodic box accelerates as v = g t with density and pressure unchanged
  (closed form of the time-centred sources);
* reflecting walls: a box with reflecting x walls evolves exactly as one half of the periodic box of twice
  the width holding the mirror image (u -> -u) in the other half, with and without gravity; likewise for
  y walls without gravity;
* hydrostatic ghost cells: density and momenta copied from the row next to the wall, pressure
  p_edge + rho g (y - y_edge);
* Rayleigh-Taylor: the set-up without its perturbation is close to hydrostatic balance (velocities stay a
  small fraction of free fall), and the perturbed run stays mirror-symmetric about x = 1/2;
* the buoyant bubble (Table 1's `bubble`): its density deficit rises and the run stays mirror-symmetric.
"""
import numpy as np
import pytest

import hydro_problems as hp
import oracle

NG = 4


def _interior(U):
    return U[:, NG:-NG, NG:-NG]


def _params(pr, **kw):
    xmin, xmax, ymin, ymax = pr.domain
    return oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl, xmin=xmin, xmax=xmax, ymin=ymin,
                         ymax=ymax, grav=pr.grav, **kw)


def _state(rho, u, v, p, gamma=1.4):
    return hp._pack(rho, u, v, p, gamma)


def test_free_fall_of_a_uniform_state():
    n, g = 16, -2.0
    one = np.ones((n, n))
    pr = hp.Problem("fall", n, n, _state(one, 0 * one, 0 * one, one), ("periodic",) * 4, grav=g)
    P = _params(pr)
    U = pr.U.copy()
    t, steps = oracle.advance(P, U, nsteps=12)
    I = _interior(U)
    np.testing.assert_array_equal(I[0], 1.0)
    np.testing.assert_allclose(I[2] / I[0], g * t, rtol=1e-13)
    assert np.all(I[1] == 0.0)
    pres = (pr.gamma - 1.0) * (I[3] - 0.5 * (I[1] ** 2 + I[2] ** 2) / I[0])
    np.testing.assert_allclose(pres, 1.0, rtol=1e-13)


def _mirror_x(U):
    """State of the doubled periodic box: the original on [0, 1], its mirror image (u -> -u) on [1, 2]."""
    I = _interior(U)
    M = I[:, :, ::-1].copy()
    M[1] *= -1.0
    D = np.zeros((4, I.shape[1] + 2 * NG, 2 * I.shape[2] + 2 * NG))
    D[:, NG:-NG, NG:NG + I.shape[2]] = I
    D[:, NG:-NG, NG + I.shape[2]:-NG] = M
    return D


@pytest.mark.parametrize("grav", [0.0, -1.0])
def test_reflecting_x_walls_equal_the_mirrored_periodic_box(grav):
    rng = np.random.default_rng(11)
    nx, ny = 12, 10
    rho = 1.0 + 0.5 * rng.random((ny, nx))
    u = rng.uniform(-0.5, 0.5, (ny, nx))
    v = rng.uniform(-0.5, 0.5, (ny, nx))
    p = 1.0 + rng.random((ny, nx))
    U0 = _state(rho, u, v, p)
    walls = hp.Problem("walls", nx, ny, U0, ("reflect", "reflect", "periodic", "periodic"), grav=grav)
    box = hp.Problem("box", 2 * nx, ny, _mirror_x(U0), ("periodic",) * 4, domain=(0.0, 2.0, 0.0, 1.0), grav=grav)
    Uw, Ub = walls.U.copy(), box.U.copy()
    tw, nw = oracle.advance(_params(walls), Uw, nsteps=6)
    tb, nb = oracle.advance(_params(box), Ub, nsteps=6)
    assert nw == nb and tw == pytest.approx(tb, rel=1e-14)
    left = _interior(Ub)[:, :, :nx]
    np.testing.assert_allclose(_interior(Uw), left, rtol=1e-12, atol=1e-12)


def test_reflecting_y_walls_equal_the_mirrored_periodic_box():
    rng = np.random.default_rng(12)
    nx, ny = 10, 12
    rho = 1.0 + 0.5 * rng.random((ny, nx))
    u = rng.uniform(-0.5, 0.5, (ny, nx))
    v = rng.uniform(-0.5, 0.5, (ny, nx))
    p = 1.0 + rng.random((ny, nx))
    U0 = _state(rho, u, v, p)
    walls = hp.Problem("walls", nx, ny, U0, ("periodic", "periodic", "reflect", "reflect"))
    T = hp.transpose(U0)  # mirror in y through the transpose and the x mirror
    D = hp.transpose(_mirror_x(T))
    box = hp.Problem("box", nx, 2 * ny, D, ("periodic",) * 4, domain=(0.0, 1.0, 0.0, 2.0))
    Uw, Ub = walls.U.copy(), box.U.copy()
    oracle.advance(_params(walls), Uw, nsteps=6)
    oracle.advance(_params(box), Ub, nsteps=6)
    np.testing.assert_allclose(_interior(Uw), _interior(Ub)[:, :ny, :], rtol=1e-12, atol=1e-12)


def test_hydrostatic_ghost_cells():
    pr = hp.rt(16, 24)
    P = _params(pr)
    U = pr.U.copy()
    oracle.fill_ghost(P, U)
    dy = 3.0 / 24
    g = pr.grav
    for j, edge in [(k, NG) for k in range(NG)] + [(k, NG + 23) for k in range(NG + 24, 24 + 2 * NG)]:
        for k in range(3):
            np.testing.assert_array_equal(U[k, j, NG:-NG], U[k, edge, NG:-NG])
        rho, mx, my, E = (U[k, edge, NG:-NG] for k in range(4))
        ke = 0.5 * (mx ** 2 + my ** 2) / rho
        p_edge = 0.4 * (E - ke)
        p_ghost = 0.4 * (U[3, j, NG:-NG] - ke)
        np.testing.assert_allclose(p_ghost, p_edge + rho * g * (j - edge) * dy, rtol=1e-13)


def test_rayleigh_taylor_column_without_perturbation_stays_nearly_at_rest():
    # hydrostatic set-up (cell-centre pressures, hydrostatic ghost cells): the discrete balance is not
    # exact, so small velocities appear, but they stay a small fraction of free fall from rest
    pr = hp.rt(16, 48, amp=0.0)
    U = pr.U.copy()
    t, n = oracle.advance(_params(pr), U, nsteps=40)
    vmax = np.abs(_interior(U)[2] / _interior(U)[0]).max()
    assert vmax < 0.005 * abs(pr.grav) * t, (vmax, t)  # observed 0.0015 of free fall after 40 steps
    # the density profile keeps its place (observed change 3e-3, at the interface; without the half-step
    # gravity of the traced states the column slumps by 0.11)
    drho = np.abs(_interior(U)[0] - _interior(pr.U)[0]).max()
    assert drho < 0.01, drho


def test_rayleigh_taylor_stays_mirror_symmetric():
    pr = hp.rt(16, 48)
    U = pr.U.copy()
    oracle.advance(_params(pr), U, nsteps=20)
    I = _interior(U)
    M = I[:, :, ::-1].copy()
    M[1] *= -1.0
    # the perturbation cos(2 pi x) is even about x = 1/2 on cell centres: the run is too (to rounding)
    np.testing.assert_allclose(I, M, rtol=1e-12, atol=1e-13)
    # the seeded mode keeps its sign pattern: light fluid rising at the edges (cos(2 pi x) > 0), heavy fluid
    # falling at the centre
    v = I[2] / I[0]
    assert v[:, 0].max() > 0.3 * 0.01 and v[:, I.shape[2] // 2].min() < -0.3 * 0.01


def test_buoyant_bubble_rises_and_stays_mirror_symmetric():
    pr = hp.bubble(32, 64)
    U = pr.U.copy()
    X, Y = np.meshgrid((np.arange(32) + 0.5) / 32, (np.arange(64) + 0.5) / 32)
    atm = np.exp(-Y)

    def deficit_height(V):
        w = np.maximum(atm - _interior(V)[0], 0.0)
        return (w * Y).sum() / w.sum()

    y0 = deficit_height(U)
    oracle.advance(_params(pr), U, nsteps=120)
    # the light gas rises (observed: centroid of the density deficit from 0.49 to 0.66 in 120 steps)
    assert deficit_height(U) > y0 + 0.1
    I = _interior(U)
    M = I[:, :, ::-1].copy()
    M[1] *= -1.0
    np.testing.assert_allclose(I, M, rtol=1e-12, atol=1e-13)
