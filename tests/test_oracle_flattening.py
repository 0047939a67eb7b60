"""Pins of the oracle's flattening pass (paper §3.2: flattening "from Colella 1990", whose shock detector and
spreading rule are those of Colella & Woodward 1984).

Reading pinned here: per direction, each cell takes the stronger flattening (the smaller chi) of itself and of
its lower-pressure neighbour, xi_d(i) = min(chi_i, chi_{i-s}) with s = sign(p_{i+1} - p_{i-1}); a shock's
flattened band therefore reaches exactly one cell further into its high-pressure (post-shock) side and none
into the low-pressure side.  The two directions combine as xi = min(xi_x, xi_y).  The tests state these
properties on shaped profiles and on a shock the oracle itself produces, so that taking the other neighbour,
combining the directions by max, or moving the detector's constants each fails a pin."""
import numpy as np
import pytest

import hydro_problems as hp
import oracle

NG = 4


def _prims_x(p_line, u_line, rho_line, ny=6):
    """Primitive planes (rho, u, v, p) of a padded grid varying along x only (every row the same line)."""
    nx = len(p_line) - 2 * NG
    q = np.zeros((4, ny + 2 * NG, nx + 2 * NG))
    q[0] = rho_line
    q[1] = u_line
    q[3] = p_line
    return q, oracle.params(nx, ny)


def _chi_line(p_line, u_line):
    """The shock detector (pinned by hand values below) on every cell of a line, 1 where its stencil is cut."""
    n = len(p_line)
    chi = np.ones(n)
    for i in range(2, n - 2):
        chi[i] = oracle.flatten_chi(p_line[i - 2], p_line[i - 1], p_line[i + 1], p_line[i + 2], u_line[i - 1],
                                    u_line[i + 1])
    return chi


# two shock profiles a Godunov scheme leaves (the jump over two or three cells, gas decelerating into the
# high-pressure side); a faint background gradient keeps the sign s of every cell defined
RAMP = (np.array([1.0, 1.0, 1.02, 1.6, 8.5, 9.9, 9.98, 10.0, 10.0]),
        np.array([1.0, 1.0, 0.98, 0.8, 0.2, 0.02, 0.0, 0.0, 0.0]))
WIDE_RAMP = (np.array([1.0, 1.0, 1.1, 3.0, 8.6, 9.9, 10.0, 10.0, 10.0]),
             np.array([1.0, 1.0, 0.98, 0.8, 0.2, 0.02, 0.0, 0.0, 0.0]))


def _smeared_shock(n=28, rising_right=True, shape=RAMP):
    """A compressive jump: pressure 1 -> 10, velocity 1 -> 0, density 1 -> 3, placed left of the middle of
    n interior cells; mirrored (pressure falling to the right, velocity reversed) when rising_right is False."""
    ramp, uramp = shape
    k0 = 10
    m = n + 2 * NG
    p = np.concatenate([np.ones(k0), ramp, np.full(m - k0 - len(ramp), 10.0)]) + 1e-3 * np.arange(m)
    u = np.concatenate([np.ones(k0), uramp, np.zeros(m - k0 - len(uramp))])
    rho = 1.0 + 2.0 * (p - 1.0) / 9.0
    if not rising_right:
        p, rho, u = p[::-1].copy(), rho[::-1].copy(), -u[::-1].copy()
    return p, u, rho


@pytest.mark.parametrize("rising_right", [True, False])
def test_flattened_band_reaches_one_cell_into_the_high_pressure_side(rising_right):
    p, u, rho = _smeared_shock(rising_right=rising_right)
    q, prm = _prims_x(p, u, rho)
    xi = oracle.flatten_xi(prm, q)
    chi = _chi_line(p, u)
    row = xi[NG + 2]
    np.testing.assert_array_equal(xi[NG:-NG], np.broadcast_to(row, xi[NG:-NG].shape))  # every row alike
    inner = np.arange(3, len(p) - 3)
    detected = [i for i in inner if chi[i] < 1.0]
    flattened = [i for i in inner if row[i] < 1.0]
    assert len(detected) >= 2, detected
    lo, hi = min(detected), max(detected)
    if rising_right:  # post-shock side is to the right: the band grows by one cell there only
        assert flattened == list(range(lo, hi + 2)), (detected, flattened)
        assert row[hi + 1] == chi[hi]
    else:
        assert flattened == list(range(lo - 1, hi + 1)), (detected, flattened)
        assert row[lo - 1] == chi[lo]
    # no cell is flattened less than its own detector asks
    assert np.all(row[inner] <= chi[inner])


def test_mirror_image_gives_the_mirrored_coefficients():
    p, u, rho = _smeared_shock(rising_right=True)
    q, prm = _prims_x(p, u, rho)
    pm, um, rhom = _smeared_shock(rising_right=False)
    qm, _ = _prims_x(pm, um, rhom)
    np.testing.assert_array_equal(oracle.flatten_xi(prm, q)[:, 3:-3], oracle.flatten_xi(prm, qm)[:, ::-1][:, 3:-3])


def test_a_shock_along_x_alone_flattens_its_cells_and_transposes():
    # the y direction sees a uniform column: its detector leaves every cell alone, so the cells of the x shock
    # must keep their x flattening (the directions combine by the minimum)
    p, u, rho = _smeared_shock()
    q, prm = _prims_x(p, u, rho)
    xi = oracle.flatten_xi(prm, q)
    assert xi.min() == 0.0 or xi.min() < 0.5
    assert (xi[NG:-NG] < 1.0).sum() >= 2 * (xi.shape[0] - 2 * NG)
    # the transposed problem (shock along y, v the normal velocity) gives the transposed field bitwise
    qt = np.ascontiguousarray(np.transpose(q, (0, 2, 1)))
    qt[[1, 2]] = qt[[2, 1]]
    prmt = oracle.params(prm.ny, prm.nx)
    np.testing.assert_array_equal(oracle.flatten_xi(prmt, qt), xi.T)


def test_crossing_shocks_take_the_stronger_direction():
    # a shock along x in every row and a weaker one along y in every column: where both act, xi is the
    # smaller of the two one-direction fields
    p, u, rho = _smeared_shock()
    qx, prm = _prims_x(p, u, rho, ny=len(p) - 2 * NG)
    xix = oracle.flatten_xi(prm, qx)
    p2, u2, rho2 = _smeared_shock(shape=WIDE_RAMP)
    qw, _ = _prims_x(p2, u2, rho2, ny=len(p) - 2 * NG)
    qy = np.ascontiguousarray(np.transpose(qw, (0, 2, 1)))  # the other shock, along y
    qy[[1, 2]] = qy[[2, 1]]
    xiy = oracle.flatten_xi(prm, qy)
    assert np.any(xix != xiy.T)
    both = qx.copy()
    both[2] = qy[2]
    # a product keeps each direction's pressure profile up to a constant factor along its own lines, which
    # leaves the detector (a ratio of differences and a relative jump) and the sign s unchanged
    both[3] = qx[3] * qy[3]
    xi = oracle.flatten_xi(prm, both)
    assert ((xix < 1.0) & (xiy < 1.0) & (xix != xiy)).sum() > 0
    np.testing.assert_allclose(xi, np.minimum(xix, xiy), rtol=0, atol=1e-12)


def test_sod_shock_band_extends_into_the_post_shock_gas():
    # the Sod shock runs right into the low-pressure gas, so its post-shock (high-pressure) side is its left
    pr = hp.sod(128, 4)
    prm = oracle.params(pr.nx, pr.ny, bc=pr.bc)
    U = pr.U.copy()
    oracle.advance(prm, U, tmax=0.15)
    q = np.stack([np.array([oracle.cons_to_prim(prm, U[:, j, i]) for i in range(U.shape[2])])
                  for j in range(U.shape[1])]).transpose(2, 0, 1).copy()
    xi = oracle.flatten_xi(prm, q)[NG + 1]
    pline, uline = q[3, NG + 1], q[1, NG + 1]
    chi = _chi_line(pline, uline)
    # the shock sits where the pressure falls fastest to the right of the contact (x > 0.6)
    i_shock = NG + int(np.argmin(np.diff(pline[NG + 77:NG + 128]))) + 77
    win = range(i_shock - 6, i_shock + 7)
    detected = [i for i in win if chi[i] < 1.0]
    flattened = [i for i in win if xi[i] < 1.0]
    assert detected, "the detector must see the Sod shock"
    assert flattened == list(range(min(detected) - 1, max(detected) + 1)), (detected, flattened)


def test_detector_constants():
    # ramp between z = 0.75 (chi = 1) and z = 0.85 (chi = 0), linear in between
    for z, want in ((0.76, 0.9), (0.80, 0.5), (0.84, 0.1), (0.70, 1.0), (0.90, 0.0)):
        # |p_{+1} - p_{-1}| = 9, |p_{+2} - p_{-2}| = 9 / z
        h = 0.5 * (9.0 / z - 9.0)
        chi = oracle.flatten_chi(10.0 - h, 10.0, 19.0, 19.0 + h, 1.0, 0.0)
        assert chi == pytest.approx(want, abs=1e-12), (z, chi)
    # the jump test: |p_{+1} - p_{-1}| must exceed 0.33 of the smaller pressure (z = 1 whenever it does)
    assert oracle.flatten_chi(1.0, 1.0, 1.35, 1.35, 1.0, 0.0) == 0.0
    assert oracle.flatten_chi(1.0, 1.0, 1.32, 1.32, 1.0, 0.0) == 1.0
    assert oracle.flatten_chi(10.0, 10.0, 13.4, 13.4, 1.0, 0.0) == 0.0
    assert oracle.flatten_chi(10.0, 10.0, 13.2, 13.2, 1.0, 0.0) == 1.0
