"""Whole-step pins of the oracle: invariants, conservation, x<->y symmetry, reduction to the scalar CTU
advection scheme (§3.1, Eqs. 3-5), Sod against the exact solution (§3.2.1) and second-order convergence
on the smooth pulse (§3.1.1, Eq. 7)."""
import numpy as np
import pytest

import exact_riemann as er
import hydro_problems as hp
import oracle

NG = 4


def _params(pr, **kw):
    return oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl, **kw)


def _interior(U, ng=NG):
    return U[:, ng:-ng, ng:-ng]


# ---------------------------------------------------------------- ghost cells, totals, dt
@pytest.mark.parametrize("bc,mode", [("outflow", "edge"), ("periodic", "wrap")])
def test_ghost_fill_matches_numpy_pad(bc, mode):
    rng = np.random.default_rng(0)
    nx, ny = 13, 9
    U = np.zeros((4, ny + 2 * NG, nx + 2 * NG))
    inner = rng.normal(size=(4, ny, nx))
    U[:, NG:-NG, NG:-NG] = inner
    p = oracle.params(nx, ny, bc=(bc,) * 4)
    oracle.fill_ghost(p, U)
    expect = np.stack([np.pad(inner[k], NG, mode=mode) for k in range(4)])
    np.testing.assert_array_equal(U, expect)


def test_mixed_boundaries_fill_corners_consistently():
    rng = np.random.default_rng(1)
    nx, ny = 10, 7
    inner = rng.normal(size=(4, ny, nx))
    U = np.zeros((4, ny + 2 * NG, nx + 2 * NG))
    U[:, NG:-NG, NG:-NG] = inner
    p = oracle.params(nx, ny, bc=("outflow", "outflow", "periodic", "periodic"))
    oracle.fill_ghost(p, U)
    expect = np.stack([np.pad(np.pad(inner[k], ((0, 0), (NG, NG)), mode="edge"), ((NG, NG), (0, 0)), mode="wrap")
                       for k in range(4)])
    np.testing.assert_array_equal(U, expect)


def test_conserved_totals_match_a_plain_sum():
    pr = hp.kh(32, 24)
    p = _params(pr)
    tot = oracle.conserved_totals(p, pr.U)
    dx, dy = 1 / 32, 1 / 24
    np.testing.assert_allclose(tot, _interior(pr.U).sum(axis=(1, 2)) * dx * dy, rtol=1e-14, atol=1e-16)


def test_dt_of_a_uniform_state_has_its_closed_form():
    g = 1.4
    rho, u, v, pres = 1.7, 0.3, -1.1, 2.2
    nx, ny = 16, 8
    U = np.zeros((4, ny + 8, nx + 8))
    U[0], U[1], U[2] = rho, rho * u, rho * v
    U[3] = pres / (g - 1) + 0.5 * rho * (u * u + v * v)
    p = oracle.params(nx, ny, xmax=2.0, cfl=0.7)
    c = np.sqrt(g * pres / rho)
    expect = 0.7 * min((2.0 / nx) / (abs(u) + c), (1.0 / ny) / (abs(v) + c))
    assert oracle.cfl_dt(p, U) == pytest.approx(expect, rel=1e-14)


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("bc", ["outflow", "periodic"])
@pytest.mark.parametrize("vel", [(0.0, 0.0), (0.37, -1.3)])
def test_uniform_flow_is_a_fixed_point(bc, vel):
    g = 1.4
    rho, pres = 0.8, 1.9
    nx, ny = 12, 10
    U = np.zeros((4, ny + 8, nx + 8))
    U[0], U[1], U[2] = rho, rho * vel[0], rho * vel[1]
    U[3] = pres / (g - 1) + 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2)
    p = oracle.params(nx, ny, bc=(bc,) * 4)
    U0 = U.copy()
    for _ in range(3):
        oracle.fill_ghost(p, U)
        oracle.step(p, U, oracle.cfl_dt(p, U))
    np.testing.assert_array_equal(_interior(U), _interior(U0))


def test_periodic_run_conserves_mass_momentum_energy():
    pr = hp.kh(64, 64, seed=3)
    p = _params(pr)
    U = pr.U.copy()
    t0 = oracle.conserved_totals(p, U)
    scale = np.abs(_interior(U)).sum(axis=(1, 2)) / (64 * 64)
    oracle.advance(p, U, nsteps=30)
    t1 = oracle.conserved_totals(p, U)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale


@pytest.mark.parametrize("maker", [lambda: hp.quad(24, 24, seed=7), lambda: hp.kh(24, 24, seed=2),
                                   lambda: hp.sedov(24, 24, r_init=0.1)])
def test_transposed_problem_gives_the_transposed_answer_bitwise(maker):
    pr = maker()
    p = _params(pr)
    bcT = (pr.bc[2], pr.bc[3], pr.bc[0], pr.bc[1])
    pT = oracle.params(pr.ny, pr.nx, bc=bcT)
    U, UT = pr.U.copy(), hp.transpose(pr.U)
    for _ in range(4):
        oracle.fill_ghost(p, U)
        oracle.fill_ghost(pT, UT)
        dt = oracle.cfl_dt(p, U)
        assert oracle.cfl_dt(pT, UT) == dt
        oracle.step(p, U, dt)
        oracle.step(pT, UT, dt)
    np.testing.assert_array_equal(_interior(hp.transpose(U)), _interior(UT))


# ---------------------------------------------------------------- reduction to scalar CTU advection
def _scalar_ctu(a, u, v, dt, dx, dy, limiter=2):
    """One step of the paper's CTU advection scheme (§3.1, Eqs. 3-5) on a periodic array a[j, i], with
    the fourth-order MC slope taken from the oracle (pinned on its own in test_oracle_stages)."""
    ny, nx = a.shape
    A = np.pad(a, NG, mode="wrap")

    def slope_x(j, i):
        return oracle.slope(limiter, *A[j, i - 2:i + 3])

    def slope_y(j, i):
        return oracle.slope(limiter, *A[j - 2:j + 3, i])

    sx, sy = dt / dx, dt / dy
    H = NY, NX = A.shape
    axl, axr, ayl, ayr = (np.zeros(H) for _ in range(4))
    for j in range(2, NY - 2):
        for i in range(2, NX - 2):
            dax, day = slope_x(j, i), slope_y(j, i)
            axl[j, i] = A[j, i] + 0.5 * (1 - sx * u) * dax    # hat state at i+1/2 from cell i (Eq. 4)
            axr[j, i] = A[j, i] - 0.5 * (1 + sx * u) * dax    # hat state at i-1/2 from cell i
            ayl[j, i] = A[j, i] + 0.5 * (1 - sy * v) * day
            ayr[j, i] = A[j, i] - 0.5 * (1 + sy * v) * day

    def up_x(j, f):  # upwind (Riemann) state at x face f, between cells f-1 and f
        return axl[j, f - 1] if u > 0 else axr[j, f]

    def up_y(g, i):
        return ayl[g - 1, i] if v > 0 else ayr[g, i]

    out = np.empty_like(a)
    fx = np.zeros(H)
    fy = np.zeros(H)
    for j in range(NG, NY - NG):
        for f in range(NG, NX - NG + 1):
            L = axl[j, f - 1] - 0.5 * dt * v / dy * (up_y(j + 1, f - 1) - up_y(j, f - 1))  # Eq. 3
            R = axr[j, f] - 0.5 * dt * v / dy * (up_y(j + 1, f) - up_y(j, f))
            fx[j, f] = u * (L if u > 0 else R)
    for g in range(NG, NY - NG + 1):
        for i in range(NG, NX - NG):
            L = ayl[g - 1, i] - 0.5 * dt * u / dx * (up_x(g - 1, i + 1) - up_x(g - 1, i))
            R = ayr[g, i] - 0.5 * dt * u / dx * (up_x(g, i + 1) - up_x(g, i))
            fy[g, i] = v * (L if v > 0 else R)
    for j in range(NG, NY - NG):
        for i in range(NG, NX - NG):
            out[j - NG, i - NG] = A[j, i] - dt / dx * (fx[j, i + 1] - fx[j, i]) - dt / dy * (fy[j + 1, i] - fy[j, i])  # Eq. 5
    return out


@pytest.mark.parametrize("u,v", [(0.7, 0.4), (-0.5, 0.3), (0.2, -0.9)])
def test_contact_advection_reduces_to_the_scalar_ctu_scheme(u, v):
    # uniform velocity and pressure: only the entropy (density) wave is present, and the Euler CTU
    # step must move density exactly like the paper's scalar CTU advection
    g = 1.4
    nx, ny = 20, 16
    rng = np.random.default_rng(9)
    rho = 1.0 + 0.5 * rng.uniform(size=(ny, nx))
    U = np.zeros((4, ny + 8, nx + 8))
    s = (slice(NG, -NG), slice(NG, -NG))
    U[0][s], U[1][s], U[2][s] = rho, rho * u, rho * v
    U[3][s] = 1.0 / (g - 1) + 0.5 * rho * (u * u + v * v)
    p = oracle.params(nx, ny, xmax=1.25, bc=("periodic",) * 4)
    oracle.fill_ghost(p, U)
    dt = oracle.cfl_dt(p, U)
    expect = _scalar_ctu(rho, u, v, dt, 1.25 / nx, 1.0 / ny)
    oracle.step(p, U, dt)
    np.testing.assert_allclose(U[0][s], expect, rtol=1e-12)
    # velocity and pressure stay uniform
    np.testing.assert_allclose(U[1][s] / U[0][s], u, rtol=1e-12)
    np.testing.assert_allclose(U[2][s] / U[0][s], v, rtol=1e-12)


# ---------------------------------------------------------------- Sod vs the exact solution
def _run_sod(direction, n=128, m=4):
    pr = hp.sod(n, m) if direction == "x" else hp.sod(m, n, direction="y")
    p = _params(pr)
    U = pr.U.copy()
    t, steps = oracle.advance(p, U, tmax=0.2)
    return U, t, steps


def test_sod_matches_the_exact_solution():
    U, t, steps = _run_sod("x")
    assert t == pytest.approx(0.2, rel=1e-14)
    rho = U[0, NG, NG:-NG]
    n = rho.size
    edges = np.linspace(0.0, 1.0, n + 1)
    exact = np.array(er.cell_averaged_density(edges, 0.2, 0.5, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)))
    l1 = np.abs(rho - exact).sum() / n
    assert l1 < 4e-3, l1
    # rows are identical (the problem is one-dimensional)
    for j in range(NG, U.shape[1] - NG):
        np.testing.assert_array_equal(U[:, j, NG:-NG], U[:, NG, NG:-NG])
    # shock position: exact x_s = 0.5 + S t; numerical: where rho crosses the mid-value of the jump
    ps, us = er.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
    S = np.sqrt(1.4 * 0.1 / 0.125) * np.sqrt(2.4 / 2.8 * ps / 0.1 + 0.4 / 2.8)
    rho_post = er.sample(S * 0.999, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)[0]
    mid = 0.5 * (rho_post + 0.125)
    xc = (np.arange(n) + 0.5) / n
    k = np.where((rho[:-1] >= mid) & (rho[1:] < mid))[0][-1]
    xs = xc[k] + (rho[k] - mid) / (rho[k] - rho[k + 1]) / n
    assert abs(xs - (0.5 + S * 0.2)) < 2.0 / n


def test_sod_along_y_is_the_transposed_run_bitwise():
    Ux, _, nx_steps = _run_sod("x")
    Uy, _, ny_steps = _run_sod("y")
    assert nx_steps == ny_steps
    np.testing.assert_array_equal(hp.transpose(Ux), Uy)


# ---------------------------------------------------------------- second order on the smooth pulse
def test_smooth_pulse_converges_at_second_order():
    errs = []
    ns = (32, 64, 128)
    for n in ns:
        pr = hp.pulse(n, n)
        p = _params(pr)
        U = pr.U.copy()
        t, _ = oracle.advance(p, U, tmax=0.25)
        xc = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(xc, xc)
        exact = 1.0 + sum(np.exp(-60.0 * ((X - 0.5 - t + a) ** 2 + (Y - 0.5 - t + b) ** 2))
                          for a in (-1, 0, 1) for b in (-1, 0, 1))
        errs.append(np.abs(U[0, NG:-NG, NG:-NG] - exact).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] >= 1.8, (errs, orders)


def test_forced_nonconvergence_is_counted():
    pr = hp.sod(16, 4)
    p = oracle.params(16, 4, bc=pr.bc, riemann_maxiter=1)
    U = pr.U.copy()
    oracle.fill_ghost(p, U)
    st = oracle.OracleStats()
    oracle.step(p, U, oracle.cfl_dt(p, U), st)
    assert st.riemann_nonconv > 0 and st.riemann_maxiters_seen == 1
