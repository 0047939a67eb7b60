"""GPU parity of the gravity source and the reflecting / hydrostatic boundaries (paper §3.2: the rho g and
rho U.g sources of the Euler equations, and the Rayleigh-Taylor problem's hydrostatic walls) against the
FP64 oracle, through the C ABI.

* ghost fill: bit equality for every combination of outflow, periodic, reflecting and hydrostatic sides, in
  both state precisions (the hydrostatic energy is formed in double on both sides);
* one FP64 step and FP64 driver loops (the fused launch, which reads reflecting and hydrostatic sides through
  the boundary map): bit equality with the oracle;
* FP32: one step within the same bound as the other problems;
* ensembles: a Rayleigh-Taylor member evolves exactly as the same problem alone.
"""
import numpy as np
import pytest

import hydro_problems as hp
import oracle

pytestmark = pytest.mark.gpu

NG = 4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6883_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _mods():
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for
    return H, Solver, params_for


def _oparams(pr):
    xmin, xmax, ymin, ymax = pr.domain
    return oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl, xmin=xmin, xmax=xmax, ymin=ymin,
                         ymax=ymax, grav=pr.grav)


def _interior(U):
    return U[:, NG:-NG, NG:-NG]


def _random_box(nx, ny, bc, grav, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.5 * rng.random((ny, nx))
    u = rng.uniform(-0.5, 0.5, (ny, nx))
    v = rng.uniform(-0.5, 0.5, (ny, nx))
    p = 1.0 + rng.random((ny, nx))
    return hp.Problem("box", nx, ny, hp._pack(rho, u, v, p, 1.4), bc, grav=grav)


PROBLEMS = {
    "rt_32x96": lambda: hp.rt(32, 96),
    "rt_37x50_ragged": lambda: hp.rt(37, 50),
    "walls_grav_45x33": lambda: _random_box(45, 33, ("reflect",) * 4, -1.5, 1),
    "walls_x_periodic_y_29x40": lambda: _random_box(29, 40, ("reflect", "reflect", "periodic", "periodic"), 0.0, 2),
    "outflow_x_hydro_y_40x24": lambda: _random_box(40, 24, ("outflow", "outflow", "hydrostatic", "hydrostatic"),
                                                   -2.0, 3),
    "reflect_lo_outflow_hi_20x20": lambda: _random_box(20, 20, ("reflect", "outflow", "reflect", "outflow"), 0.7, 4),
    "fall_periodic_48x40": lambda: _random_box(48, 40, ("periodic",) * 4, -1.0, 5),
    "rt_4x4": lambda: hp.rt(4, 4),
    "bubble_32x64": lambda: hp.bubble(32, 64),
}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("bc", [("reflect",) * 4, ("reflect", "reflect", "hydrostatic", "hydrostatic"),
                                ("periodic", "periodic", "hydrostatic", "reflect"),
                                ("outflow", "reflect", "reflect", "hydrostatic"),
                                ("reflect", "outflow", "periodic", "periodic")])
@pytest.mark.parametrize("shape", [(13, 9), (64, 64), (37, 100)])
def test_ghost_fill_is_bit_exact(precision, bc, shape):
    H, Solver, params_for = _mods()
    nx, ny = shape
    rng = np.random.default_rng(nx * 1000 + ny + 7)
    U = np.zeros((4, ny + 2 * NG, nx + 2 * NG))
    U[0, NG:-NG, NG:-NG] = rng.uniform(0.5, 2.0, size=(ny, nx))
    U[1:3, NG:-NG, NG:-NG] = rng.uniform(-1.0, 1.0, size=(2, ny, nx))
    U[3, NG:-NG, NG:-NG] = rng.uniform(3.0, 6.0, size=(ny, nx))
    p = H.default_params(nx, ny, precision, bc=bc, grav=-1.25, ymax=2.0)
    s = Solver(p, U)
    s.fill_ghost()
    got = s.state_numpy()
    s.close()
    ref = np.array(U, dtype=np.float32 if precision else np.float64).astype(np.float64)
    oracle.fill_ghost(oracle.params(nx, ny, bc=bc, grav=-1.25, ymax=2.0), ref)
    if precision:
        # the hydrostatic energy is formed in double from the float state and rounded once to float
        np.testing.assert_array_equal(got, ref.astype(np.float32))
    else:
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_fp64_step_matches_the_oracle(name):
    H, Solver, params_for = _mods()
    pr = PROBLEMS[name]()
    s = Solver(params_for(pr), pr.U)
    s.fill_ghost()
    Uin = s.state_numpy()
    dt = s.cfl_dt()
    s.step(dt)
    st, _ = s.status(raise_on_error=False)
    out = s.state_numpy()
    s.close()
    assert st == 0
    po = _oparams(pr)
    U = np.array(Uin, dtype=np.float64)
    oracle.fill_ghost(po, U)
    assert oracle.cfl_dt(po, U) == dt
    oracle.step(po, U, dt)
    np.testing.assert_array_equal(_interior(out), _interior(U))


@pytest.mark.parametrize("name,nsteps", [("rt_32x96", 30), ("walls_grav_45x33", 20),
                                         ("outflow_x_hydro_y_40x24", 20), ("fall_periodic_48x40", 20),
                                         ("bubble_32x64", 40)])
def test_fp64_driver_loop_is_bit_identical_to_the_oracle_loop(name, nsteps):
    # the fused launch reads reflecting / hydrostatic sides through the boundary map (bc_cell) and periodic
    # sides through the wrap; both against the oracle's fill / dt / step loop
    H, Solver, params_for = _mods()
    pr = PROBLEMS[name]()
    s = Solver(params_for(pr), pr.U)
    s.advance(nsteps)
    t, n = s.time()
    got = s.state_numpy()
    s.close()
    U = np.array(pr.U, dtype=np.float64)
    to, no = oracle.advance(_oparams(pr), U, nsteps=nsteps)
    assert n == no == nsteps and t == to
    np.testing.assert_array_equal(_interior(got), _interior(U))


@pytest.mark.parametrize("name", ["rt_32x96", "walls_grav_45x33", "outflow_x_hydro_y_40x24", "fall_periodic_48x40",
                                  "bubble_32x64"])
def test_fp32_step_error_is_within_its_bound(name):
    # the same bound as the problems without gravity: float rounding of ~10^2 dependent operations per output.
    # Momenta are measured against rho c as well as their own size: the pressure term of the momentum flux
    # carries a float error ~eps p, which a step of dt ~ dx / c turns into ~eps rho c of momentum, however
    # small the momentum itself (the Rayleigh-Taylor run starts with u = 0 and v of order 1e-2)
    H, Solver, params_for = _mods()
    pr = PROBLEMS[name]()
    s = Solver(params_for(pr, H.HYDRO_FP32), pr.U)
    s.fill_ghost()
    Uin = s.state_numpy()
    dt = s.cfl_dt()
    s.step(dt)
    st, _ = s.status(raise_on_error=False)
    out = s.state_numpy()
    s.close()
    assert st == 0
    po = _oparams(pr)
    U = np.array(Uin, dtype=np.float64)
    oracle.fill_ghost(po, U)
    dto = oracle.cfl_dt(po, U)
    assert abs(dt - dto) <= 1e-6 * dto
    oracle.step(po, U, dt)
    ref = _interior(U)
    scale = np.abs(ref).reshape(4, -1).max(axis=1)
    pres = (pr.gamma - 1.0) * (ref[3] - 0.5 * (ref[1] ** 2 + ref[2] ** 2) / ref[0])
    rho_c = np.sqrt(pr.gamma * pres * ref[0]).max()
    scale[1:3] = np.maximum(scale[1:3], rho_c)
    err = np.abs(_interior(out).astype(np.float64) - ref).reshape(4, -1).max(axis=1) / scale
    assert np.all(err <= 2e-5), err


def test_rayleigh_taylor_fp32_run_tracks_the_fp64_run():
    # 200 steps of the paper's Rayleigh-Taylor set-up at 64 x 192: the FP32 state stays within float
    # rounding accumulated over the run of the FP64 one (L1 relative, density and energy)
    H, Solver, params_for = _mods()
    pr = hp.rt(64, 192)
    runs = {}
    for precision in (0, 1):
        s = Solver(params_for(pr, precision), pr.U)
        s.advance(200)
        runs[precision] = (_interior(s.state_numpy()).astype(np.float64), s.time())
        s.close()
    (a, (ta, na)), (b, (tb, nb)) = runs[0], runs[1]
    assert na == nb == 200 and tb == pytest.approx(ta, rel=1e-5)
    l1 = np.abs(b - a).reshape(4, -1).sum(1) / np.abs(a).reshape(4, -1).sum(1)
    assert l1[0] < 1e-5 and l1[3] < 1e-5, l1


@pytest.mark.parametrize("precision", [0, 1])
def test_rayleigh_taylor_member_evolves_as_alone(precision):
    from paper_1306_6883_gb300.solver import Ensemble, Solver, params_for
    probs = [hp.rt(32, 96), hp.quad(40, 40, seed=3), hp.rt(24, 72, grav=-0.5),
             _random_box(30, 30, ("reflect",) * 4, -1.0, 9)]
    e = Ensemble([params_for(p, precision) for p in probs], [p.U for p in probs])
    e.run(8)
    st, _ = e.status()
    assert st == 0
    for i, pr in enumerate(probs):
        s = Solver(params_for(pr, precision), pr.U)
        s.advance(8)
        ref = _interior(s.state_numpy())
        s.close()
        got = _interior(e.state_numpy(i))
        if precision == 0:
            np.testing.assert_array_equal(got, ref)
        else:
            np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-6)
    e.close()
