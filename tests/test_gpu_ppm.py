"""GPU parity of piecewise-parabolic reconstruction (the PPM upgrade paper §3.2 points to) against the FP64
oracle, through the C ABI: FP64 steps with either Riemann solver and driver loops (fused unsplit launch, the
fused launch with reflecting / hydrostatic sides and gravity, and the split sweeps) equal the oracle's bit
for bit; FP32 steps stay within the bound of the piecewise-linear path.
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


def _oparams(pr, **kw):
    xmin, xmax, ymin, ymax = pr.domain
    return oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl, xmin=xmin, xmax=xmax, ymin=ymin,
                         ymax=ymax, grav=pr.grav, reconstruction="ppm", **kw)


def _interior(U):
    return U[:, NG:-NG, NG:-NG]


PROBLEMS = {
    "sod_x_128x8": lambda: hp.sod(128, 8),
    "sod_y_8x128": lambda: hp.sod(8, 128, direction="y"),
    "kh_100x70": lambda: hp.kh(100, 70, seed=1),
    "sedov_100": lambda: hp.sedov(100, 100, r_init=0.05),
    "quad_70x50": lambda: hp.quad(70, 50, seed=3),
    "pulse_64": lambda: hp.pulse(64, 64),
    "quad_1x1": lambda: hp.quad(1, 1, seed=4),
    "quad_17x33": lambda: hp.quad(17, 33, seed=6),
    "rt_32x96": lambda: hp.rt(32, 96),
    "bubble_32x64": lambda: hp.bubble(32, 64),
}


@pytest.mark.parametrize("solver", ["two-shock", "hllc"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_fp64_ppm_step_matches_the_oracle(name, solver):
    H, Solver, params_for = _mods()
    pr = PROBLEMS[name]()
    s = Solver(params_for(pr, reconstruction="ppm", riemann_solver=solver), pr.U)
    s.fill_ghost()
    Uin = s.state_numpy()
    dt = s.cfl_dt()
    s.step(dt)
    st, stats = s.status(raise_on_error=False)
    out = s.state_numpy()
    s.close()
    assert st == 0 and stats[0] > 0
    po = _oparams(pr, riemann_solver=solver)
    U = np.array(Uin, dtype=np.float64)
    oracle.fill_ghost(po, U)
    oracle.step(po, U, dt)
    np.testing.assert_array_equal(_interior(out), _interior(U))


@pytest.mark.parametrize("name,nsteps,split,solver", [("kh_100x70", 25, False, "two-shock"),
                                                      ("sedov_100", 15, False, "two-shock"),
                                                      ("quad_70x50", 20, False, "hllc"),
                                                      ("rt_32x96", 20, False, "two-shock"),
                                                      ("kh_100x70", 20, True, "two-shock"),
                                                      ("sedov_100", 15, True, "hllc"),
                                                      ("bubble_32x64", 20, True, "hllc")])
def test_fp64_ppm_driver_loop_is_bit_identical_to_the_oracle_loop(name, nsteps, split, solver):
    H, Solver, params_for = _mods()
    pr = PROBLEMS[name]()
    s = Solver(params_for(pr, reconstruction="ppm", riemann_solver=solver, split=int(split)), pr.U)
    s.advance(nsteps)
    t, n = s.time()
    got = s.state_numpy()
    s.close()
    U = np.array(pr.U, dtype=np.float64)
    to, no = oracle.advance(_oparams(pr, riemann_solver=solver), U, nsteps=nsteps, split=split)
    assert n == no == nsteps and t == to
    np.testing.assert_array_equal(_interior(got), _interior(U))


@pytest.mark.parametrize("name", ["sod_x_128x8", "kh_100x70", "sedov_100", "quad_70x50", "pulse_64"])
def test_fp32_ppm_step_error_is_within_its_bound(name):
    H, Solver, params_for = _mods()
    pr = PROBLEMS[name]()
    s = Solver(params_for(pr, H.HYDRO_FP32, reconstruction="ppm"), pr.U)
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
    oracle.step(po, U, dt)
    ref = _interior(U)
    scale = np.abs(ref).reshape(4, -1).max(axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    err = np.abs(_interior(out).astype(np.float64) - ref).reshape(4, -1).max(axis=1) / scale
    assert np.all(err <= 2e-5), err
