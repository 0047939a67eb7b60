"""GPU parity of the dimensionally split variant (paper §3.1: one-dimensional sweeps along x and y, each on
the state the other left, order alternating from step to step) against the FP64 oracle, through the C ABI.
The sweeps read cells outside the domain through the boundary map (outflow, periodic, reflecting and
hydrostatic sides), where the oracle fills ghost cells before each sweep.

FP64: one split step from identical input equals the oracle's bit for bit, for both sweep orders, every
option and ragged / degenerate grids; whole driver loops (the order alternating) equal the oracle's loop bit
for bit, and the Riemann solve counts equal the oracle's.  FP32: one step within the bound of the unsplit
step; 50 KH 1024^2 steps track the FP64 run.
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
                         ymax=ymax, grav=pr.grav, **kw)


def _interior(U):
    return U[:, NG:-NG, NG:-NG]


def _random_box(nx, ny, bc, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.5 * rng.random((ny, nx))
    u = rng.uniform(-0.5, 0.5, (ny, nx))
    v = rng.uniform(-0.5, 0.5, (ny, nx))
    p = 1.0 + rng.random((ny, nx))
    return hp.Problem("box", nx, ny, hp._pack(rho, u, v, p, 1.4), bc)


PROBLEMS = {
    "sod_x_128x8": lambda: hp.sod(128, 8),
    "sod_y_8x128": lambda: hp.sod(8, 128, direction="y"),
    "kh_100x70": lambda: hp.kh(100, 70, seed=1),
    "sedov_100": lambda: hp.sedov(100, 100, r_init=0.05),
    "quad_70x50": lambda: hp.quad(70, 50, seed=3),
    "quad_131x37": lambda: hp.quad(131, 37, seed=8),
    "pulse_64": lambda: hp.pulse(64, 64),
    "quad_1x1": lambda: hp.quad(1, 1, seed=4),
    "quad_5x3": lambda: hp.quad(5, 3, seed=5),
    "kh_4x4": lambda: hp.kh(4, 4, seed=2),
    "walls_45x33": lambda: _random_box(45, 33, ("reflect",) * 4, 1),
    "mixed_walls_70x66": lambda: _random_box(70, 66, ("reflect", "outflow", "hydrostatic", "reflect"), 2),
    "rt_32x96": lambda: hp.rt(32, 96),
    "bubble_32x64": lambda: hp.bubble(32, 64),
    "rt_37x50": lambda: hp.rt(37, 50),
}


def _gpu_steps(pr, nsteps, precision=0, **kw):
    """nsteps host-driven split steps (fill, dt, step) from pr.U; returns (inputs, outputs, dts, stats)."""
    H, Solver, params_for = _mods()
    s = Solver(params_for(pr, precision, split=1, **kw), pr.U)
    ins, outs, dts = [], [], []
    for _ in range(nsteps):
        s.fill_ghost()
        ins.append(s.state_numpy())
        dt = s.cfl_dt()
        s.step(dt)
        dts.append(dt)
        outs.append(s.state_numpy())
    st, stats = s.status(raise_on_error=False)
    s.close()
    assert st == 0
    return ins, outs, dts, stats


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_fp64_split_steps_match_the_oracle(name):
    # two steps: the first sweeps x first, the second y first
    pr = PROBLEMS[name]()
    ins, outs, dts, stats = _gpu_steps(pr, 2)
    po = _oparams(pr)
    ost = oracle.OracleStats()
    for k in range(2):
        U = np.array(ins[k], dtype=np.float64)
        oracle.fill_ghost(po, U)
        assert oracle.cfl_dt(po, U) == dts[k]
        oracle.step_split(po, U, dts[k], k % 2, ost)
        np.testing.assert_array_equal(_interior(outs[k]), _interior(U))
    assert (stats[0], stats[1], stats[2]) == (ost.riemann_solves, ost.riemann_iters, ost.riemann_nonconv)


@pytest.mark.parametrize("opts", [dict(limiter=0), dict(limiter=1), dict(use_flattening=0), dict(cvisc=0.0)])
def test_fp64_split_step_matches_the_oracle_for_every_option(opts):
    pr = hp.quad(45, 38, seed=11)
    ins, outs, dts, _ = _gpu_steps(pr, 2, **opts)
    po = _oparams(pr, **opts)
    for k in range(2):
        U = np.array(ins[k], dtype=np.float64)
        oracle.fill_ghost(po, U)
        oracle.step_split(po, U, dts[k], k % 2)
        np.testing.assert_array_equal(_interior(outs[k]), _interior(U))


@pytest.mark.parametrize("name,nsteps", [("kh_100x70", 25), ("quad_131x37", 20), ("sedov_100", 15),
                                         ("sod_x_128x8", 30), ("mixed_walls_70x66", 20), ("rt_32x96", 30)])
def test_fp64_split_driver_loop_is_bit_identical_to_the_oracle_loop(name, nsteps):
    H, Solver, params_for = _mods()
    pr = PROBLEMS[name]()
    s = Solver(params_for(pr, split=1), pr.U)
    s.advance(nsteps)
    t, n = s.time()
    got = s.state_numpy()
    s.close()
    U = np.array(pr.U, dtype=np.float64)
    to, no = oracle.advance(_oparams(pr), U, nsteps=nsteps, split=True)
    assert n == no == nsteps and t == to
    np.testing.assert_array_equal(_interior(got), _interior(U))


def test_fused_entry_points_run_the_split_passes():
    # hydro_step_fused and hydro_step_device_dt with split = 1 equal the host-driven loop bit for bit
    H, Solver, params_for = _mods()
    pr = hp.kh(64, 48, seed=5)
    a = Solver(params_for(pr, split=1), pr.U)
    b = Solver(params_for(pr, split=1), pr.U)
    for k in range(6):
        a.step_fused()
        b.fill_ghost()
        b.cfl_dt_async()
        b.step_device_dt()
    np.testing.assert_array_equal(_interior(a.state_numpy()), _interior(b.state_numpy()))
    assert a.time() == b.time()
    a.close()
    b.close()


@pytest.mark.parametrize("name", ["sod_x_128x8", "kh_100x70", "sedov_100", "quad_70x50", "pulse_64", "rt_32x96"])
def test_fp32_split_step_error_is_within_its_bound(name):
    pr = PROBLEMS[name]()
    ins, outs, dts, _ = _gpu_steps(pr, 1, precision=1)
    po = _oparams(pr)
    U = np.array(ins[0], dtype=np.float64)
    oracle.fill_ghost(po, U)
    dto = oracle.cfl_dt(po, U)
    assert abs(dts[0] - dto) <= 1e-6 * dto
    oracle.step_split(po, U, dts[0], 0)
    ref = _interior(U)
    scale = np.abs(ref).reshape(4, -1).max(axis=1)
    # momenta also against rho c: a step's float error in the pressure term is ~eps rho c of momentum, however
    # small the momentum (the Rayleigh-Taylor run starts with u = 0)
    pres = (pr.gamma - 1.0) * (ref[3] - 0.5 * (ref[1] ** 2 + ref[2] ** 2) / ref[0])
    scale[1:3] = np.maximum(scale[1:3], np.sqrt(pr.gamma * pres * ref[0]).max())
    err = np.abs(_interior(outs[0]).astype(np.float64) - ref).reshape(4, -1).max(axis=1) / scale
    assert np.all(err <= 2e-5), err


def test_kh_1024_fp32_split_run_tracks_the_fp64_split_run():
    H, Solver, params_for = _mods()
    pr = hp.kh(1024, 1024, seed=0)
    out = {}
    for precision in (0, 1):
        s = Solver(params_for(pr, precision, split=1), pr.U)
        tot0 = np.array(s.totals())
        s.advance(50)
        out[precision] = (_interior(s.state_numpy()).astype(np.float64), s.time(), np.array(s.totals()) - tot0)
        s.close()
    (a, (ta, na), da), (b, (tb, nb), db) = out[0], out[1]
    assert na == nb == 50 and tb == pytest.approx(ta, rel=1e-6)
    l1 = np.abs(b - a).reshape(4, -1).sum(1) / np.abs(a).reshape(4, -1).sum(1)
    # the unsplit FP32 path after 50 KH steps: 1.4e-7, 2.4e-7, 1.6e-4 (the small rho v field), 1.0e-7
    assert np.all(l1 <= np.array([2e-6, 3e-6, 2e-3, 1.5e-6])), l1
    scale = np.abs(a).sum(axis=(1, 2)) / a[0].size
    assert np.all(np.abs(da) <= 1e-13 * scale) and np.all(np.abs(db) <= 1e-8 * scale), (da, db)
