"""FP64 energy recovery of the FP32 path (paper §3.2, Eqs. 11-12: e = E - rho |u|^2 / 2), against the oracle.

At high Mach the internal energy is a small difference of two large numbers.  The FP32 path keeps the state
and the stencil in float but forms that difference in double wherever the kinetic energy exceeds 0.999 of the
total energy (recover_ke_frac): in the conversion of each tile cell (cons_to_prim), in the transversely
corrected face states (correct_state) and in the CFL value of a cell (cfl_value).  The workload is a Mach-100
uniform stream along x with seeded 1 % density noise, on a grid 1000 times finer in y than in x, so that the
time step is set by the sound speed (dy / c) and the y-direction solves are driven by pressure differences of
a part in 10^4: every cell takes the recovery branch.

Bounds (one FP32 step against the oracle's step from the same float-representable state, errors relative to
the largest change the oracle makes in that field over the step; GB300 measurements in brackets):
* rho, rho u, E: max 0.1 (0.015), mean 0.06 (0.0097); rho v: max 0.4 (0.069); CFL dt: 5e-7 (8.6e-8).
* With the recovery switched off (recover_ke_frac = 2) the same step errs by 0.53 (max) and the dt by 1.8e-4.
  Without the cell conversion's branch alone the step errs by 0.31, without the corrected states' by 0.23,
  and without the CFL branch the dt errs by 1.8e-4: each part of the recovery is needed for the bounds.
At low Mach the branch never fires: the Kelvin-Helmholtz step is the same bit for bit with and without it.
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


def _oracle_step(pr, U):
    xmin, xmax, ymin, ymax = pr.domain
    p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl, xmin=xmin, xmax=xmax, ymin=ymin,
                      ymax=ymax)
    U = U.copy()
    oracle.fill_ghost(p, U)
    dt = oracle.cfl_dt(p, U)
    Uin = U.copy()
    oracle.step(p, U, dt)
    return Uin[:, NG:-NG, NG:-NG], U[:, NG:-NG, NG:-NG], dt


def _gpu_step(pr, U, dt, **kw):
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for
    s = Solver(params_for(pr, H.HYDRO_FP32, **kw), U)
    s.fill_ghost()
    dt_gpu = s.cfl_dt()
    s.step(dt)
    st, _ = s.status(raise_on_error=False)
    out = s.interior().astype(np.float64)
    s.close()
    return out, dt_gpu, st


def _errors(got, ref, ref_in):
    change = np.abs(ref - ref_in).reshape(4, -1)
    d = np.abs(got - ref).reshape(4, -1)
    return d.max(1) / change.max(1), d.mean(1) / change.mean(1)


def _stream():
    pr = hp.stream(128, 128, mach=100.0, domain=(0.0, 1.0, 0.0, 0.001))
    U = pr.U.astype(np.float32).astype(np.float64)  # the float state both sides start from
    return pr, U


def test_every_cell_of_the_hypersonic_stream_takes_the_branch():
    pr, U = _stream()
    I = U[:, NG:-NG, NG:-NG].astype(np.float32)
    # the FP32 test of cons_to_prim: ke = rho (u^2 + v^2) / 2 from u = (rho u) / rho, against 0.999 E
    u, v = I[1] / I[0], I[2] / I[0]
    ke = np.float32(0.5) * I[0] * (u * u + v * v)
    assert np.all(ke > np.float32(0.999) * I[3])
    ke64 = 0.5 * (U[1] ** 2 + U[2] ** 2)[NG:-NG, NG:-NG] / U[0, NG:-NG, NG:-NG]
    frac = ke64 / U[3, NG:-NG, NG:-NG]
    assert frac.min() > 0.9996 and frac.max() < 0.99965  # 1 - 1 / (1 + gamma (gamma - 1) M^2 / 2) at M = 100


def test_recovered_step_and_dt_match_the_oracle_at_mach_100():
    pr, U = _stream()
    ref_in, ref, dt = _oracle_step(pr, U)
    got, dt_gpu, st = _gpu_step(pr, U, dt)
    assert st == 0
    mx, mean = _errors(got, ref, ref_in)
    assert np.all(mx[[0, 1, 3]] <= 0.1), mx
    assert np.all(mean[[0, 1, 3]] <= 0.06), mean
    assert mx[2] <= 0.4, mx
    assert abs(dt_gpu - dt) <= 5e-7 * dt, (dt_gpu, dt)


def test_without_recovery_the_same_step_is_worse():
    # the ablation: recover_ke_frac above 1 leaves E - rho |u|^2 / 2 to float arithmetic everywhere
    pr, U = _stream()
    ref_in, ref, dt = _oracle_step(pr, U)
    on, dt_on, _ = _gpu_step(pr, U, dt)
    off, dt_off, _ = _gpu_step(pr, U, dt, recover_ke_frac=2.0)
    mx_on, _ = _errors(on, ref, ref_in)
    mx_off, _ = _errors(off, ref, ref_in)
    assert np.all(mx_off[[0, 1, 3]] >= 0.3), mx_off
    assert np.all(mx_off[[0, 1, 3]] >= 10 * mx_on[[0, 1, 3]]), (mx_on, mx_off)
    assert abs(dt_off - dt) >= 100 * abs(dt_on - dt) and abs(dt_off - dt) >= 1e-5 * dt


def test_low_mach_flow_never_takes_the_branch():
    # Kelvin-Helmholtz (Mach ~0.4): the threshold never fires, so switching the recovery off changes nothing;
    # recovering every cell (recover_ke_frac = 0) stays within the FP32 step bound of the oracle
    pr = hp.kh(128, 96, seed=3)
    U = pr.U.astype(np.float32).astype(np.float64)
    ref_in, ref, dt = _oracle_step(pr, U)
    a, dta, _ = _gpu_step(pr, U, dt)
    b, dtb, _ = _gpu_step(pr, U, dt, recover_ke_frac=2.0)
    np.testing.assert_array_equal(a, b)
    assert dta == dtb
    c, dtc, st = _gpu_step(pr, U, dt, recover_ke_frac=0.0)
    scale = np.abs(ref).reshape(4, -1).max(1)
    assert st == 0 and np.all(np.abs(c - ref).reshape(4, -1).max(1) <= 2e-5 * scale)
    assert dtc == pytest.approx(dt, rel=1e-6)


def test_density_magnitude_alone_needs_no_recovery():
    # float keeps the same relative precision over its normal range, so a near-vacuum state is as accurate
    # as the same state at unit density: scaling rho, rho u, rho v and E by 2^-24 (velocities and sound speeds
    # unchanged, floors far below) scales the FP32 step's result by the same power of two.  The cancellation
    # the recovery removes depends on the ratio of kinetic to total energy only, which the scaling keeps.
    pr = hp.kh(96, 64, seed=7)
    U = pr.U.astype(np.float32).astype(np.float64)
    s = 2.0 ** -24
    ref_in, ref, dt = _oracle_step(pr, U)
    a, dta, _ = _gpu_step(pr, U, dt)
    b, dtb, st = _gpu_step(pr, U * s, dt)
    assert st == 0
    assert dtb == pytest.approx(dta, rel=1e-6)
    scale = np.abs(a).reshape(4, -1).max(1)
    assert np.all(np.abs(b / s - a).reshape(4, -1).max(1) <= 1e-6 * scale)
    # and the scaled run keeps the FP32 bound against the oracle's unscaled step
    assert np.all(np.abs(b / s - ref).reshape(4, -1).max(1) <= 2e-5 * np.abs(ref).reshape(4, -1).max(1))
