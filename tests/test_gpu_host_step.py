"""hydro_step_host (upload in chunks per band of tile rows, fused step in concurrent bands, each band's rows
downloaded while later bands compute) gives exactly the interior that hydro_upload + hydro_step_fused +
hydro_download give, step after step, in both precisions, for ragged grids (whose unpadded rows are not
16-byte multiples: the staging copy is then read cell by cell), general boundaries with gravity, a tmax clamp
and the split variant (which runs the three calls in turn); 16 tile rows or more (KH 1024^2 has 64, RT 64x400 has 25) take
the eight-band schedule of the chained step.  hydro_step_host_chained, which reuses the time
step the previous host step reduced and overlaps the upload with the step, gives the same results; its chain
breaks (the time step is reduced again) when the input is another buffer, when another call stepped the
state in between, or when tmax changes."""
import numpy as np
import pytest

import hydro_problems as hp

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


PROBLEMS = {"kh_100x70": lambda: hp.kh(100, 70, seed=1), "kh_1024": lambda: hp.kh(1024, 1024, seed=0),
            "rt_40x150": lambda: hp.rt(40, 150), "quad_33x5": lambda: hp.quad(33, 5, seed=2),
            "kh_64_split": lambda: hp.kh(64, 64, seed=4), "sedov_96_tmax": lambda: hp.sedov(96, 96, r_init=0.05),
            "bubble_37x75": lambda: hp.bubble(37, 75), "quad_1x1": lambda: hp.quad(1, 1, seed=3),
            "rt_64x400": lambda: hp.rt(64, 400)}
CASES = [("kh_100x70", {}), ("kh_1024", {}), ("rt_40x150", {}), ("quad_33x5", {}), ("kh_64_split", {"split": 1}),
         ("sedov_96_tmax", {}), ("bubble_37x75", {}), ("quad_1x1", {}), ("rt_64x400", {})]


def _interior(x):
    return x[:, NG:-NG, NG:-NG]


def _pinned_pair(pr, precision):
    import torch
    dt = torch.float32 if precision else torch.float64
    return [torch.from_numpy(np.ascontiguousarray(pr.U)).to(dt).pin_memory() for _ in range(2)]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,kw", CASES)
def test_host_steps_equal_upload_step_download(precision, name, kw):
    import torch
    from paper_1306_6883_gb300.solver import Solver, params_for
    pr = PROBLEMS[name]()
    tmax = 2e-4 if name == "sedov_96_tmax" else 0.0
    a = Solver(params_for(pr, precision, **kw), pr.U)
    c = Solver(params_for(pr, precision, **kw), pr.U)
    b = Solver(params_for(pr, precision, **kw), pr.U)
    ha, hc, hb = _pinned_pair(pr, precision), _pinned_pair(pr, precision), _pinned_pair(pr, precision)
    for k in range(5):
        a.step_host(ha[k % 2], ha[(k + 1) % 2], tmax)
        c.step_host(hc[k % 2], hc[(k + 1) % 2], tmax, chained=True)
        b.upload(hb[k % 2])
        b.step_fused(tmax)
        b.download(hb[(k + 1) % 2])
        ref = _interior(hb[(k + 1) % 2])
        torch.testing.assert_close(_interior(ha[(k + 1) % 2]), ref, rtol=0, atol=0)
        torch.testing.assert_close(_interior(hc[(k + 1) % 2]), ref, rtol=0, atol=0)
    # the context's current buffer holds the new state as well
    torch.testing.assert_close(_interior(torch.from_numpy(a.state_numpy())), _interior(hb[1]).cpu(), rtol=0, atol=0)
    torch.testing.assert_close(_interior(torch.from_numpy(c.state_numpy())), _interior(hb[1]).cpu(), rtol=0, atol=0)
    assert a.time() == b.time() == c.time()
    for s in (a, c):
        st, _ = s.status()
        assert st == 0
    if tmax > 0:
        assert a.time()[0] == pytest.approx(tmax, rel=1e-12)
    for s in (a, b, c):
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_the_chain_breaks_when_the_state_changes_under_it(precision):
    # each break must reduce the time step of host_in again: the result then equals the three calls from it
    import torch
    from paper_1306_6883_gb300.solver import Solver, params_for
    pr = hp.kh(96, 80, seed=6)
    c = Solver(params_for(pr, precision), pr.U)
    b = Solver(params_for(pr, precision), pr.U)
    h = _pinned_pair(pr, precision)
    other = h[0].clone().pin_memory()
    out = h[1].clone().pin_memory()

    def reference(src):
        b.upload(src)
        b.step_fused()
        b.download(out)
        return _interior(out).clone()

    c.step_host(h[0], h[1], chained=True)
    ref = reference(h[0])
    torch.testing.assert_close(_interior(h[1]), ref, rtol=0, atol=0)
    # another input buffer (here the initial state again, whose time step differs from the last output's)
    c.step_host(other, h[0], chained=True)
    torch.testing.assert_close(_interior(h[0]), reference(other), rtol=0, atol=0)
    # a device step in between: the host buffer no longer holds the context's state
    c.step_fused()
    c.step_host(h[0], h[1], chained=True)
    torch.testing.assert_close(_interior(h[1]), reference(h[0]), rtol=0, atol=0)
    # another tmax, one that clamps this step: the step's length is then tmax - t, not the carried time step
    t = c.time()[0]
    tmax = t + 1e-5
    c.step_host(h[1], h[0], tmax=tmax, chained=True)
    assert c.time()[0] == pytest.approx(tmax, rel=1e-13, abs=0)
    st, _ = c.status()
    assert st == 0
    c.close()
    b.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_pageable_host_buffers_give_the_same_steps(precision):
    # host memory that is not pinned takes the copies as they come (no captured graph); same results
    import torch
    from paper_1306_6883_gb300.solver import Solver, params_for
    pr = hp.kh(128, 96, seed=8)
    a = Solver(params_for(pr, precision), pr.U)
    b = Solver(params_for(pr, precision), pr.U)
    hp_ = _pinned_pair(pr, precision)
    hq = [x.clone() for x in hp_]
    assert not hq[0].is_pinned()
    for k in range(4):
        a.step_host(hp_[k % 2], hp_[(k + 1) % 2], chained=True)
        b.step_host(hq[k % 2], hq[(k + 1) % 2], chained=True)
        torch.testing.assert_close(_interior(hq[(k + 1) % 2]), _interior(hp_[(k + 1) % 2]), rtol=0, atol=0)
    assert a.time() == b.time()
    for s in (a, b):
        st, _ = s.status()
        assert st == 0
        s.close()
