"""hydro_step_host (upload, fused step in concurrent bands of tile rows, each band's rows downloaded while
later bands compute) gives exactly what hydro_upload + hydro_step_fused + hydro_download give, step after
step, in both precisions, for ragged grids, general boundaries with gravity, a tmax clamp and the split
variant (which runs the three calls in turn)."""
import numpy as np
import pytest

import hydro_problems as hp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6883_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,kw", [("kh_100x70", {}), ("kh_1024", {}), ("rt_40x150", {}), ("quad_33x5", {}),
                                     ("kh_64_split", {"split": 1}), ("sedov_96_tmax", {})])
def test_host_step_equals_upload_step_download(precision, name, kw):
    import torch
    from paper_1306_6883_gb300.solver import Solver, params_for
    pr = {"kh_100x70": lambda: hp.kh(100, 70, seed=1), "kh_1024": lambda: hp.kh(1024, 1024, seed=0),
          "rt_40x150": lambda: hp.rt(40, 150), "quad_33x5": lambda: hp.quad(33, 5, seed=2),
          "kh_64_split": lambda: hp.kh(64, 64, seed=4), "sedov_96_tmax": lambda: hp.sedov(96, 96, r_init=0.05)}[name]()
    tmax = 2e-4 if name == "sedov_96_tmax" else 0.0
    dt = torch.float32 if precision else torch.float64
    a = Solver(params_for(pr, precision, **kw), pr.U)
    b = Solver(params_for(pr, precision, **kw), pr.U)
    ha = [torch.from_numpy(np.ascontiguousarray(pr.U)).to(dt).pin_memory() for _ in range(2)]
    hb = [x.clone().pin_memory() for x in ha]
    for k in range(4):
        a.step_host(ha[k % 2], ha[(k + 1) % 2], tmax)
        b.upload(hb[k % 2])
        b.step_fused(tmax)
        b.download(hb[(k + 1) % 2])
        torch.testing.assert_close(ha[(k + 1) % 2], hb[(k + 1) % 2], rtol=0, atol=0)
    assert a.time() == b.time()
    st, _ = a.status()
    assert st == 0
    if tmax > 0:
        assert a.time()[0] == pytest.approx(tmax, rel=1e-12)
    a.close()
    b.close()
