"""The allocation-free totals entry point, for callers that cannot allocate device memory (code running
while another allocator owns the device memory, or diagnostics after an out-of-memory error).

It must agree with hydro_conserved_totals, the allocating entry point, within the 1e-13 tolerance the
totals tests use, on two calls in a row (the second call reuses the shared file-scope scratch the first
one left behind).  This file is collected last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import hydro_problems as hp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6883_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def _noalloc(H, p, ptr, stream):
    out = (ctypes.c_double * 4)()
    st = H.load().hydro_conserved_totals_noalloc(ctypes.byref(p), ctypes.c_void_p(ptr), ctypes.c_void_p(stream), out)
    return st, np.array(out)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_totals_match_the_allocating_entry_point_twice(cuda, precision):
    from paper_1306_6883_gb300 import hydro as H
    from paper_1306_6883_gb300.solver import Solver, params_for

    # grids with fewer rows than the kernel's 304 blocks (one row per block), more rows (blocks take several
    # rows in turn), and the row limit itself on a narrow grid
    for pr in (hp.kh(300, 200, seed=4), hp.quad(77, 131, seed=2), hp.kh(64, 1000, seed=5),
               hp.quad(8, H.NOALLOC_MAX_ROWS, seed=6)):
        p = params_for(pr, precision)
        s = Solver(p, pr.U)
        s.advance(3)  # a state that is not the initial one
        ref = np.array(s.totals())
        scale = np.abs(s.interior().astype(np.float64)).sum(axis=(1, 2)) / (pr.nx * pr.ny)
        ptr = H.hydro_state(s.ctx)
        for call in range(2):
            st, got = _noalloc(H, p, ptr, s.stream.cuda_stream)
            assert st == H.HYDRO_OK
            assert np.all(np.abs(got - ref) <= 1e-13 * np.maximum(scale, 1e-300)), (call, got, ref)
        s.close()


def test_noalloc_rejects_grids_beyond_its_row_limit(cuda):
    from paper_1306_6883_gb300 import hydro as H

    p = H.default_params(8, H.NOALLOC_MAX_ROWS + 1)
    st, _ = _noalloc(H, p, 256, 0)
    assert st == H.HYDRO_ERANGE
    bad = H.default_params(0, 8)
    st, _ = _noalloc(H, bad, 256, 0)
    assert st == H.HYDRO_EINVAL
