"""Golden fixtures (tests/golden/, written by tests/golden/make_golden.py from the oracle alone): the oracle
must keep reproducing them bit for bit, and so must the FP64 GPU path, whose kernels round like the oracle."""
import os

import numpy as np
import pytest

import hydro_problems as hp
import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NG = 4


def _read(name):
    t = n = None
    fields = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            if line.startswith("# t = "):
                a, b = line[2:].split(",")
                t = float(a.split("=")[1])
                n = int(b.split("=")[1])
            elif not line.startswith("#"):
                label, *vals = line.split()
                fields[label] = np.array([float(v) for v in vals])
    return t, n, fields


def _oracle_sod():
    pr = hp.sod(128, 4)
    p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl)
    U = pr.U.copy()
    t, n = oracle.advance(p, U, tmax=0.2)
    return pr, U, t, n


def test_oracle_reproduces_the_sod_fixture():
    t0, n0, g = _read("sod_x_128_t0.2.txt")
    pr, U, t, n = _oracle_sod()
    assert (t, n) == (t0, n0)
    for k, name in enumerate(("rho", "rhou", "rhov", "rhoE")):
        np.testing.assert_array_equal(U[k, NG, NG:-NG], g[name], err_msg=name)


def test_oracle_reproduces_the_kh_fixture():
    t0, n0, g = _read("kh_16_20steps.txt")
    pr = hp.kh(16, 16, seed=0)
    p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl)
    U = pr.U.copy()
    t, n = oracle.advance(p, U, nsteps=20)
    assert (t, n) == (t0, n0)
    for k, name in enumerate(("rho", "rhou", "rhov", "rhoE")):
        np.testing.assert_array_equal(U[k, NG:-NG, NG:-NG].ravel(), g[name], err_msg=name)
    np.testing.assert_array_equal(oracle.conserved_totals(oracle.params(16, 16, bc=pr.bc), U), g["totals"])


@pytest.mark.gpu
def test_fp64_gpu_runs_reproduce_the_fixtures():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_6883_gb300 import build
    build.build()
    from paper_1306_6883_gb300.solver import Solver, params_for
    t0, n0, g = _read("sod_x_128_t0.2.txt")
    pr = hp.sod(128, 4)
    s = Solver(params_for(pr), pr.U)
    s.advance(n0, 0.2)
    t, n = s.time()
    U = s.state_numpy()
    s.close()
    assert (t, n) == (t0, n0)
    for k, name in enumerate(("rho", "rhou", "rhov", "rhoE")):
        np.testing.assert_array_equal(U[k, NG, NG:-NG], g[name], err_msg=name)
    t0, n0, g = _read("kh_16_20steps.txt")
    pr = hp.kh(16, 16, seed=0)
    s = Solver(params_for(pr), pr.U)
    s.advance(20)
    t, n = s.time()
    U = s.state_numpy()
    tot = np.array(s.totals())
    s.close()
    assert (t, n) == (t0, n0)
    for k, name in enumerate(("rho", "rhou", "rhov", "rhoE")):
        np.testing.assert_array_equal(U[k, NG:-NG, NG:-NG].ravel(), g[name], err_msg=name)
    np.testing.assert_allclose(tot, g["totals"], rtol=1e-13, atol=1e-13)
