"""The command-line driver (after the paper's ./pyro.py solver problem): one JSON line per run, for the
paper's step and for the variants, with the run reaching its end state and the counters filled in."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("args", [["sod", "--nx", "64", "--tmax", "0.05"],
                                  ["kh", "--nx", "96", "--precision", "fp32", "--steps", "20"],
                                  ["rt", "--nx", "32", "--steps", "12", "--riemann", "hllc", "--recon", "ppm"],
                                  ["sedov", "--nx", "64", "--precision", "fp32", "--steps", "10", "--split"],
                                  ["bubble", "--nx", "32", "--steps", "15", "--split"],
                                  ["kh", "--nx", "64", "--precision", "fp32", "--steps", "12", "--host"]])
def test_cli_runs_and_reports(args):
    r = subprocess.run([sys.executable, "-m", "paper_1306_6883_gb300", *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["status"] == "HYDRO_OK" and out["steps"] > 0 and out["riemann_solves"] > 0
    if "--tmax" in args:
        assert out["t"] == pytest.approx(float(args[args.index("--tmax") + 1]), rel=1e-12)
    else:
        assert out["steps"] == int(args[args.index("--steps") + 1])
    if "--riemann" in args:
        assert out["riemann"] == "hllc" and out["recon"] == "ppm" and out["riemann_iters"] == 0
    assert out["split"] == ("--split" in args)


def _run(args, tmp_path, name):
    dump = os.path.join(str(tmp_path), name + ".npy")
    r = subprocess.run([sys.executable, "-m", "paper_1306_6883_gb300", *args, "--dump", dump], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), dump


@pytest.mark.parametrize("args", [["sod", "--nx", "64", "--tmax", "0.05"], ["rt", "--nx", "32", "--steps", "30"]])
def test_host_resident_run_equals_the_device_run(args, tmp_path):
    # --host takes every step through hydro_step_host_chained: FP64, the same run bit for bit
    import numpy as np
    dev, fd = _run(args, tmp_path, "dev")
    host, fh = _run(args + ["--host"], tmp_path, "host")
    assert host["host"] and not dev["host"]
    assert host["t"] == dev["t"] and host["steps"] == dev["steps"] and host["totals"] == dev["totals"]
    np.testing.assert_array_equal(np.load(fh)[:, 4:-4, 4:-4], np.load(fd)[:, 4:-4, 4:-4])
