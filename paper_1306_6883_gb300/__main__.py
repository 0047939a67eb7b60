"""Command-line driver, after the paper's single driver (§2: ./pyro.py solver problem infile):

    python -m paper_1306_6883_gb300 PROBLEM [--nx N] [--ny N] [--precision fp32|fp64]
                                            [--steps K | --tmax T] [--seed S] [--split]
                                            [--riemann two-shock|hllc] [--recon plm|ppm] [--host]
                                            [--dump FILE]

PROBLEM is one of sod, sod_y, kh, sedov, quad, pulse, rt, bubble (seeded set-ups of hydro_problems; rt is
the Rayleigh-Taylor column with gravity, nx x 3nx by default; bubble a buoyant bubble in a stratified
atmosphere, nx x 2nx by default).  Runs the device-resident loop (fill ghost
cells, CFL dt, CTU step; --split: the dimensionally split step; --riemann and --recon choose the Riemann
solver and the reconstruction; --host keeps the state in pinned host memory and takes every step through
hydro_step_host_chained, the whole state going up and down each step) and prints one JSON line with the simulated
time, step count, wall time, conserved totals and the Riemann-solver counters.  --dump writes the final
state (dense float64 array, shape (4, ny+8, nx+8)) with numpy.save.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make_problem(name, nx, ny, seed):
    import hydro_problems as hp
    if name == "sod":
        return hp.sod(nx, ny)
    if name == "sod_y":
        return hp.sod(nx, ny, direction="y")
    if name == "kh":
        return hp.kh(nx, ny, seed=seed)
    if name == "sedov":
        return hp.sedov(nx, ny, seed=seed)
    if name == "quad":
        return hp.quad(nx, ny, seed=seed)
    if name == "pulse":
        return hp.pulse(nx, ny)
    if name == "rt":
        return hp.rt(nx, ny)
    if name == "bubble":
        return hp.bubble(nx, ny)
    raise SystemExit(f"unknown problem {name}")


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1306_6883_gb300")
    ap.add_argument("problem")
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp64")
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--tmax", type=float, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--split", action="store_true")
    ap.add_argument("--riemann", choices=["two-shock", "hllc"], default="two-shock")
    ap.add_argument("--recon", choices=["plm", "ppm"], default="plm")
    ap.add_argument("--host", action="store_true")
    ap.add_argument("--dump", default=None)
    a = ap.parse_args(argv)

    import torch

    from . import build
    from . import hydro as H
    from .solver import Solver, params_for

    build.build()
    ny = a.ny or (3 * a.nx if a.problem == "rt" else 2 * a.nx if a.problem == "bubble" else a.nx)
    pr = make_problem(a.problem, a.nx, ny, a.seed)
    prec = H.HYDRO_FP32 if a.precision == "fp32" else H.HYDRO_FP64
    s = Solver(params_for(pr, prec, split=int(a.split), riemann_solver=a.riemann, reconstruction=a.recon), pr.U)
    tmax = a.tmax if a.tmax is not None else (pr.tmax if np.isfinite(pr.tmax) and a.steps is None else 0.0)
    steps = a.steps if a.steps is not None else 10 ** 9
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    chunk = 64
    done = 0
    if a.host:  # the run lives in two pinned host buffers, each step's output the next step's input
        dt_ = torch.float32 if prec == H.HYDRO_FP32 else torch.float64
        host = [torch.from_numpy(np.ascontiguousarray(pr.U)).to(dt_).pin_memory() for _ in range(2)]
    while done < steps:
        n = min(chunk, steps - done)
        if a.host:
            for k in range(done, done + n):
                s.step_host(host[k % 2], host[(k + 1) % 2], tmax, chained=True)
        else:
            s.advance(n, tmax)
        done += n
        if tmax > 0.0:
            t, _ = s.time()
            if t >= tmax:
                break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st, stats = s.status(raise_on_error=False)
    t, nsteps = s.time()
    out = {"problem": a.problem, "nx": pr.nx, "ny": pr.ny, "precision": a.precision, "split": a.split, "riemann": a.riemann,
           "recon": a.recon, "host": a.host, "t": t,
           "steps": nsteps,
           "wall_s": wall, "zone_updates_per_s": pr.nx * pr.ny * nsteps / wall if wall > 0 else None,
           "totals": s.totals(), "status": H.STATUS_NAMES[st], "riemann_solves": stats[0],
           "riemann_iters": stats[1], "riemann_nonconverged": stats[2]}
    if a.dump:
        np.save(a.dump, s.state_numpy().astype(np.float64))
    s.close()
    print(json.dumps(out))
    return 0 if st == H.HYDRO_OK else 1


if __name__ == "__main__":
    sys.exit(main())
