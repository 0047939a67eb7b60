"""Writes the golden fixtures of this folder from the oracle alone (no CUDA code is imported).

The paper prints no numbers for its test problems (its Sod result is a plot, §3.2.1), so these fixtures are
not the paper's values: they pin the oracle's own output on two of the paper's problems, bit for bit, so that
a later change to the oracle's arithmetic shows up as a failing test that names the fixture.  The Sod profile
is also checked against the exact Riemann solution by tests/test_oracle_step.py.

    python tests/golden/make_golden.py      # rewrites the .txt files next to this script
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import hydro_problems as hp  # noqa: E402
import oracle  # noqa: E402

NG = 4


def sod_case():
    """Sod shock tube along x (paper §3.2.1), 128 x 4 cells, to t = 0.2, FP64 oracle, default options."""
    pr = hp.sod(128, 4)
    p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl)
    U = pr.U.copy()
    t, n = oracle.advance(p, U, tmax=0.2)
    return pr, U, t, n


def kh_case():
    """Kelvin-Helmholtz layer (the KH workload's recipe, seed 0) on 16 x 16 cells, 20 steps, FP64 oracle."""
    pr = hp.kh(16, 16, seed=0)
    p = oracle.params(pr.nx, pr.ny, bc=pr.bc, gamma=pr.gamma, cfl=pr.cfl)
    U = pr.U.copy()
    t, n = oracle.advance(p, U, nsteps=20)
    return pr, U, t, n


def write(name, header, t, n, arrays):
    with open(os.path.join(HERE, name), "w") as f:
        f.write(header.rstrip() + "\n")
        f.write(f"# t = {t!r}, steps = {n}\n")
        for label, a in arrays:
            f.write(f"{label} " + " ".join(repr(float(x)) for x in np.ravel(a)) + "\n")


def main():
    pr, U, t, n = sod_case()
    row = U[:, NG, NG:-NG]
    write("sod_x_128_t0.2.txt",
          "# Sod shock tube (paper §3.2.1) along x, 128 x 4 cells, outflow / periodic, gamma 1.4, CFL 0.8, to t = 0.2;\n"
          "# FP64 oracle, 4th-order MC slopes, flattening, cvisc 0.1.  One row of the conserved fields (all rows are\n"
          "# equal).  Written by tests/golden/make_golden.py from the oracle only.",
          t, n, [("rho", row[0]), ("rhou", row[1]), ("rhov", row[2]), ("rhoE", row[3])])
    pr, U, t, n = kh_case()
    tot = oracle.conserved_totals(oracle.params(pr.nx, pr.ny, bc=pr.bc), U)
    write("kh_16_20steps.txt",
          "# Kelvin-Helmholtz shear layer (rho 2 / 1, u +-0.5, p 2.5, seeded v noise, seed 0), 16 x 16 cells, periodic,\n"
          "# 20 steps of the FP64 oracle driver loop; the interior conserved fields row by row, and the totals.\n"
          "# Written by tests/golden/make_golden.py from the oracle only.",
          t, n, [("rho", U[0, NG:-NG, NG:-NG]), ("rhou", U[1, NG:-NG, NG:-NG]), ("rhov", U[2, NG:-NG, NG:-NG]),
                 ("rhoE", U[3, NG:-NG, NG:-NG]), ("totals", tot)])


if __name__ == "__main__":
    main()
