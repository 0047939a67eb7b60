"""The pins catch plausible mistakes: each case plants one mistake in a copy of the oracle's C source (on the
CPU, in a temporary directory), rebuilds it and runs the pin suite against it, which must fail."""
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "transverse correction dropped": [
        ("UL[k] = UL[k] - hy * (AT(fyh, k, j + 1, f - 1) - AT(fyh, k, j, f - 1));\n"
         "        UR[k] = UR[k] - hy * (AT(fyh, k, j + 1, f) - AT(fyh, k, j, f));", "UL[k] = UL[k]; UR[k] = UR[k];"),
        ("UL[k] = UL[k] - hx * (AT(fxh, k, gg - 1, i + 1) - AT(fxh, k, gg - 1, i));\n"
         "        UR[k] = UR[k] - hx * (AT(fxh, k, gg, i + 1) - AT(fxh, k, gg, i));", "UL[k] = UL[k]; UR[k] = UR[k];")],
    "transverse factor 1 instead of 1/2": [
        ("const double hx = 0.5 * dt / dx, hy = 0.5 * dt / dy;", "const double hx = dt / dx, hy = dt / dy;")],
    "tracing reference speed": [
        ("double sl = q[m] + 0.5 * (1.0 - sigma * lam[3]) * dq[m];", "double sl = q[m] + 0.5 * (1.0 - sigma * lam[0]) * dq[m];")],
    "left eigenvector sign": [
        ("{{0.0, -0.5 * rho / c, 0.0, 0.5 / (c * c)},", "{{0.0, 0.5 * rho / c, 0.0, 0.5 / (c * c)},")],
    "fourth-order slope constant": [("double d4 = (4.0 / 3.0) * dc", "double d4 = (1.0) * dc")],
    "flattening compression test": [("int compress = (um1 - up1) > 0.0;", "int compress = (um1 - up1) < 0.0;")],
    "flattening takes the higher-pressure neighbour in x": [
        ("chix[(size_t)j * NX + i - sx]", "chix[(size_t)j * NX + i + sx]")],
    "flattening takes the higher-pressure neighbour in y": [
        ("chiy[(size_t)(j - sy) * NX + i]", "chiy[(size_t)(j + sy) * NX + i]")],
    "flattening directions combined by max": [("AT(xi, 0, j, i) = fmin(xix, xiy);", "AT(xi, 0, j, i) = fmax(xix, xiy);")],
    "flattening ramp start": [("const double z0 = 0.75, z1 = 0.85, delta = 0.33;",
                               "const double z0 = 0.7, z1 = 0.85, delta = 0.33;")],
    "flattening ramp end": [("const double z0 = 0.75, z1 = 0.85, delta = 0.33;",
                             "const double z0 = 0.75, z1 = 0.9, delta = 0.33;")],
    "flattening jump threshold": [("const double z0 = 0.75, z1 = 0.85, delta = 0.33;",
                                   "const double z0 = 0.75, z1 = 0.85, delta = 0.4;")],
    "shock mass flux": [("const double g1 = (g + 1.0) / (2.0 * g);", "const double g1 = (g + 1.0) / (2.0);")],
    "star density sign": [("double rst = 1.0 / (1.0 / ro - (pst - po) / (wo * wo));",
                           "double rst = 1.0 / (1.0 / ro + (pst - po) / (wo * wo));")],
    "energy flux": [("F[3] = un * (rhoE + pres);", "F[3] = un * (rhoE);")],
    "gravity energy source not time-centred": [
        ("AT(U, 3, j, i) = AT(U, 3, j, i) + hdtg * (my_n + AT(U, 2, j, i));",
         "AT(U, 3, j, i) = AT(U, 3, j, i) + hdtg * (2.0 * my_n);")],
    "gravity half-step of the y states dropped": [
        ("        ql[1] = ql[1] + hdtg;\n        qr[1] = qr[1] + hdtg;", "")],
    "reflecting wall keeps the normal momentum": [
        ("const double flip = (k == IMX) ? -1.0 : 1.0;", "const double flip = 1.0;")],
    "hydrostatic ghost pressure sign": [
        ("const double pg = pe + rho * p->grav * ((double)(j - edge) * dy);",
         "const double pg = pe - rho * p->grav * ((double)(j - edge) * dy);")],
    "artificial viscosity strength": [
        ("double av = p->cvisc * fmax(-div * dx, 0.0);", "double av = 10 * p->cvisc * fmax(-div * dx, 0.0);"),
        ("double av = p->cvisc * fmax(-div * dy, 0.0);", "double av = 10 * p->cvisc * fmax(-div * dy, 0.0);")],
    "split: viscosity from the transverse velocity": [
        ("double div = (q[1 * N + f] - q[1 * N + f - 1]) / h;", "double div = (q[2 * N + f] - q[2 * N + f - 1]) / h;")],
    "split: y sweep keeps the x components": [
        ("const int kn = dir == 0 ? 1 : 2, kt = dir == 0 ? 2 : 1;", "const int kn = 1, kt = 2;")],
    "split: both sweeps use the x spacing": [
        ("const double h = dir == 0 ? (p->xmax - p->xmin) / nx : (p->ymax - p->ymin) / ny;",
         "const double h = (p->xmax - p->xmin) / nx;")],
    "split: no ghost fill between the sweeps": [
        ("  if (!err) err = oracle_fill_ghost(p, U);\n  if (!err) err = sweep", "  if (!err) err = sweep")],
    "hllc: star energy term": [
        ("f * (El / rl + (sst - ul) * (sst + pl / (rl * (SL - ul))))",
         "f * (El / rl + (sst - ul) * (sst - pl / (rl * (SL - ul))))")],
    "hllc: contact speed with the pressure jump reversed": [
        ("double sst = (pr - pl + rl * ul", "double sst = (pl - pr + rl * ul")],
    "hllc: left speed from the left state only": [
        ("double SL = fmin(qL[1] - cl, qR[1] - cr);", "double SL = qL[1] - cl;")],
    "ppm: interface correction sign": [
        ("double r = a[2] + 0.5 * (a[3] - a[2]) - (dp - d0) / 6.0;",
         "double r = a[2] + 0.5 * (a[3] - a[2]) + (dp - d0) / 6.0;")],
    "ppm: overshoot moved to the wrong edge": [("      l = 3.0 * c - 2.0 * r;", "      r = 3.0 * c - 2.0 * l;")],
    "ppm: curvature term of the right-edge average": [
        ("double ip = aR[m] - 0.5 * sn * (da[m] - (1.0 - (2.0 / 3.0) * sn) * a6[m]);",
         "double ip = aR[m] - 0.5 * sn * (da[m] + (1.0 - (2.0 / 3.0) * sn) * a6[m]);")],
    "ppm: reference state from the slowest wave": [
        ("double s4 = sigma * lam[3] > 0.0 ? sigma * lam[3] : 0.0;",
         "double s4 = sigma * lam[1] > 0.0 ? sigma * lam[1] : 0.0;")],
    "split: gravity sources in both sweeps": [
        ("      if (dir == 1 && p->grav != 0.0) {\n        C(2, m)", "      if (p->grav != 0.0) {\n        C(2, m)")],
    "split: flux difference reversed": [
        ("C(k, m) = C(k, m) + sigma * (G[k * (N + 1) + m] - G[k * (N + 1) + m + 1]);",
         "C(k, m) = C(k, m) + sigma * (G[k * (N + 1) + m + 1] - G[k * (N + 1) + m]);")],
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_pins_catch_the_planted_mistake(name):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        for sub in ("oracle", "tests", "hydro_problems"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                            ignore=shutil.ignore_patterns("*.so", "__pycache__", "test_oracle_mutations.py"))
        shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
        path = os.path.join(d, "oracle", "oracle.c")
        src = open(path).read()
        for a, b in MUTATIONS[name]:
            assert src.count(a) == 1, a
            src = src.replace(a, b)
        open(path, "w").write(src)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                            "tests/test_oracle_riemann.py", "tests/test_oracle_stages.py", "tests/test_oracle_flattening.py",
                            "tests/test_oracle_step.py",
                            "tests/test_oracle_gravity.py", "tests/test_oracle_split.py",
                            "tests/test_oracle_hllc.py", "tests/test_oracle_ppm.py"],
                           cwd=d, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"mistake '{name}' was not caught:\n{r.stdout[-2000:]}"
        assert "FAILED" in r.stdout
    finally:
        shutil.rmtree(d, ignore_errors=True)
