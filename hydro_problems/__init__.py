"""Seeded synthetic initial conditions shared by the oracle side and the CUDA side.

This module builds problem set-ups only (paper §2 "problems/": initial conditions plus default
parameters; Table 1).  It holds none of the CTU method's arithmetic: no slopes, tracing, Riemann
solves or updates.  Each generator returns a ``Problem``: conserved state U of shape
(4, ny + 2 ng, nx + 2 ng) float64 with the interior set and ghost cells zero, plus the boundary
conditions, domain, gamma, CFL and end time.  Random draws use numpy's PCG64 generator with a fixed
seed, drawn per cell in row-major order (row j outer, column i inner).
"""
from dataclasses import dataclass, field

import numpy as np

NG = 4


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    U: np.ndarray                    # (4, ny+2ng, nx+2ng) float64, interior set, ghosts zero
    bc: tuple                        # (xlo, xhi, ylo, yhi): "outflow", "periodic", "reflect" or
                                     # "hydrostatic" (y sides)
    gamma: float = 1.4
    cfl: float = 0.8
    tmax: float = 0.2
    domain: tuple = (0.0, 1.0, 0.0, 1.0)
    ng: int = NG
    extra: dict = field(default_factory=dict)
    grav: float = 0.0                # constant gravitational acceleration along y


def _centres(nx, ny, domain=(0.0, 1.0, 0.0, 1.0)):
    xmin, xmax, ymin, ymax = domain
    dx, dy = (xmax - xmin) / nx, (ymax - ymin) / ny
    x = xmin + (np.arange(nx) + 0.5) * dx
    y = ymin + (np.arange(ny) + 0.5) * dy
    return np.meshgrid(x, y, indexing="xy")  # arrays of shape (ny, nx)


def _pack(rho, u, v, p, gamma, ng=NG):
    """Conserved state from primitive initial data: rho E = p/(gamma-1) + rho |U|^2 / 2 (Eqs. 11-12)."""
    ny, nx = rho.shape
    U = np.zeros((4, ny + 2 * ng, nx + 2 * ng))
    s = (slice(ng, ng + ny), slice(ng, ng + nx))
    U[0][s] = rho
    U[1][s] = rho * u
    U[2][s] = rho * v
    U[3][s] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return U


def sod(nx=128, ny=128, direction="x", gamma=1.4):
    """Sod shock tube (paper §3.2.1): rho, p = (1, 1) left of the mid-plane, (0.125, 0.1) right, at rest.
    Outflow along the tube, periodic across it."""
    X, Y = _centres(nx, ny)
    s = X if direction == "x" else Y
    left = s < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    z = np.zeros_like(rho)
    bc = ("outflow", "outflow", "periodic", "periodic") if direction == "x" else \
        ("periodic", "periodic", "outflow", "outflow")
    return Problem("sod_" + direction, nx, ny, _pack(rho, z, z, p, gamma), bc, gamma=gamma, cfl=0.8, tmax=0.2)


def rt(nx=128, ny=384, rho1=1.0, rho2=2.0, grav=-1.0, p0=5.0, amp=0.01, sigma=0.1, gamma=1.4, lx=1.0, ly=3.0):
    """Single-mode Rayleigh-Taylor instability (paper §3.2, Rayleigh-Taylor set-up and Fig. 4): rho = rho1
    below y_c = ly/2 and rho2 above (2:1 ratio); pressure in hydrostatic equilibrium for constant g,
    p = p0 + rho1 g y below y_c, p0 + rho1 g y_c + rho2 g (y - y_c) above (evaluated at cell centres);
    v = amp cos(2 pi x / lx) exp(-(y - y_c)^2 / sigma^2), u = 0.  Periodic in x, hydrostatic boundaries
    in y, gravity along -y.  The paper ran 128 x 384 zones at CFL 0.8; it does not state p0, amp, sigma or
    the domain, which are this generator's choices (p0 keeps the pressure positive over the column)."""
    domain = (0.0, lx, 0.0, ly)
    X, Y = _centres(nx, ny, domain)
    yc = 0.5 * ly
    below = Y < yc
    rho = np.where(below, rho1, rho2)
    p = np.where(below, p0 + rho1 * grav * Y, p0 + rho1 * grav * yc + rho2 * grav * (Y - yc))
    v = amp * np.cos(2.0 * np.pi * X / lx) * np.exp(-((Y - yc) ** 2) / sigma ** 2)
    u = np.zeros_like(rho)
    return Problem("rt", nx, ny, _pack(rho, u, v, p, gamma), ("periodic", "periodic", "hydrostatic", "hydrostatic"),
                   gamma=gamma, cfl=0.8, tmax=3.0, domain=domain, grav=grav)


def bubble(nx=128, ny=256, grav=-1.0, rho0=1.0, H=1.0, amp=2.0, radius=0.1, yc=0.5, gamma=1.4, lx=1.0, ly=2.0):
    """Buoyant bubble in a stratified atmosphere (the paper's Table 1 `bubble` problem; it gives no set-up,
    so this one is the generator's choice): an isothermal atmosphere in hydrostatic equilibrium,
    rho_atm = rho0 exp(-y / H), p = rho_atm |g| H (so dp/dy = rho g), with a hot, light bubble at
    (lx / 2, yc): rho = rho_atm / (1 + amp exp(-r^2 / radius^2)) at the same pressure; at rest.  Reflecting
    walls in x, hydrostatic boundaries in y, gravity along -y."""
    domain = (0.0, lx, 0.0, ly)
    X, Y = _centres(nx, ny, domain)
    rho_atm = rho0 * np.exp(-Y / H)
    p = rho_atm * abs(grav) * H
    r2 = (X - 0.5 * lx) ** 2 + (Y - yc) ** 2
    rho = rho_atm / (1.0 + amp * np.exp(-r2 / radius ** 2))
    z = np.zeros_like(rho)
    return Problem("bubble", nx, ny, _pack(rho, z, z, p, gamma), ("reflect", "reflect", "hydrostatic", "hydrostatic"),
                   gamma=gamma, cfl=0.8, tmax=3.0, domain=domain, grav=grav)


def kh(nx=1024, ny=1024, seed=0, gamma=1.4):
    """Kelvin-Helmholtz shear layer (Table 1 "kh"): rho = 2, u = +0.5 for |y - 0.5| < 0.25, else rho = 1,
    u = -0.5; p = 2.5; v = 0.01 sin(4 pi x) * w with w ~ U[-1, 1] per cell (seeded).  Periodic."""
    X, Y = _centres(nx, ny)
    inner = np.abs(Y - 0.5) < 0.25
    rho = np.where(inner, 2.0, 1.0)
    u = np.where(inner, 0.5, -0.5)
    w = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(ny, nx))
    v = 0.01 * np.sin(4.0 * np.pi * X) * w
    p = np.full_like(rho, 2.5)
    return Problem("kh", nx, ny, _pack(rho, u, v, p, gamma), ("periodic",) * 4, gamma=gamma, tmax=np.inf,
                   extra={"steps": 200, "seed": seed})


def sedov(nx=4096, ny=4096, E=1.0, r_init=0.01, gamma=1.4, rho_amb=1.0, p_amb=1e-5, density_noise=0.0, seed=0):
    """Sedov-Taylor blast (paper §3.2.2, Eq. 14): pressure (gamma-1) E / (pi r_init^2) inside r_init of the
    centre, averaged over 4x4 sub-zones per cell; ambient rho_amb, p_amb, at rest; outflow.
    Optional seeded density noise rho_amb (1 + density_noise * U[-1, 1])."""
    xmin, xmax, ymin, ymax = 0.0, 1.0, 0.0, 1.0
    dx, dy = (xmax - xmin) / nx, (ymax - ymin) / ny
    xc, yc = 0.5 * (xmin + xmax), 0.5 * (ymin + ymax)
    p_in = (gamma - 1.0) * E / (np.pi * r_init * r_init)
    # only cells near the centre can contain sub-zones inside r_init
    n_in = np.zeros((ny, nx), dtype=np.int64)
    i0 = max(int((xc - r_init - xmin) / dx) - 2, 0)
    i1 = min(int((xc + r_init - xmin) / dx) + 3, nx)
    j0 = max(int((yc - r_init - ymin) / dy) - 2, 0)
    j1 = min(int((yc + r_init - ymin) / dy) + 3, ny)
    sub = (np.arange(4) + 0.5) / 4.0
    for a in sub:
        for b in sub:
            xs = xmin + (np.arange(i0, i1) + a) * dx
            ys = ymin + (np.arange(j0, j1) + b) * dy
            XS, YS = np.meshgrid(xs, ys, indexing="xy")
            n_in[j0:j1, i0:i1] += ((XS - xc) ** 2 + (YS - yc) ** 2 <= r_init * r_init)
    p = (n_in * p_in + (16 - n_in) * p_amb) / 16.0
    rho = np.full((ny, nx), rho_amb)
    if density_noise > 0.0:
        rho = rho_amb * (1.0 + density_noise * np.random.default_rng(seed).uniform(-1.0, 1.0, size=(ny, nx)))
    z = np.zeros_like(rho)
    return Problem("sedov", nx, ny, _pack(rho, z, z, p, gamma), ("outflow",) * 4, gamma=gamma, tmax=0.1,
                   extra={"E": E, "r_init": r_init, "n_subzones_inside": int(n_in.sum()), "seed": seed,
                          "density_noise": density_noise})


def quad(nx=256, ny=256, rng=None, seed=0, gamma=1.4):
    """Four-quadrant 2-D Riemann problem (Table 1 "quad"): quadrants split at (0.5, 0.5), each with
    rho ~ logU[0.1, 1], p ~ logU[0.01, 10], u, v ~ U[-1, 1] (drawn in quadrant order
    lower-left, lower-right, upper-left, upper-right); outflow on all sides."""
    g = rng if rng is not None else np.random.default_rng(seed)
    st = []
    for _ in range(4):
        rho = float(np.exp(g.uniform(np.log(0.1), np.log(1.0))))
        p = float(np.exp(g.uniform(np.log(0.01), np.log(10.0))))
        u = float(g.uniform(-1.0, 1.0))
        v = float(g.uniform(-1.0, 1.0))
        st.append((rho, u, v, p))
    X, Y = _centres(nx, ny)
    quadrant = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)
    fields = [np.choose(quadrant, [s[k] for s in st]).astype(np.float64) for k in range(4)]
    return Problem("quad", nx, ny, _pack(fields[0], fields[1], fields[2], fields[3], gamma), ("outflow",) * 4,
                   gamma=gamma, tmax=np.inf, extra={"states": st})


def pulse(nx=64, ny=64, A=60.0, u0=1.0, v0=1.0, p0=1.0, gamma=1.4):
    """Advected smooth density pulse (paper §3.1.1, Eq. 7): rho = 1 + exp(-A r^2) about the domain centre,
    uniform velocity (u0, v0) and pressure p0; periodic.  The exact solution at time t is the initial
    profile translated by (u0 t, v0 t)."""
    X, Y = _centres(nx, ny)
    rho = 1.0 + np.exp(-A * ((X - 0.5) ** 2 + (Y - 0.5) ** 2))
    u = np.full_like(rho, u0)
    v = np.full_like(rho, v0)
    p = np.full_like(rho, p0)
    return Problem("pulse", nx, ny, _pack(rho, u, v, p, gamma), ("periodic",) * 4, gamma=gamma, tmax=1.0,
                   extra={"A": A, "u0": u0, "v0": v0})


def stream(nx=256, ny=256, mach=100.0, angle=0.0, rho0=1.0, p0=1.0, density_noise=0.01, seed=0, gamma=1.4,
           domain=(0.0, 1.0, 0.0, 1.0), collide=False):
    """Hypersonic stream, the regime where E - rho |u|^2 / 2 cancels (not one of the paper's problems, which
    run at low Mach): speed mach * c0 (c0 = sqrt(gamma p0 / rho0)) at `angle` radians to x, uniform
    pressure p0, density rho0 (1 + density_noise U[-1, 1]) per cell (seeded, row-major); periodic.  Kinetic
    over total energy 1 - 1 / (1 + gamma (gamma - 1) mach^2 / 2) (0.99964 at Mach 100, gamma 1.4).
    collide: the stream runs along +x in the left half and along -x in the right half (two strong shocks
    form at x = 1/2), outflow in x."""
    X, Y = _centres(nx, ny, domain)
    c0 = np.sqrt(gamma * p0 / rho0)
    rho = np.full((ny, nx), rho0)
    if density_noise > 0.0:
        rho = rho0 * (1.0 + density_noise * np.random.default_rng(seed).uniform(-1.0, 1.0, size=(ny, nx)))
    sgn = np.where(X < 0.5 * (domain[0] + domain[1]), 1.0, -1.0) if collide else np.ones((ny, nx))
    u = sgn * mach * c0 * np.cos(angle)
    v = sgn * mach * c0 * np.sin(angle)
    p = np.full((ny, nx), p0)
    bc = ("outflow", "outflow", "periodic", "periodic") if collide else ("periodic",) * 4
    return Problem("stream", nx, ny, _pack(rho, u, v, p, gamma), bc, gamma=gamma, tmax=np.inf, domain=domain,
                   extra={"mach": mach, "angle": angle, "seed": seed, "density_noise": density_noise,
                          "collide": collide})


def ensemble_sizes(n=256, seed=0, choices=(64, 128, 256, 512)):
    """Grid sizes of an ensemble of independent problems: n square sizes drawn uniformly from choices."""
    g = np.random.default_rng(seed)
    return [int(choices[k]) for k in g.integers(0, len(choices), size=n)]


def ensemble(n=256, seed=0, choices=(64, 128, 256, 512)):
    """Ensemble of n independent four-quadrant problems on uneven square grids (seeded)."""
    sizes = ensemble_sizes(n, seed, choices)
    g = np.random.default_rng(seed + 1)
    return [quad(s, s, rng=g) for s in sizes]


def transpose(U):
    """x<->y mirror of a state: swap axes and the two momentum components."""
    T = np.ascontiguousarray(np.transpose(U, (0, 2, 1)))
    T[[1, 2]] = T[[2, 1]]
    return T
