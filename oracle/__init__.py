"""FP64 CPU oracle of the unsplit CTU step (paper §3.2, §3.1 Eqs. 3-6) -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this package.  It is a
ctypes binding of liboracle.so (plain C, FP64) and shares no code with the CUDA library.

Arrays are numpy float64 of shape (4, ny + 2 ng, nx + 2 ng), C-contiguous: U[k, j, i] with
k in (rho, rho u, rho v, rho E), j the row (y) and i the column (x).
"""
import ctypes

import numpy as np

from . import build as _build

_LIB = None


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("ng", ctypes.c_int),
        ("xmin", ctypes.c_double), ("xmax", ctypes.c_double), ("ymin", ctypes.c_double), ("ymax", ctypes.c_double),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bc_xlo", ctypes.c_int), ("bc_xhi", ctypes.c_int), ("bc_ylo", ctypes.c_int), ("bc_yhi", ctypes.c_int),
        ("limiter", ctypes.c_int), ("use_flattening", ctypes.c_int), ("cvisc", ctypes.c_double),
        ("riemann_maxiter", ctypes.c_int), ("riemann_tol", ctypes.c_double),
        ("small_dens", ctypes.c_double), ("small_pres", ctypes.c_double), ("grav", ctypes.c_double),
        ("riemann_solver", ctypes.c_int), ("reconstruction", ctypes.c_int),
    ]


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("riemann_solves", ctypes.c_longlong), ("riemann_iters", ctypes.c_longlong),
        ("riemann_nonconv", ctypes.c_longlong), ("riemann_maxiters_seen", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(OracleParams)
        L.oracle_fill_ghost.argtypes = [P, _D]
        L.oracle_cfl_dt.argtypes = [P, _D, _D]
        L.oracle_step.argtypes = [P, _D, ctypes.c_double, ctypes.POINTER(OracleStats)]
        L.oracle_step_split.argtypes = [P, _D, ctypes.c_double, ctypes.c_int, ctypes.POINTER(OracleStats)]
        L.oracle_conserved_totals.argtypes = [P, _D, _D]
        L.oracle_cons_to_prim.argtypes = [P, _D, _D]
        L.oracle_prim_to_cons.argtypes = [P, _D, _D]
        L.oracle_slope.argtypes = [ctypes.c_int] + [ctypes.c_double] * 5
        L.oracle_slope.restype = ctypes.c_double
        L.oracle_flatten_chi.argtypes = [ctypes.c_double] * 7
        L.oracle_flatten_chi.restype = ctypes.c_double
        L.oracle_flatten_xi.argtypes = [P, _D, _D]
        L.oracle_trace.argtypes = [P, ctypes.c_double, _D, _D, _D, _D]
        L.oracle_riemann.argtypes = [P, _D, _D, ctypes.c_double, _D, _D, _D, _D, ctypes.POINTER(ctypes.c_int)]
        L.oracle_euler_flux.argtypes = [P, _D, _D]
        L.oracle_ppm_edges.argtypes = [_D, ctypes.c_double, _D]
        L.oracle_trace_ppm.argtypes = [P, ctypes.c_double, _D, _D, _D, _D, _D]
        L.oracle_hllc.argtypes = [P, _D, _D, _D, _D]
        L.oracle_hllc_core.argtypes = [P, _D, _D, ctypes.c_double, ctypes.c_double, _D, _D]
        L.oracle_num_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def params(nx, ny, *, ng=4, xmin=0.0, xmax=1.0, ymin=0.0, ymax=1.0, gamma=1.4, cfl=0.8,
           bc=("outflow", "outflow", "outflow", "outflow"), limiter=2, use_flattening=1, cvisc=0.1,
           riemann_maxiter=32, riemann_tol=1e-14, small_dens=1e-10, small_pres=1e-20, grav=0.0, riemann_solver=0,
           reconstruction=0):
    """riemann_solver: 0 (or "two-shock") the two-shock iteration, 1 (or "hllc") HLLC.
    reconstruction: 0 (or "plm") piecewise linear, 1 (or "ppm") piecewise parabolic."""
    code = {"outflow": 0, "periodic": 1, "reflect": 2, "hydrostatic": 3}
    solver = {"two-shock": 0, "hllc": 1}.get(riemann_solver, riemann_solver)
    recon = {"plm": 0, "ppm": 1}.get(reconstruction, reconstruction)
    return OracleParams(nx, ny, ng, xmin, xmax, ymin, ymax, gamma, cfl,
                        code[bc[0]], code[bc[1]], code[bc[2]], code[bc[3]],
                        limiter, use_flattening, cvisc, riemann_maxiter, riemann_tol, small_dens, small_pres, grav,
                        solver, recon)


def _ptr(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what} failed with status {rc}")


def fill_ghost(p, U):
    _check(lib().oracle_fill_ghost(ctypes.byref(p), _ptr(U)), "oracle_fill_ghost")
    return U


def cfl_dt(p, U):
    out = ctypes.c_double()
    _check(lib().oracle_cfl_dt(ctypes.byref(p), _ptr(U), ctypes.byref(out)), "oracle_cfl_dt")
    return out.value


def step(p, U, dt, stats=None):
    """One CTU step of length dt, in place on the interior of the ghost-filled state U."""
    st = stats if stats is not None else OracleStats()
    _check(lib().oracle_step(ctypes.byref(p), _ptr(U), float(dt), ctypes.byref(st)), "oracle_step")
    return U


def step_split(p, U, dt, first_dir, stats=None):
    """One dimensionally split step (§3.1): sweep along first_dir (0 x, 1 y), ghost fill, sweep along the
    other direction, in place on the ghost-filled state U."""
    st = stats if stats is not None else OracleStats()
    _check(lib().oracle_step_split(ctypes.byref(p), _ptr(U), float(dt), int(first_dir), ctypes.byref(st)),
           "oracle_step_split")
    return U


def conserved_totals(p, U):
    out = np.zeros(4)
    _check(lib().oracle_conserved_totals(ctypes.byref(p), _ptr(U), _ptr(out)), "oracle_conserved_totals")
    return out


def cons_to_prim(p, U4):
    U4 = np.ascontiguousarray(U4, dtype=np.float64)
    q = np.zeros(4)
    lib().oracle_cons_to_prim(ctypes.byref(p), _ptr(U4), _ptr(q))
    return q


def prim_to_cons(p, q4):
    q4 = np.ascontiguousarray(q4, dtype=np.float64)
    U = np.zeros(4)
    lib().oracle_prim_to_cons(ctypes.byref(p), _ptr(q4), _ptr(U))
    return U


def slope(limiter, qm2, qm1, q0, qp1, qp2):
    return lib().oracle_slope(limiter, qm2, qm1, q0, qp1, qp2)


def flatten_chi(pm2, pm1, pp1, pp2, um1, up1, small_pres=1e-20):
    return lib().oracle_flatten_chi(pm2, pm1, pp1, pp2, um1, up1, small_pres)


def flatten_xi(p, q):
    """Flattening coefficient xi[j, i] of every cell from the primitive planes q[k, j, i] (rho, u, v, p),
    shape (4, ny + 2 ng, nx + 2 ng) (§3.2 flattening; 1 on the outer three rings of cells)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    assert q.shape == (4, p.ny + 2 * p.ng, p.nx + 2 * p.ng)
    xi = np.zeros(q.shape[1:])
    _check(lib().oracle_flatten_xi(ctypes.byref(p), _ptr(q), _ptr(xi)), "oracle_flatten_xi")
    return xi


def trace(p, sigma, q, dq):
    q = np.ascontiguousarray(q, dtype=np.float64)
    dq = np.ascontiguousarray(dq, dtype=np.float64)
    ql, qr = np.zeros(4), np.zeros(4)
    lib().oracle_trace(ctypes.byref(p), float(sigma), _ptr(q), _ptr(dq), _ptr(ql), _ptr(qr))
    return ql, qr


def riemann(p, qL, qR, guess=0.0):
    """Two-shock Riemann solve in the face frame.  Returns dict(face, flux, pstar, ustar, iters, converged)."""
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    face, flux = np.zeros(4), np.zeros(4)
    ps, us = ctypes.c_double(), ctypes.c_double()
    it = ctypes.c_int()
    ok = lib().oracle_riemann(ctypes.byref(p), _ptr(qL), _ptr(qR), float(guess), _ptr(face), _ptr(flux),
                              ctypes.byref(ps), ctypes.byref(us), ctypes.byref(it))
    return dict(face=face, flux=flux, pstar=ps.value, ustar=us.value, iters=it.value, converged=bool(ok))


def euler_flux(p, q):
    q = np.ascontiguousarray(q, dtype=np.float64)
    F = np.zeros(4)
    lib().oracle_euler_flux(ctypes.byref(p), _ptr(q), _ptr(F))
    return F


def ppm_edges(a5, xi=1.0):
    """PPM edge values (aL, aR) of the middle cell of five cell averages."""
    a5 = np.ascontiguousarray(a5, dtype=np.float64)
    e = np.zeros(2)
    lib().oracle_ppm_edges(_ptr(a5), float(xi), _ptr(e))
    return e[0], e[1]


def trace_ppm(p, sigma, q, aL, aR):
    """PPM traced states (left at i+1/2, right at i-1/2) of one cell in the face frame."""
    q, aL, aR = (np.ascontiguousarray(x, dtype=np.float64) for x in (q, aL, aR))
    ql, qr = np.zeros(4), np.zeros(4)
    lib().oracle_trace_ppm(ctypes.byref(p), float(sigma), _ptr(q), _ptr(aL), _ptr(aR), _ptr(ql), _ptr(qr))
    return ql, qr


def hllc(p, qL, qR):
    """HLLC flux in the face frame with estimated wave speeds.  Returns (flux, (S_L, S*, S_R))."""
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    F, sp = np.zeros(4), np.zeros(3)
    lib().oracle_hllc(ctypes.byref(p), _ptr(qL), _ptr(qR), _ptr(F), _ptr(sp))
    return F, tuple(sp)


def hllc_core(p, qL, qR, SL, SR):
    """HLLC flux with the outer wave speeds given.  Returns (flux, S*)."""
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    F, sst = np.zeros(4), ctypes.c_double()
    lib().oracle_hllc_core(ctypes.byref(p), _ptr(qL), _ptr(qR), float(SL), float(SR), _ptr(F), ctypes.byref(sst))
    return F, sst.value


def num_threads():
    return lib().oracle_num_threads()


def advance(p, U, nsteps=None, tmax=None, stats=None, split=False):
    """The paper's driver loop (§2): fill ghosts, get dt (clamped to reach tmax), step; returns (t, n).
    split: dimensionally split steps, x first on even steps and y first on odd ones."""
    t, n = 0.0, 0
    while True:
        if nsteps is not None and n >= nsteps:
            break
        if tmax is not None and t >= tmax:
            break
        fill_ghost(p, U)
        dt = cfl_dt(p, U)
        if tmax is not None and t + dt > tmax:
            dt = tmax - t
        if split:
            step_split(p, U, dt, n % 2, stats)
        else:
            step(p, U, dt, stats)
        t += dt
        n += 1
    fill_ghost(p, U)
    return t, n
