/*
 * Plain FP64 CPU oracle of the unsplit piecewise-linear CTU step (paper §3.2 "Compressible
 * hydrodynamics", Eqs. 8-13; CTU construction of §3.1, Eqs. 3-6).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the CPU-baseline leg of
 * bench.py.  It shares no code with the CUDA library.  Compiled with -O2 -ffp-contract=off so every
 * + - * / sqrt is a separately rounded IEEE double operation.
 *
 * One stage per loop, in the paper's order:
 *   primitives q = (rho, u, v, p)                         (§3.2, Eqs. 11-12)
 *   flattening coefficient xi                             (§3.2, flattening "from Colella 1990")
 *   limited slopes, fourth-order MC                       (§3.1, limiter of Colella 1985)
 *   characteristic tracing to half-step face states       (§3.2, Eq. 13)
 *   Riemann solves on the traced ("hat") states           (§3.1 CTU / §3.2 Riemann problem)
 *   transverse flux-difference correction                 (§3.1, Eqs. 3-4; §3.2)
 *   final Riemann solves + artificial viscosity           (§3.2)
 *   conservative update                                   (§3.1, Eq. 5)
 * The readings taken where the paper defers to its references are listed in the repository's design
 * notes; each is restated at the function that applies it.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NVAR 4
enum { IR = 0, IMX = 1, IMY = 2, IE = 3 };

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int params_ok(const oracle_params* p) {
  if (!p) return 0;
  if (p->nx < 1 || p->ny < 1 || p->ng < 4) return 0;
  if (!(p->xmax > p->xmin) || !(p->ymax > p->ymin)) return 0;
  if (!(p->gamma > 1.0) || !(p->cfl > 0.0)) return 0;
  if ((p->bc_xlo == 1) != (p->bc_xhi == 1) || (p->bc_ylo == 1) != (p->bc_yhi == 1)) return 0;
  if (p->bc_xlo < 0 || p->bc_xlo > 2 || p->bc_xhi < 0 || p->bc_xhi > 2) return 0; /* hydrostatic: y only */
  if (p->bc_ylo < 0 || p->bc_ylo > 3 || p->bc_yhi < 0 || p->bc_yhi > 3) return 0;
  if (p->bc_xlo == 1 && p->nx < p->ng) return 0;
  if (p->bc_ylo == 1 && p->ny < p->ng) return 0;
  if (p->limiter < 0 || p->limiter > 2) return 0;
  if (p->riemann_maxiter < 1 || !(p->riemann_tol > 0.0)) return 0;
  if (p->riemann_solver != 0 && p->riemann_solver != 1) return 0;
  if (p->reconstruction != 0 && p->reconstruction != 1) return 0;
  if (!(p->small_dens > 0.0) || !(p->small_pres > 0.0) || p->cvisc < 0.0) return 0;
  return 1;
}

/* ------------------------------------------------------------------------------------------------ */
/* Equation of state and variable conversions: E = e + |U|^2/2 (Eq. 11), p = rho e (gamma-1) (Eq. 12). */

void oracle_cons_to_prim(const oracle_params* p, const double U[4], double q[4]) {
  double rho = U[IR];
  if (rho < p->small_dens) rho = p->small_dens;
  double u = U[IMX] / rho;
  double v = U[IMY] / rho;
  double ke = 0.5 * rho * (u * u + v * v);
  double pres = (p->gamma - 1.0) * (U[IE] - ke);
  if (pres < p->small_pres) pres = p->small_pres;
  q[0] = rho;
  q[1] = u;
  q[2] = v;
  q[3] = pres;
}

void oracle_prim_to_cons(const oracle_params* p, const double q[4], double U[4]) {
  U[IR] = q[0];
  U[IMX] = q[0] * q[1];
  U[IMY] = q[0] * q[2];
  U[IE] = q[3] / (p->gamma - 1.0) + 0.5 * q[0] * (q[1] * q[1] + q[2] * q[2]);
}

/* Flux of the Euler equations (Eqs. 8-10 with g = 0) in the face frame q = (rho, un, ut, p):
 * (rho un, rho un^2 + p, rho un ut, un (rho E + p)). */
void oracle_euler_flux(const oracle_params* p, const double q[4], double F[4]) {
  double rho = q[0], un = q[1], ut = q[2], pres = q[3];
  double rhoE = pres / (p->gamma - 1.0) + 0.5 * rho * (un * un + ut * ut);
  F[0] = rho * un;
  F[1] = rho * un * un + pres;
  F[2] = rho * un * ut;
  F[3] = un * (rhoE + pres);
}

/* ------------------------------------------------------------------------------------------------ */
/* Limited slopes (§3.1: "4th-order MC limiter from Colella 1985").
 * MC:            dl = q0-qm, dr = qp-q0, dc = (qp-qm)/2; if dl*dr > 0 the slope is
 *                sign(dc) min(|dc|, 2|dl|, 2|dr|), else 0.
 * fourth order:  d4 = (4/3) dc - (1/6)(s_{+1} + s_{-1}) with s_{+-1} the MC slopes of the neighbours;
 *                if dl*dr > 0 the slope is sign(d4) min(|d4|, 2|dl|, 2|dr|), else 0. */
static double mc_slope(double qm, double q0, double qp) {
  double dl = q0 - qm, dr = qp - q0, dc = 0.5 * (qp - qm);
  if (!(dl * dr > 0.0)) return 0.0;
  double dlim = 2.0 * fmin(fabs(dl), fabs(dr));
  double mag = fmin(fabs(dc), dlim);
  return dc >= 0.0 ? mag : -mag;
}

double oracle_slope(int limiter, double qm2, double qm1, double q0, double qp1, double qp2) {
  if (limiter == 0) return 0.0;
  if (limiter == 1) return mc_slope(qm1, q0, qp1);
  double dl = q0 - qm1, dr = qp1 - q0, dc = 0.5 * (qp1 - qm1);
  if (!(dl * dr > 0.0)) return 0.0;
  double dlim = 2.0 * fmin(fabs(dl), fabs(dr));
  double d4 = (4.0 / 3.0) * dc - (1.0 / 6.0) * (mc_slope(q0, qp1, qp2) + mc_slope(qm2, qm1, q0));
  double mag = fmin(fabs(d4), dlim);
  return d4 >= 0.0 ? mag : -mag;
}

/* ------------------------------------------------------------------------------------------------ */
/* Flattening near shocks (§3.2, "flattening ... from Colella 1990").  Shock detector on one line of
 * cells: z = |p_{+1}-p_{-1}| / max(|p_{+2}-p_{-2}|, small_pres).  Inside a compression
 * (u_{-1} - u_{+1} > 0) with a pressure jump |p_{+1}-p_{-1}| > 0.33 min(p_{+1}, p_{-1}),
 * chi = clamp(1 - (z - 0.75)/(0.85 - 0.75), 0, 1); elsewhere chi = 1. */
double oracle_flatten_chi(double pm2, double pm1, double pp1, double pp2, double um1, double up1,
                          double small_pres) {
  const double z0 = 0.75, z1 = 0.85, delta = 0.33;
  double dp1 = pp1 - pm1;
  double dp2 = pp2 - pm2;
  double z = fabs(dp1) / fmax(fabs(dp2), small_pres);
  int compress = (um1 - up1) > 0.0;
  int jump = fabs(dp1) > delta * fmin(pp1, pm1);
  if (!(compress && jump)) return 1.0;
  double chi = 1.0 - (z - z0) / (z1 - z0);
  if (chi < 0.0) chi = 0.0;
  if (chi > 1.0) chi = 1.0;
  return chi;
}

/* ------------------------------------------------------------------------------------------------ */
/* Characteristic tracing (§3.2, Eq. 13): q = (rho, un, ut, p), dq the limited slope, sigma = dt/dx.
 * Eigenvalues (un-c, un, un, un+c); left eigenvectors
 *   l1 = (0, -rho/(2c), 0, 1/(2c^2)), l2 = (1, 0, 0, -1/c^2), l3 = (0, 0, 1, 0), l4 = (0, rho/(2c), 0, 1/(2c^2))
 * and right eigenvectors
 *   r1 = (1, -c/rho, 0, c^2), r2 = (1, 0, 0, 0), r3 = (0, 0, 1, 0), r4 = (1, c/rho, 0, c^2).
 * Left state at the i+1/2 face: start from the reference extrapolation with the fastest right-moving
 * speed, q + (1 - sigma lam4) dq / 2, and add (sigma/2)(lam4 - lam_nu) beta_nu r_nu for each wave with
 * lam_nu >= 0 (moving toward that face).  Right state at the i-1/2 face: q - (1 + sigma lam1) dq / 2 plus
 * (sigma/2)(lam1 - lam_nu) beta_nu r_nu for each wave with lam_nu <= 0.  beta_nu = l_nu . dq. */
static void eigenvectors(double rho, double c, double l[4][4], double r[4][4]) {
  const double L[4][4] = {{0.0, -0.5 * rho / c, 0.0, 0.5 / (c * c)},
                          {1.0, 0.0, 0.0, -1.0 / (c * c)},
                          {0.0, 0.0, 1.0, 0.0},
                          {0.0, 0.5 * rho / c, 0.0, 0.5 / (c * c)}};
  const double R[4][4] = {{1.0, -c / rho, 0.0, c * c}, {1.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 1.0, 0.0},
                          {1.0, c / rho, 0.0, c * c}};
  memcpy(l, L, sizeof L);
  memcpy(r, R, sizeof R);
}

void oracle_trace(const oracle_params* p, double sigma, const double q[4], const double dq[4], double qL[4],
                  double qR[4]) {
  double rho = q[0], un = q[1], pres = q[3];
  double c = sqrt(p->gamma * pres / rho);
  double lam[4] = {un - c, un, un, un + c};
  double l[4][4], r[4][4];
  eigenvectors(rho, c, l, r);
  double beta[4];
  for (int nu = 0; nu < 4; ++nu) {
    double s = 0.0;
    for (int m = 0; m < 4; ++m) s += l[nu][m] * dq[m];
    beta[nu] = s;
  }
  for (int m = 0; m < 4; ++m) {
    double sl = q[m] + 0.5 * (1.0 - sigma * lam[3]) * dq[m];
    double sr = q[m] - 0.5 * (1.0 + sigma * lam[0]) * dq[m];
    for (int nu = 0; nu < 4; ++nu) {
      if (lam[nu] >= 0.0) sl += 0.5 * sigma * (lam[3] - lam[nu]) * beta[nu] * r[nu][m];
      if (lam[nu] <= 0.0) sr += 0.5 * sigma * (lam[0] - lam[nu]) * beta[nu] * r[nu][m];
    }
    qL[m] = sl;
    qR[m] = sr;
  }
  /* floors on the traced working copies */
  if (qL[0] < p->small_dens) qL[0] = p->small_dens;
  if (qR[0] < p->small_dens) qR[0] = p->small_dens;
  if (qL[3] < p->small_pres) qL[3] = p->small_pres;
  if (qR[3] < p->small_pres) qR[3] = p->small_pres;
}

/* ------------------------------------------------------------------------------------------------ */
/* Piecewise-parabolic reconstruction, the upgrade of the piecewise-linear one the paper points to (§3.2:
 * PPM of Colella & Woodward 1984, tracing as discussed by Miller & Colella 2002).  Edge values of cell i
 * from the cell averages a = (a_{i-2}, ..., a_{i+2}) of one primitive variable along one direction:
 *   interface value a_{i+1/2} = a_i + (a_{i+1} - a_i)/2 - (da_{i+1} - da_i)/6 with da the MC-limited slopes
 *     (for unlimited slopes the fourth-order 7/12 (a_i + a_{i+1}) - 1/12 (a_{i-1} + a_{i+2}));
 *   aL = a_{i-1/2}, aR = a_{i+1/2}, then the monotonicity constraints: at a local extremum,
 *     (aR - a_i)(a_i - aL) <= 0, the profile is flat, aL = aR = a_i; otherwise if the parabola's extremum
 *     falls inside the cell, (aR - aL)(a_i - (aL + aR)/2) > (aR - aL)^2 / 6 moves it to the left edge,
 *     aL = 3 a_i - 2 aR, and -(aR - aL)^2 / 6 > (aR - aL)(a_i - (aL + aR)/2) to the right one, aR = 3 a_i - 2 aL;
 *   flattening blends the edges with the cell average: aL = xi aL + (1 - xi) a_i, likewise aR.
 * edges[0] = aL, edges[1] = aR. */
void oracle_ppm_edges(const double a[5], double xi, double edges[2]) {
  double dm = mc_slope(a[0], a[1], a[2]);
  double d0 = mc_slope(a[1], a[2], a[3]);
  double dp = mc_slope(a[2], a[3], a[4]);
  double c = a[2];
  double l = a[1] + 0.5 * (a[2] - a[1]) - (d0 - dm) / 6.0;
  double r = a[2] + 0.5 * (a[3] - a[2]) - (dp - d0) / 6.0;
  if ((r - c) * (c - l) <= 0.0) {
    l = c;
    r = c;
  } else {
    double da = r - l, mid = c - 0.5 * (l + r);
    if (da * mid > da * da / 6.0)
      l = 3.0 * c - 2.0 * r;
    else if (-(da * da) / 6.0 > da * mid)
      r = 3.0 * c - 2.0 * l;
  }
  edges[0] = xi * l + (1.0 - xi) * c;
  edges[1] = xi * r + (1.0 - xi) * c;
}

/* PPM characteristic tracing (Eq. 13 with parabolic profiles).  In the cell, a(x) = aL + x (da + a6 (1 - x))
 * for x in [0, 1] with da = aR - aL, a6 = 6 (a_i - (aL + aR)/2).  The average over the fraction s of the cell
 * next to the right edge is Ip(s) = aR - (s/2)(da - (1 - 2s/3) a6), next to the left edge
 * Im(s) = aL + (s/2)(da + (1 - 2s/3) a6).  A wave of speed lam reaches the right face from the region of
 * width s = sigma lam (sigma = dt/dx) in a step.  Left state at i+1/2: reference ref = Ip(max(sigma lam4, 0))
 * (the fastest right-moving wave; the edge value if none moves right), then for each wave with lam_nu >= 0
 * subtract its part of ref - Ip(sigma lam_nu): qL = ref - sum_nu (l_nu . (ref - Ip(sigma lam_nu))) r_nu.
 * Right state at i-1/2 likewise with Im, ref = Im(max(-sigma lam1, 0)) and the waves with lam_nu <= 0.
 * Eigenvectors and floors as in oracle_trace.  With a linear profile (a6 = 0, aR - aL = dq) this is
 * oracle_trace with the slope dq. */
void oracle_trace_ppm(const oracle_params* p, double sigma, const double q[4], const double aL[4], const double aR[4],
                      double qL[4], double qR[4]) {
  double rho = q[0], un = q[1], pres = q[3];
  double c = sqrt(p->gamma * pres / rho);
  double lam[4] = {un - c, un, un, un + c};
  double l[4][4], r[4][4];
  eigenvectors(rho, c, l, r);
  double da[4], a6[4];
  for (int m = 0; m < 4; ++m) {
    da[m] = aR[m] - aL[m];
    a6[m] = 6.0 * (q[m] - 0.5 * (aL[m] + aR[m]));
  }
  /* left state at i+1/2 */
  {
    double s4 = sigma * lam[3] > 0.0 ? sigma * lam[3] : 0.0;
    double ref[4], out[4];
    for (int m = 0; m < 4; ++m) {
      ref[m] = aR[m] - 0.5 * s4 * (da[m] - (1.0 - (2.0 / 3.0) * s4) * a6[m]);
      out[m] = ref[m];
    }
    for (int nu = 0; nu < 4; ++nu) {
      if (!(lam[nu] >= 0.0)) continue;
      double sn = sigma * lam[nu];
      double beta = 0.0;
      for (int m = 0; m < 4; ++m) {
        double ip = aR[m] - 0.5 * sn * (da[m] - (1.0 - (2.0 / 3.0) * sn) * a6[m]);
        beta += l[nu][m] * (ref[m] - ip);
      }
      for (int m = 0; m < 4; ++m) out[m] -= beta * r[nu][m];
    }
    for (int m = 0; m < 4; ++m) qL[m] = out[m];
  }
  /* right state at i-1/2 */
  {
    double s1 = -sigma * lam[0] > 0.0 ? -sigma * lam[0] : 0.0;
    double ref[4], out[4];
    for (int m = 0; m < 4; ++m) {
      ref[m] = aL[m] + 0.5 * s1 * (da[m] + (1.0 - (2.0 / 3.0) * s1) * a6[m]);
      out[m] = ref[m];
    }
    for (int nu = 0; nu < 4; ++nu) {
      if (!(lam[nu] <= 0.0)) continue;
      double sn = -sigma * lam[nu];
      double beta = 0.0;
      for (int m = 0; m < 4; ++m) {
        double im = aL[m] + 0.5 * sn * (da[m] + (1.0 - (2.0 / 3.0) * sn) * a6[m]);
        beta += l[nu][m] * (ref[m] - im);
      }
      for (int m = 0; m < 4; ++m) out[m] -= beta * r[nu][m];
    }
    for (int m = 0; m < 4; ++m) qR[m] = out[m];
  }
  if (qL[0] < p->small_dens) qL[0] = p->small_dens;
  if (qR[0] < p->small_dens) qR[0] = p->small_dens;
  if (qL[3] < p->small_pres) qL[3] = p->small_pres;
  if (qR[3] < p->small_pres) qR[3] = p->small_pres;
}

/* Traced states of one cell along one direction, in the face frame, from the selected reconstruction:
 * piecewise linear (the limited slope dq) or piecewise parabolic (edges from the five cells a5[k][0..4]). */
static void trace_cell(const oracle_params* p, double sigma, const double q[4], const double dq[4],
                       const double a5[4][5], double xi, double qL[4], double qR[4]) {
  if (p->reconstruction == 1) {
    double aL[4], aR[4], e[2];
    for (int k = 0; k < 4; ++k) {
      oracle_ppm_edges(a5[k], xi, e);
      aL[k] = e[0];
      aR[k] = e[1];
    }
    oracle_trace_ppm(p, sigma, q, aL, aR, qL, qR);
  } else {
    oracle_trace(p, sigma, q, dq, qL, qR);
  }
}

/* ------------------------------------------------------------------------------------------------ */
/* Two-shock approximate Riemann solver (§3.2, solver "described in almgren:2010").  Both waves are
 * treated as shocks: with C_K = sqrt(gamma p_K rho_K) and the shock mass flux
 *   W_K(p) = C_K sqrt(1 + (gamma+1)/(2 gamma) (p/p_K - 1)),
 * the star velocity seen from each side is u*_L = u_L - (p - p_L)/W_L, u*_R = u_R + (p - p_R)/W_R, and p*
 * solves u*_L(p) = u*_R(p).  Newton iteration with slopes Z_K = 2 W_K^3 / (W_K^2 + C_K^2)
 * (= |dp/du*| along each Hugoniot), started from the acoustic guess, stopped when |dp| <= tol p or when
 * the velocity mismatch |dp| (1/Z_L + 1/Z_R) of the step is <= tol (|u_L| + |u_R| + c_L + c_R).
 * Sampling at x/t = 0: upwind side o from the sign of u*; star density from the Hugoniot
 * 1/rho* = 1/rho_o - (p* - p_o)/W_o^2; a shock (p* > p_o) moving at u_o -+ W_o/rho_o, else a fan between
 * u_o -+ c_o and u* -+ c*, interpolated linearly when the face lies inside it. */
int oracle_riemann(const oracle_params* p, const double qL[4], const double qR[4], double guess, double face[4],
                   double flux[4], double* pstar_out, double* ustar_out, int* iters_out) {
  const double g = p->gamma;
  const double g1 = (g + 1.0) / (2.0 * g);
  double rl = qL[0], ul = qL[1], vl = qL[2], pl = qL[3];
  double rr = qR[0], ur = qR[1], vr = qR[2], pr = qR[3];
  double cl = sqrt(g * pl * rl);
  double cr = sqrt(g * pr * rr);
  /* velocity scale |u_L| + |u_R| + c_L + c_R (c = C/rho): a Newton step |dp| equals a velocity mismatch
   * |dp| (1/Z_L + 1/Z_R); the iteration also stops once that mismatch is below tol times this scale,
   * which rounding allows even when p* << rho u^2 (where |dp| <= tol p* may be out of reach) */
  double vscale = fabs(ul) + fabs(ur) + cl / rl + cr / rr;
  double pst;
  if (guess > 0.0) {
    pst = guess;
  } else {
    pst = (cr * pl + cl * pr + cl * cr * (ul - ur)) / (cl + cr);
  }
  if (pst < p->small_pres) pst = p->small_pres;
  int it = 0, converged = 0;
  while (it < p->riemann_maxiter) {
    double wl = cl * sqrt(1.0 + g1 * (pst / pl - 1.0));
    double wr = cr * sqrt(1.0 + g1 * (pst / pr - 1.0));
    double usl = ul - (pst - pl) / wl;
    double usr = ur + (pst - pr) / wr;
    double zl = 2.0 * wl * wl * wl / (wl * wl + cl * cl);
    double zr = 2.0 * wr * wr * wr / (wr * wr + cr * cr);
    double pnew = pst - zl * zr * (usr - usl) / (zl + zr);
    if (pnew < p->small_pres) pnew = p->small_pres;
    double dp = fabs(pnew - pst);
    pst = pnew;
    ++it;
    if (dp <= p->riemann_tol * pst || dp * (zl + zr) / (zl * zr) <= p->riemann_tol * vscale) {
      converged = 1;
      break;
    }
  }
  double wl = cl * sqrt(1.0 + g1 * (pst / pl - 1.0));
  double wr = cr * sqrt(1.0 + g1 * (pst / pr - 1.0));
  double ust = ((wl * ul + wr * ur) + (pl - pr)) / (wl + wr);

  double f[4];
  if (ust == 0.0) {
    /* face on a stationary contact: normal velocity zero, pressure p*; density and transverse velocity
     * are the mean of the two sides (they do not enter the flux, which is (0, p*, 0, 0)). */
    f[0] = 0.5 * (rl + rr);
    f[1] = 0.0;
    f[2] = 0.5 * (vl + vr);
    f[3] = pst;
  } else {
    double s, ro, uo, vo, po, wo;
    if (ust > 0.0) {
      s = 1.0; ro = rl; uo = ul; vo = vl; po = pl; wo = wl;
    } else {
      s = -1.0; ro = rr; uo = ur; vo = vr; po = pr; wo = wr;
    }
    double rst = 1.0 / (1.0 / ro - (pst - po) / (wo * wo));
    if (pst > po) {
      double S = uo - s * wo / ro;
      if (s * S >= 0.0) {
        f[0] = ro; f[1] = uo; f[2] = vo; f[3] = po;
      } else {
        f[0] = rst; f[1] = ust; f[2] = vo; f[3] = pst;
      }
    } else {
      double co = sqrt(g * po / ro);
      double cst = sqrt(g * pst / rst);
      double SH = uo - s * co;
      double ST = ust - s * cst;
      if (s * SH >= 0.0) {
        f[0] = ro; f[1] = uo; f[2] = vo; f[3] = po;
      } else if (s * ST <= 0.0) {
        f[0] = rst; f[1] = ust; f[2] = vo; f[3] = pst;
      } else {
        double frac = SH / (SH - ST);
        f[0] = ro + frac * (rst - ro);
        f[1] = uo + frac * (ust - uo);
        f[2] = vo;
        f[3] = po + frac * (pst - po);
      }
    }
  }
  if (face) memcpy(face, f, sizeof f);
  if (flux) oracle_euler_flux(p, f, flux);
  if (pstar_out) *pstar_out = pst;
  if (ustar_out) *ustar_out = ust;
  if (iters_out) *iters_out = it;
  return converged;
}

/* ------------------------------------------------------------------------------------------------ */
/* HLLC approximate Riemann solver, the alternative the paper names (§3.2, after Toro 1997), in the face
 * frame q = (rho, u_normal, u_transverse, p).  Three waves S_L <= S* <= S_R bound two star states; the flux
 * at the face (x/t = 0) is the one of the region the face lies in:
 *   0 <= S_L:        F(U_L)
 *   S_L < 0 <= S*:   F(U_L) + S_L (U*_L - U_L)
 *   S* < 0 <= S_R:   F(U_R) + S_R (U*_R - U_R)
 *   S_R < 0:         F(U_R)
 * with the contact speed
 *   S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R)) / (rho_L (S_L - u_L) - rho_R (S_R - u_R))
 * and the star states (K = L, R)
 *   U*_K = rho_K (S_K - u_K) / (S_K - S*) (1, S*, v_K, E_K / rho_K + (S* - u_K) (S* + p_K / (rho_K (S_K - u_K)))).
 * oracle_hllc_core takes S_L and S_R as given.  oracle_hllc takes the direct (Davis) estimates that bound
 * the sound waves of both sides, S_L = min(u_L - c_L, u_R - c_R) and S_R = max(u_L + c_L, u_R + c_R).  (The
 * linearised-pressure estimates underestimate strong collisions so badly that S_L can come out positive
 * while the true left shock moves left; the bounds above keep the face inside the fan.) */
void oracle_hllc_core(const oracle_params* p, const double qL[4], const double qR[4], double SL, double SR,
                      double flux[4], double* sstar_out) {
  const double g = p->gamma;
  double rl = qL[0], ul = qL[1], vl = qL[2], pl = qL[3];
  double rr = qR[0], ur = qR[1], vr = qR[2], pr = qR[3];
  double El = pl / (g - 1.0) + 0.5 * rl * (ul * ul + vl * vl);
  double Er = pr / (g - 1.0) + 0.5 * rr * (ur * ur + vr * vr);
  double sst = (pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur)) / (rl * (SL - ul) - rr * (SR - ur));
  if (sstar_out) *sstar_out = sst;
  double F[4];
  if (0.0 <= SL) {
    oracle_euler_flux(p, qL, flux);
  } else if (0.0 <= sst) {
    oracle_euler_flux(p, qL, F);
    double Ul[4] = {rl, rl * ul, rl * vl, El};
    double f = rl * (SL - ul) / (SL - sst);
    double Us[4] = {f, f * sst, f * vl, f * (El / rl + (sst - ul) * (sst + pl / (rl * (SL - ul))))};
    for (int k = 0; k < 4; ++k) flux[k] = F[k] + SL * (Us[k] - Ul[k]);
  } else if (0.0 <= SR) {
    oracle_euler_flux(p, qR, F);
    double Ur[4] = {rr, rr * ur, rr * vr, Er};
    double f = rr * (SR - ur) / (SR - sst);
    double Us[4] = {f, f * sst, f * vr, f * (Er / rr + (sst - ur) * (sst + pr / (rr * (SR - ur))))};
    for (int k = 0; k < 4; ++k) flux[k] = F[k] + SR * (Us[k] - Ur[k]);
  } else {
    oracle_euler_flux(p, qR, flux);
  }
}

void oracle_hllc(const oracle_params* p, const double qL[4], const double qR[4], double flux[4], double speeds[3]) {
  const double g = p->gamma;
  double cl = sqrt(g * qL[3] / qL[0]), cr = sqrt(g * qR[3] / qR[0]);
  double SL = fmin(qL[1] - cl, qR[1] - cr);
  double SR = fmax(qL[1] + cl, qR[1] + cr);
  double sst;
  oracle_hllc_core(p, qL, qR, SL, SR, flux, &sst);
  if (speeds) {
    speeds[0] = SL;
    speeds[1] = sst;
    speeds[2] = SR;
  }
}

/* Flux at a face from the selected solver: the two-shock iteration (riemann_solver 0) or HLLC (1, no
 * iterations).  Returns 1 when the solve converged. */
static int face_flux(const oracle_params* p, const double qL[4], const double qR[4], double F[4], int* iters) {
  if (p->riemann_solver == 1) {
    oracle_hllc(p, qL, qR, F, NULL);
    *iters = 0;
    return 1;
  }
  return oracle_riemann(p, qL, qR, 0.0, NULL, F, NULL, NULL, iters);
}

/* ------------------------------------------------------------------------------------------------ */
/* Ghost cells (§2 CellCenterData2d "filling ghost cells"; Fig. 1; zero-gradient copy as described for
 * the RT problem in §3.2.3): outflow copies the last valid cell, periodic wraps.  The x pass fills the
 * ghost columns of the interior rows, then the y pass fills whole ghost rows, so corners are defined. */
/* Ghost cells (paper §2 and the RT set-up of §3.2): x pass over the interior rows, then y pass over the
 * full padded width, so that corners are consistent.
 *   outflow (0): copy of the nearest interior cell (zero gradient);
 *   periodic (1): wrap;
 *   reflecting (2): mirror image of the interior across the wall, normal momentum negated;
 *   hydrostatic (3, y sides): density and both momenta copied from the row next to the wall; the pressure
 *     of that row's cell integrated with dp/dy = rho g at constant rho into the ghost cells,
 *     p = p_edge + rho g (y - y_edge), and the energy rebuilt from it (p/(gamma-1) + kinetic). */
int oracle_fill_ghost(const oracle_params* p, double* U) {
  if (!params_ok(p) || !U) return 1;
  const int ng = p->ng, nx = p->nx, ny = p->ny, NX = nx + 2 * ng, NY = ny + 2 * ng;
  const size_t plane = (size_t)NX * NY;
  const double dy = (p->ymax - p->ymin) / ny;
  for (int k = 0; k < NVAR; ++k) {
    double* a = U + (size_t)k * plane;
    const double flip = (k == IMX) ? -1.0 : 1.0;
    for (int j = ng; j < ng + ny; ++j) {
      double* row = a + (size_t)j * NX;
      for (int i = 0; i < ng; ++i)
        row[i] = p->bc_xlo == 1 ? row[i + nx] : p->bc_xlo == 2 ? flip * row[2 * ng - 1 - i] : row[ng];
      for (int i = ng + nx; i < NX; ++i)
        row[i] = p->bc_xhi == 1   ? row[i - nx]
                 : p->bc_xhi == 2 ? flip * row[2 * (ng + nx) - 1 - i]
                                  : row[ng + nx - 1];
    }
  }
  for (int side = 0; side < 2; ++side) {
    const int bc = side == 0 ? p->bc_ylo : p->bc_yhi;
    const int edge = side == 0 ? ng : ng + ny - 1;
    for (int j = (side == 0 ? 0 : ng + ny); j < (side == 0 ? ng : NY); ++j) {
      const int src = bc == 1 ? (side == 0 ? j + ny : j - ny)
                      : bc == 2 ? (side == 0 ? 2 * ng - 1 - j : 2 * (ng + ny) - 1 - j)
                                : edge;
      for (int i = 0; i < NX; ++i) {
        const size_t d = (size_t)j * NX + i, s = (size_t)src * NX + i;
        if (bc == 3) {
          const double rho = U[s], mx = U[s + plane], my = U[s + 2 * plane];
          const double ke = 0.5 * (mx * mx + my * my) / rho;
          const double pe = (p->gamma - 1.0) * (U[s + 3 * plane] - ke);
          const double pg = pe + rho * p->grav * ((double)(j - edge) * dy);
          U[d] = rho;
          U[d + plane] = mx;
          U[d + 2 * plane] = my;
          U[d + 3 * plane] = pg / (p->gamma - 1.0) + ke;
        } else {
          for (int k = 0; k < NVAR; ++k) {
            const double flip = (bc == 2 && k == IMY) ? -1.0 : 1.0;
            U[d + k * plane] = flip * U[s + k * plane];
          }
        }
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------------ */
/* CFL time step (§3.1, Eq. 6, with the signal speed |u|+c of the Euler system):
 * dt = cfl * min over interior cells of min(dx/(|u|+c), dy/(|v|+c)). */
int oracle_cfl_dt(const oracle_params* p, const double* U, double* dt_out) {
  if (!params_ok(p) || !U || !dt_out) return 1;
  const int ng = p->ng, nx = p->nx, ny = p->ny, NX = nx + 2 * ng, NY = ny + 2 * ng;
  const size_t plane = (size_t)NX * NY;
  const double dx = (p->xmax - p->xmin) / nx, dy = (p->ymax - p->ymin) / ny;
  double best = INFINITY;
#pragma omp parallel for reduction(min : best)
  for (int j = ng; j < ng + ny; ++j) {
    for (int i = ng; i < ng + nx; ++i) {
      size_t c = (size_t)j * NX + i;
      double Uc[4] = {U[c], U[c + plane], U[c + 2 * plane], U[c + 3 * plane]};
      double q[4];
      oracle_cons_to_prim(p, Uc, q);
      double cs = sqrt(p->gamma * q[3] / q[0]);
      double tx = dx / (fabs(q[1]) + cs);
      double ty = dy / (fabs(q[2]) + cs);
      double t = fmin(tx, ty);
      if (t < best) best = t;
    }
  }
  *dt_out = p->cfl * best;
  return 0;
}

/* Conserved totals sum_ij U_k dx dy over the interior (compensated summation, row-major order). */
int oracle_conserved_totals(const oracle_params* p, const double* U, double out[4]) {
  if (!params_ok(p) || !U || !out) return 1;
  const int ng = p->ng, nx = p->nx, ny = p->ny, NX = nx + 2 * ng, NY = ny + 2 * ng;
  const double dx = (p->xmax - p->xmin) / nx, dy = (p->ymax - p->ymin) / ny;
  for (int k = 0; k < NVAR; ++k) {
    const double* a = U + (size_t)k * NX * NY;
    double s = 0.0, comp = 0.0;
    for (int j = ng; j < ng + ny; ++j)
      for (int i = ng; i < ng + nx; ++i) {
        double x = a[(size_t)j * NX + i];
        double t = s + x;
        if (fabs(s) >= fabs(x))
          comp += (s - t) + x;
        else
          comp += (x - t) + s;
        s = t;
      }
    out[k] = (s + comp) * dx * dy;
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------------ */
/* One CTU step of length dt on a ghost-filled state, in place on the interior. */

typedef struct {
  double* a;
  int NX, NY;
} grid_arr;

#define AT(arr, k, j, i) ((arr)[((size_t)(k) * NY + (j)) * NX + (i)])

/* ------------------------------------------------------------------------------------------------ */
/* Flattening coefficient of every cell (§3.2, flattening "from Colella 1990", whose detector is that of
 * Colella & Woodward 1984).  q: primitives [4][NY][NX] (rho, u, v, p planes); xi: [NY][NX] output.
 * Per direction, chi_i is the shock detector of oracle_flatten_chi on the line through cell i (normal
 * velocity u along x, v along y).  Each cell then also takes the detector of its lower-pressure
 * neighbour: xi_d(i) = min(chi_i, chi_{i-s}) with s = sign(p_{i+1} - p_{i-1}) (s = +1 where the two are
 * equal), so the flattened band of a shock reaches one cell further into its high-pressure (post-shock)
 * side and no further into the low-pressure side.  xi = min(xi_x, xi_y): a cell is flattened as much as
 * its stronger direction asks.  Defined on cells [3, NX-3) x [3, NY-3); 1 elsewhere
 * and everywhere when use_flattening = 0.  Returns 0, or 2 when out of memory. */
int oracle_flatten_xi(const oracle_params* p, const double* q, double* xi) {
  const int NX = p->nx + 2 * p->ng, NY = p->ny + 2 * p->ng;
  const size_t plane = (size_t)NX * NY;
#pragma omp parallel for
  for (int j = 0; j < NY; ++j)
    for (int i = 0; i < NX; ++i) AT(xi, 0, j, i) = 1.0;
  if (!p->use_flattening) return 0;
  double* chix = calloc(plane, sizeof(double));
  double* chiy = calloc(plane, sizeof(double));
  if (!chix || !chiy) {
    free(chix);
    free(chiy);
    return 2;
  }
#pragma omp parallel for
  for (int j = 0; j < NY; ++j)
    for (int i = 0; i < NX; ++i) {
      chix[(size_t)j * NX + i] = 1.0;
      chiy[(size_t)j * NX + i] = 1.0;
      if (i >= 2 && i < NX - 2)
        chix[(size_t)j * NX + i] =
            oracle_flatten_chi(AT(q, 3, j, i - 2), AT(q, 3, j, i - 1), AT(q, 3, j, i + 1), AT(q, 3, j, i + 2),
                               AT(q, 1, j, i - 1), AT(q, 1, j, i + 1), p->small_pres);
      if (j >= 2 && j < NY - 2)
        chiy[(size_t)j * NX + i] =
            oracle_flatten_chi(AT(q, 3, j - 2, i), AT(q, 3, j - 1, i), AT(q, 3, j + 1, i), AT(q, 3, j + 2, i),
                               AT(q, 2, j - 1, i), AT(q, 2, j + 1, i), p->small_pres);
    }
#pragma omp parallel for
  for (int j = 3; j < NY - 3; ++j)
    for (int i = 3; i < NX - 3; ++i) {
      int sx = (AT(q, 3, j, i + 1) - AT(q, 3, j, i - 1)) >= 0.0 ? 1 : -1;
      int sy = (AT(q, 3, j + 1, i) - AT(q, 3, j - 1, i)) >= 0.0 ? 1 : -1;
      double xix = fmin(chix[(size_t)j * NX + i], chix[(size_t)j * NX + i - sx]);
      double xiy = fmin(chiy[(size_t)j * NX + i], chiy[(size_t)(j - sy) * NX + i]);
      AT(xi, 0, j, i) = fmin(xix, xiy);
    }
  free(chix);
  free(chiy);
  return 0;
}

int oracle_step(const oracle_params* p, double* U, double dt, oracle_stats* st) {
  if (!params_ok(p) || !U || !(dt >= 0.0)) return 1;
  const int ng = p->ng, nx = p->nx, ny = p->ny, NX = nx + 2 * ng, NY = ny + 2 * ng;
  const size_t plane = (size_t)NX * NY;
  const double dx = (p->xmax - p->xmin) / nx, dy = (p->ymax - p->ymin) / ny;
  const double g = p->gamma;

  /* work arrays, all NX x NY per component */
  double* q = calloc(4 * plane, sizeof(double));      /* primitives */
  double* xi = calloc(plane, sizeof(double));         /* flattening coefficient */
  double* dqx = calloc(4 * plane, sizeof(double));    /* limited x slopes */
  double* dqy = calloc(4 * plane, sizeof(double));    /* limited y slopes */
  double* qxl = calloc(4 * plane, sizeof(double));    /* traced x states: left state at i+1/2 */
  double* qxr = calloc(4 * plane, sizeof(double));    /*                  right state at i-1/2 */
  double* qyl = calloc(4 * plane, sizeof(double));    /* traced y states: left (lower) state at j+1/2 */
  double* qyr = calloc(4 * plane, sizeof(double));    /*                  right (upper) state at j-1/2 */
  double* fxh = calloc(4 * plane, sizeof(double));    /* hat x fluxes, face f = between cells f-1 and f */
  double* fyh = calloc(4 * plane, sizeof(double));    /* hat y fluxes, face g = between rows g-1 and g */
  double* fx = calloc(4 * plane, sizeof(double));     /* final x fluxes */
  double* fy = calloc(4 * plane, sizeof(double));     /* final y fluxes */
  int err = 0;
  if (!q || !xi || !dqx || !dqy || !qxl || !qxr || !qyl || !qyr || !fxh || !fyh || !fx || !fy) {
    err = 2;
    goto done;
  }
  long long n_solves = 0, n_iters = 0, n_nonconv = 0;
  int max_iters = 0;

  /* 1. primitive variables on every cell (Eqs. 11-12) */
#pragma omp parallel for
  for (int j = 0; j < NY; ++j)
    for (int i = 0; i < NX; ++i) {
      double Uc[4], qc[4];
      for (int k = 0; k < 4; ++k) Uc[k] = AT(U, k, j, i);
      oracle_cons_to_prim(p, Uc, qc);
      for (int k = 0; k < 4; ++k) AT(q, k, j, i) = qc[k];
    }

  /* 2. flattening coefficient xi (oracle_flatten_xi) */
  if (oracle_flatten_xi(p, q, xi)) {
    err = 2;
    goto done;
  }

  /* 3. limited slopes of the primitives in x and y, multiplied by xi */
#pragma omp parallel for
  for (int j = 0; j < NY; ++j)
    for (int i = 0; i < NX; ++i)
      for (int k = 0; k < 4; ++k) {
        double sx = 0.0, sy = 0.0;
        if (i >= 2 && i < NX - 2)
          sx = oracle_slope(p->limiter, AT(q, k, j, i - 2), AT(q, k, j, i - 1), AT(q, k, j, i), AT(q, k, j, i + 1),
                            AT(q, k, j, i + 2));
        if (j >= 2 && j < NY - 2)
          sy = oracle_slope(p->limiter, AT(q, k, j - 2, i), AT(q, k, j - 1, i), AT(q, k, j, i), AT(q, k, j + 1, i),
                            AT(q, k, j + 2, i));
        AT(dqx, k, j, i) = AT(xi, 0, j, i) * sx;
        AT(dqy, k, j, i) = AT(xi, 0, j, i) * sy;
      }

  /* 4. characteristic tracing to the four half-step face states of each cell (Eq. 13) on cells
   *    [3, NX-3) x [3, NY-3).  In y the normal velocity is v and the transverse one u.  With gravity
   *    (the rho g source of §3.2's Euler equations) the half-step states of v gain dt g / 2. */
  const double sigx = dt / dx, sigy = dt / dy;
  const double hdtg = 0.5 * dt * p->grav;
#pragma omp parallel for
  for (int j = 3; j < NY - 3; ++j)
    for (int i = 3; i < NX - 3; ++i) {
      double qc[4] = {AT(q, 0, j, i), AT(q, 1, j, i), AT(q, 2, j, i), AT(q, 3, j, i)};
      double dx4[4] = {AT(dqx, 0, j, i), AT(dqx, 1, j, i), AT(dqx, 2, j, i), AT(dqx, 3, j, i)};
      double a5[4][5], b5[4][5]; /* the five cells along x and along y (face frame), for PPM */
      for (int m = 0; m < 5; ++m) {
        for (int k = 0; k < 4; ++k) a5[k][m] = AT(q, k, j, i - 2 + m);
        b5[0][m] = AT(q, 0, j - 2 + m, i);
        b5[1][m] = AT(q, 2, j - 2 + m, i);
        b5[2][m] = AT(q, 1, j - 2 + m, i);
        b5[3][m] = AT(q, 3, j - 2 + m, i);
      }
      double ql[4], qr[4];
      trace_cell(p, sigx, qc, dx4, (const double(*)[5])a5, AT(xi, 0, j, i), ql, qr);
      if (p->grav != 0.0) { /* half-step gravity on v (transverse in x) */
        ql[2] = ql[2] + hdtg;
        qr[2] = qr[2] + hdtg;
      }
      for (int k = 0; k < 4; ++k) {
        AT(qxl, k, j, i) = ql[k];
        AT(qxr, k, j, i) = qr[k];
      }
      double qn[4] = {qc[0], qc[2], qc[1], qc[3]};
      double dy4[4] = {AT(dqy, 0, j, i), AT(dqy, 2, j, i), AT(dqy, 1, j, i), AT(dqy, 3, j, i)};
      trace_cell(p, sigy, qn, dy4, (const double(*)[5])b5, AT(xi, 0, j, i), ql, qr);
      if (p->grav != 0.0) { /* half-step gravity on v (normal in y) */
        ql[1] = ql[1] + hdtg;
        qr[1] = qr[1] + hdtg;
      }
      /* back to (rho, u, v, p) order */
      double yl[4] = {ql[0], ql[2], ql[1], ql[3]}, yr[4] = {qr[0], qr[2], qr[1], qr[3]};
      for (int k = 0; k < 4; ++k) {
        AT(qyl, k, j, i) = yl[k];
        AT(qyr, k, j, i) = yr[k];
      }
    }

  /* 5. Riemann solves on the hat states.  x face f (between cells f-1 and f) for f in [4, NX-3),
   *    rows [3, NY-3); y face g for g in [4, NY-3), columns [3, NX-3). */
#pragma omp parallel for reduction(+ : n_solves, n_iters, n_nonconv) reduction(max : max_iters)
  for (int j = 3; j < NY - 3; ++j)
    for (int f = 4; f < NX - 3; ++f) {
      double a[4] = {AT(qxl, 0, j, f - 1), AT(qxl, 1, j, f - 1), AT(qxl, 2, j, f - 1), AT(qxl, 3, j, f - 1)};
      double b[4] = {AT(qxr, 0, j, f), AT(qxr, 1, j, f), AT(qxr, 2, j, f), AT(qxr, 3, j, f)};
      double F[4];
      int it;
      int ok = face_flux(p, a, b, F, &it);
      n_solves++;
      n_iters += it;
      if (!ok) n_nonconv++;
      if (it > max_iters) max_iters = it;
      AT(fxh, 0, j, f) = F[0];
      AT(fxh, 1, j, f) = F[1];
      AT(fxh, 2, j, f) = F[2];
      AT(fxh, 3, j, f) = F[3];
    }
#pragma omp parallel for reduction(+ : n_solves, n_iters, n_nonconv) reduction(max : max_iters)
  for (int gg = 4; gg < NY - 3; ++gg)
    for (int i = 3; i < NX - 3; ++i) {
      double a[4] = {AT(qyl, 0, gg - 1, i), AT(qyl, 2, gg - 1, i), AT(qyl, 1, gg - 1, i), AT(qyl, 3, gg - 1, i)};
      double b[4] = {AT(qyr, 0, gg, i), AT(qyr, 2, gg, i), AT(qyr, 1, gg, i), AT(qyr, 3, gg, i)};
      double F[4];
      int it;
      int ok = face_flux(p, a, b, F, &it);
      n_solves++;
      n_iters += it;
      if (!ok) n_nonconv++;
      if (it > max_iters) max_iters = it;
      /* face-frame flux (mass, normal mom, transverse mom, energy) -> (rho, rho u, rho v, rho E) */
      AT(fyh, 0, gg, i) = F[0];
      AT(fyh, 1, gg, i) = F[2];
      AT(fyh, 2, gg, i) = F[1];
      AT(fyh, 3, gg, i) = F[3];
    }

  /* 6. transverse correction of the conserved face states and final Riemann solves.
   *    x face f, row j (interior faces f in [ng, ng+nx], rows [ng, ng+ny)):
   *      U_L = cons(qxl[f-1]) - dt/(2dy) (fyh[j+1][f-1] - fyh[j][f-1])
   *      U_R = cons(qxr[f])   - dt/(2dy) (fyh[j+1][f]   - fyh[j][f])
   *    y faces likewise with dt/(2dx) and the hat x fluxes. */
  const double hx = 0.5 * dt / dx, hy = 0.5 * dt / dy;
#pragma omp parallel for reduction(+ : n_solves, n_iters, n_nonconv) reduction(max : max_iters)
  for (int j = ng; j < ng + ny; ++j)
    for (int f = ng; f <= ng + nx; ++f) {
      double a[4] = {AT(qxl, 0, j, f - 1), AT(qxl, 1, j, f - 1), AT(qxl, 2, j, f - 1), AT(qxl, 3, j, f - 1)};
      double b[4] = {AT(qxr, 0, j, f), AT(qxr, 1, j, f), AT(qxr, 2, j, f), AT(qxr, 3, j, f)};
      double UL[4], UR[4];
      oracle_prim_to_cons(p, a, UL);
      oracle_prim_to_cons(p, b, UR);
      for (int k = 0; k < 4; ++k) {
        UL[k] = UL[k] - hy * (AT(fyh, k, j + 1, f - 1) - AT(fyh, k, j, f - 1));
        UR[k] = UR[k] - hy * (AT(fyh, k, j + 1, f) - AT(fyh, k, j, f));
      }
      double ql[4], qr[4];
      oracle_cons_to_prim(p, UL, ql);
      oracle_cons_to_prim(p, UR, qr);
      double F[4];
      int it;
      int ok = face_flux(p, ql, qr, F, &it);
      n_solves++;
      n_iters += it;
      if (!ok) n_nonconv++;
      if (it > max_iters) max_iters = it;
      for (int k = 0; k < 4; ++k) AT(fx, k, j, f) = F[k];
    }
#pragma omp parallel for reduction(+ : n_solves, n_iters, n_nonconv) reduction(max : max_iters)
  for (int gg = ng; gg <= ng + ny; ++gg)
    for (int i = ng; i < ng + nx; ++i) {
      double a[4] = {AT(qyl, 0, gg - 1, i), AT(qyl, 1, gg - 1, i), AT(qyl, 2, gg - 1, i), AT(qyl, 3, gg - 1, i)};
      double b[4] = {AT(qyr, 0, gg, i), AT(qyr, 1, gg, i), AT(qyr, 2, gg, i), AT(qyr, 3, gg, i)};
      double UL[4], UR[4];
      oracle_prim_to_cons(p, a, UL);
      oracle_prim_to_cons(p, b, UR);
      for (int k = 0; k < 4; ++k) {
        UL[k] = UL[k] - hx * (AT(fxh, k, gg - 1, i + 1) - AT(fxh, k, gg - 1, i));
        UR[k] = UR[k] - hx * (AT(fxh, k, gg, i + 1) - AT(fxh, k, gg, i));
      }
      double ql[4], qr[4];
      oracle_cons_to_prim(p, UL, ql);
      oracle_cons_to_prim(p, UR, qr);
      double qln[4] = {ql[0], ql[2], ql[1], ql[3]}, qrn[4] = {qr[0], qr[2], qr[1], qr[3]};
      double F[4];
      int it;
      int ok = face_flux(p, qln, qrn, F, &it);
      n_solves++;
      n_iters += it;
      if (!ok) n_nonconv++;
      if (it > max_iters) max_iters = it;
      AT(fy, 0, gg, i) = F[0];
      AT(fy, 1, gg, i) = F[2];
      AT(fy, 2, gg, i) = F[1];
      AT(fy, 3, gg, i) = F[3];
    }

  /* 7. artificial viscosity (§3.2, "artificial viscosity ... from Colella 1990"): at x face f, row j,
   *    div = (u[f]-u[f-1])/dx + (v[j+1][f] + v[j+1][f-1] - v[j-1][f] - v[j-1][f-1])/(4 dy),
   *    F += cvisc max(-div dx, 0) (U[f-1] - U[f]); y faces symmetric. */
  if (p->cvisc > 0.0) {
#pragma omp parallel for
    for (int j = ng; j < ng + ny; ++j)
      for (int f = ng; f <= ng + nx; ++f) {
        double div = (AT(q, 1, j, f) - AT(q, 1, j, f - 1)) / dx +
                     (AT(q, 2, j + 1, f) + AT(q, 2, j + 1, f - 1) - AT(q, 2, j - 1, f) - AT(q, 2, j - 1, f - 1)) /
                         (4.0 * dy);
        double av = p->cvisc * fmax(-div * dx, 0.0);
        for (int k = 0; k < 4; ++k) AT(fx, k, j, f) += av * (AT(U, k, j, f - 1) - AT(U, k, j, f));
      }
#pragma omp parallel for
    for (int gg = ng; gg <= ng + ny; ++gg)
      for (int i = ng; i < ng + nx; ++i) {
        double div = (AT(q, 2, gg, i) - AT(q, 2, gg - 1, i)) / dy +
                     (AT(q, 1, gg, i + 1) + AT(q, 1, gg - 1, i + 1) - AT(q, 1, gg, i - 1) - AT(q, 1, gg - 1, i - 1)) /
                         (4.0 * dx);
        double av = p->cvisc * fmax(-div * dy, 0.0);
        for (int k = 0; k < 4; ++k) AT(fy, k, gg, i) += av * (AT(U, k, gg - 1, i) - AT(U, k, gg, i));
      }
  }

  /* 8. conservative update (Eq. 5); with gravity, the time-centred sources of §3.2's Euler equations:
   *    (rho v) += dt g (rho^n + rho^{n+1}) / 2, then (rho E) += dt g ((rho v)^n + (rho v)^{n+1}) / 2 */
  {
    const double sx = dt / dx, sy = dt / dy;
#pragma omp parallel for
    for (int j = ng; j < ng + ny; ++j)
      for (int i = ng; i < ng + nx; ++i) {
        const double rho_n = AT(U, 0, j, i), my_n = AT(U, 2, j, i);
        for (int k = 0; k < 4; ++k)
          AT(U, k, j, i) = AT(U, k, j, i) + (sx * (AT(fx, k, j, i) - AT(fx, k, j, i + 1)) +
                                             sy * (AT(fy, k, j, i) - AT(fy, k, j + 1, i)));
        if (p->grav != 0.0) {
          AT(U, 2, j, i) = AT(U, 2, j, i) + hdtg * (rho_n + AT(U, 0, j, i));
          AT(U, 3, j, i) = AT(U, 3, j, i) + hdtg * (my_n + AT(U, 2, j, i));
        }
      }
  }
  (void)g;
  if (st) {
    st->riemann_solves += n_solves;
    st->riemann_iters += n_iters;
    st->riemann_nonconv += n_nonconv;
    if (max_iters > st->riemann_maxiters_seen) st->riemann_maxiters_seen = max_iters;
  }

done:
  free(q); free(xi); free(dqx); free(dqy); free(qxl); free(qxr); free(qyl); free(qyr);
  free(fxh); free(fyh); free(fx); free(fy);
  return err;
}

/* ------------------------------------------------------------------------------------------------ */
/* Dimensionally split variant (§3.1: the fluxes of a directional update are built without knowledge of
 * the transverse flow, each directional update acts on the state left by the previous one, and the order
 * of the directions alternates from step to step for second-order accuracy).  One sweep along dir
 * (0: x, 1: y) applies the one-dimensional piecewise-linear Godunov method of §3.2 to every interior line:
 *   1. primitives of the line's cells, in the face frame (rho, u_normal, u_transverse, p);
 *   2. flattening along the line only: xi_m = min(chi_m, chi_{m-s}), s = sign(p_{m+1} - p_{m-1});
 *   3. limited slopes along the line, times xi;
 *   4. characteristic tracing (Eq. 13) to the two half-step face states of each cell, sigma = dt / h;
 *   5. Riemann solves at the interior faces of the line;
 *   6. artificial viscosity with the divergence along the line, (u_m - u_{m-1}) / h;
 *   7. conservative update of the line's interior cells, U += sigma (F_{m-1/2} - F_{m+1/2}).
 * Gravity (along y): as in the unsplit step, every traced state's v gains dt g / 2 (transverse in the x
 * sweep, normal in the y sweep); the time-centred sources (rho v) += dt g (rho^n + rho^{n+1}) / 2,
 * (rho E) += dt g ((rho v)^n + (rho v)^{n+1}) / 2 are added once per step, by the y sweep, with n the state
 * the y sweep starts from.
 * The state must be ghost-filled on entry.  Lines are independent; each keeps its own work arrays. */
static int sweep(const oracle_params* p, double* U, double dt, int dir, oracle_stats* st) {
  const int ng = p->ng, nx = p->nx, ny = p->ny, NX = nx + 2 * ng, NY = ny + 2 * ng;
  const size_t plane = (size_t)NX * NY;
  const double h = dir == 0 ? (p->xmax - p->xmin) / nx : (p->ymax - p->ymin) / ny;
  const int n = dir == 0 ? nx : ny;         /* interior cells along a line */
  const int N = n + 2 * ng;                 /* cells along a line, ghosts included */
  const int nlines = dir == 0 ? ny : nx;    /* interior lines */
  const size_t sa = dir == 0 ? 1 : (size_t)NX;  /* stride along the line */
  const size_t sl = dir == 0 ? (size_t)NX : 1;  /* stride between lines */
  const int kn = dir == 0 ? 1 : 2, kt = dir == 0 ? 2 : 1;  /* normal and transverse momentum components */
  const double sigma = dt / h;
  const double hdtg = 0.5 * dt * p->grav;
  long long n_solves = 0, n_iters = 0, n_nonconv = 0;
  int max_iters = 0, err = 0;

#pragma omp parallel for reduction(+ : n_solves, n_iters, n_nonconv) reduction(max : max_iters) reduction(| : err)
  for (int l = 0; l < nlines; ++l) {
    const size_t base = (size_t)(ng + l) * sl;  /* cell m of the line is base + m * sa */
    double* w = calloc((size_t)N * 19 + 4 * ((size_t)N + 1), sizeof(double));
    if (!w) {
      err |= 2;
      continue;
    }
    double* q = w;                /* [4][N] primitives, face frame */
    double* chi = q + 4 * N;      /* [N] */
    double* xi = chi + N;         /* [N] */
    double* dq = xi + N;          /* [4][N] limited slopes */
    double* ql = dq + 4 * N;      /* [4][N] left state at m+1/2 of cell m */
    double* qr = ql + 4 * N;      /* [4][N] right state at m-1/2 of cell m */
    double* G = qr + 4 * N;       /* [4][N+1] flux at face f (between cells f-1 and f), conserved order */
#define C(k, m) U[(size_t)(k) * plane + base + (size_t)(m) * sa]
    /* 1. primitives */
    for (int m = 0; m < N; ++m) {
      double Uc[4] = {C(0, m), C(1, m), C(2, m), C(3, m)}, qc[4];
      oracle_cons_to_prim(p, Uc, qc);
      q[0 * N + m] = qc[0];
      q[1 * N + m] = qc[kn];
      q[2 * N + m] = qc[kt];
      q[3 * N + m] = qc[3];
    }
    /* 2. flattening along the line */
    for (int m = 0; m < N; ++m) {
      chi[m] = 1.0;
      xi[m] = 1.0;
    }
    if (p->use_flattening) {
      for (int m = 2; m < N - 2; ++m)
        chi[m] = oracle_flatten_chi(q[3 * N + m - 2], q[3 * N + m - 1], q[3 * N + m + 1], q[3 * N + m + 2],
                                    q[1 * N + m - 1], q[1 * N + m + 1], p->small_pres);
      for (int m = 3; m < N - 3; ++m) {
        int s = (q[3 * N + m + 1] - q[3 * N + m - 1]) >= 0.0 ? 1 : -1;
        xi[m] = fmin(chi[m], chi[m - s]);
      }
    }
    /* 3. slopes */
    for (int k = 0; k < 4; ++k)
      for (int m = 2; m < N - 2; ++m)
        dq[k * N + m] = xi[m] * oracle_slope(p->limiter, q[k * N + m - 2], q[k * N + m - 1], q[k * N + m],
                                             q[k * N + m + 1], q[k * N + m + 2]);
    /* 4. tracing */
    for (int m = 3; m < N - 3; ++m) {
      double qc[4], d4[4], a[4], b[4], a5[4][5];
      for (int k = 0; k < 4; ++k) {
        qc[k] = q[k * N + m];
        d4[k] = dq[k * N + m];
        for (int t = 0; t < 5; ++t) a5[k][t] = q[k * N + m - 2 + t];
      }
      trace_cell(p, sigma, qc, d4, (const double(*)[5])a5, xi[m], a, b);
      if (p->grav != 0.0) { /* half-step gravity on v: transverse in the x sweep, normal in the y sweep */
        const int kv = dir == 0 ? 2 : 1;
        a[kv] = a[kv] + hdtg;
        b[kv] = b[kv] + hdtg;
      }
      for (int k = 0; k < 4; ++k) {
        ql[k * N + m] = a[k];
        qr[k * N + m] = b[k];
      }
    }
    /* 5.-6. Riemann solves and artificial viscosity at the faces f in [ng, ng + n] */
    for (int f = ng; f <= ng + n; ++f) {
      double a[4], b[4], F[4];
      for (int k = 0; k < 4; ++k) {
        a[k] = ql[k * N + f - 1];
        b[k] = qr[k * N + f];
      }
      int it;
      int ok = face_flux(p, a, b, F, &it);
      n_solves++;
      n_iters += it;
      if (!ok) n_nonconv++;
      if (it > max_iters) max_iters = it;
      double Gf[4];
      Gf[0] = F[0];
      Gf[kn] = F[1];
      Gf[kt] = F[2];
      Gf[3] = F[3];
      if (p->cvisc > 0.0) {
        double div = (q[1 * N + f] - q[1 * N + f - 1]) / h;
        double av = p->cvisc * fmax(-div * h, 0.0);
        for (int k = 0; k < 4; ++k) Gf[k] += av * (C(k, f - 1) - C(k, f));
      }
      for (int k = 0; k < 4; ++k) G[k * (N + 1) + f] = Gf[k];
    }
    /* 7. update; the y sweep adds the time-centred gravity sources as the unsplit step does */
    for (int m = ng; m < ng + n; ++m) {
      const double rho_n = C(0, m), my_n = C(2, m);
      for (int k = 0; k < 4; ++k) C(k, m) = C(k, m) + sigma * (G[k * (N + 1) + m] - G[k * (N + 1) + m + 1]);
      if (dir == 1 && p->grav != 0.0) {
        C(2, m) = C(2, m) + hdtg * (rho_n + C(0, m));
        C(3, m) = C(3, m) + hdtg * (my_n + C(2, m));
      }
    }
#undef C
    free(w);
  }
  if (st) {
    st->riemann_solves += n_solves;
    st->riemann_iters += n_iters;
    st->riemann_nonconv += n_nonconv;
    if (max_iters > st->riemann_maxiters_seen) st->riemann_maxiters_seen = max_iters;
  }
  return err;
}

int oracle_step_split(const oracle_params* p, double* U, double dt, int first_dir, oracle_stats* st) {
  if (!params_ok(p) || !U || !(dt >= 0.0) || (first_dir != 0 && first_dir != 1)) return 1;
  int err = sweep(p, U, dt, first_dir, st);
  if (!err) err = oracle_fill_ghost(p, U);
  if (!err) err = sweep(p, U, dt, 1 - first_dir, st);
  return err;
}
