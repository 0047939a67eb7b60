// Device-side building blocks of the unsplit CTU step (paper §3.2; CTU construction of §3.1), templated
// on the arithmetic type R (double for the FP64 path, float for the FP32 path).
//
// Each function states the passage it implements.  For R = double the operations are written in the same
// association order as a plain left-to-right evaluation of the formulas, so results differ from a
// reference evaluation only by FMA contraction.  For R = float, divisions and square roots use the fast
// hardware approximations (a few ulp), and the internal-energy recovery is done in double where the
// kinetic energy is within 0.1% of the total energy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace hydro {

// Parameters as the kernels see them (plain values, passed by value).
struct KParams {
  int nx, ny, ng, pitch;  // interior size, ghost width, row pitch (elements)
  int NX, NY;             // padded extents nx + 2 ng, ny + 2 ng
  int bc[4];              // xlo, xhi, ylo, yhi: 0 outflow, 1 periodic
  double dx, dy;
  double gamma, gm1, g1;  // gamma, gamma - 1, (gamma + 1)/(2 gamma)
  double cfl;
  int limiter, use_flattening;
  double cvisc;
  int riemann_maxiter;
  double riemann_tol;
  double small_dens, small_pres;
};

// Scratch words the kernels share with the host, one block per context (device memory).
struct DevScratch {
  unsigned long long dt_min_bits;  // running min of the per-cell CFL time (double bits, all positive)
  unsigned int dt_blocks_done;     // last-block detection of the dt reduction
  unsigned int tot_blocks_done;    // last-block detection of the totals reduction
  double dt;                       // last reduced (and clamped) time step
  double t;                        // simulated time (device driver loop)
  long long nsteps;                // steps taken
  unsigned int status;             // bit flags, see STATUS_*
  unsigned int pad_;
  unsigned long long stats[3];     // riemann solves, iterations, unconverged solves
  double totals[4];                // last conserved totals
};

enum : unsigned int {
  STATUS_NONFINITE = 1u,
  STATUS_NEGATIVE = 2u,
  STATUS_NONCONV = 4u,
};

// ---------------------------------------------------------------------------------------------------
// arithmetic helpers per precision
template <typename R>
struct M;

template <>
struct M<double> {
  static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
  static __device__ __forceinline__ double dv(double a, double b) { return a / b; }
  static __device__ __forceinline__ double mn(double a, double b) { return fmin(a, b); }
  static __device__ __forceinline__ double mx(double a, double b) { return fmax(a, b); }
  static __device__ __forceinline__ double ab(double a) { return fabs(a); }
};

template <>
struct M<float> {
  // arguments are strictly positive wherever sq is used (floored pressures and densities)
  static __device__ __forceinline__ float sq(float x) { return x * rsqrtf(x); }
  static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float mn(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float mx(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float ab(float a) { return fabsf(a); }
};

// Per-precision copies of the scalar parameters used in the stencil.
template <typename R>
struct SP {
  R gamma, gm1, g1, small_dens, small_pres, tol, cvisc;
  int maxiter, limiter, flatten;
  __device__ __forceinline__ void load(const KParams& P) {
    gamma = (R)P.gamma;
    gm1 = (R)P.gm1;
    g1 = (R)P.g1;
    small_dens = (R)P.small_dens;
    small_pres = (R)P.small_pres;
    tol = (R)P.riemann_tol;
    cvisc = (R)P.cvisc;
    maxiter = P.riemann_maxiter;
    limiter = P.limiter;
    flatten = P.use_flattening;
  }
};

// ---------------------------------------------------------------------------------------------------
// EOS (Eqs. 11-12): conserved (rho, mx, my, E) -> primitive (rho, u, v, p), floors on the copy.
template <typename R>
__device__ __forceinline__ void cons_to_prim(const SP<R>& s, R U0, R U1, R U2, R U3, R& rho, R& u, R& v, R& p) {
  rho = U0 < s.small_dens ? s.small_dens : U0;
  u = M<R>::dv(U1, rho);
  v = M<R>::dv(U2, rho);
  R ke = (R)0.5 * rho * (u * u + v * v);
  if constexpr (std::is_same<R, float>::value) {
    if (ke > 0.999f * U3) {
      // kinetic energy within 0.1% of the total: recover e = E - rho |u|^2 / 2 in double
      double rd = (double)rho, ud = (double)U1 / rd, vd = (double)U2 / rd;
      double ked = 0.5 * rd * (ud * ud + vd * vd);
      p = (float)(((double)s.gm1) * ((double)U3 - ked));
    } else {
      p = s.gm1 * (U3 - ke);
    }
  } else {
    p = s.gm1 * (U3 - ke);
  }
  p = p < s.small_pres ? s.small_pres : p;
}

// primitive (rho, u, v, p) -> conserved
template <typename R>
__device__ __forceinline__ void prim_to_cons(const SP<R>& s, R rho, R u, R v, R p, R& U0, R& U1, R& U2, R& U3) {
  U0 = rho;
  U1 = rho * u;
  U2 = rho * v;
  U3 = M<R>::dv(p, s.gm1) + (R)0.5 * rho * (u * u + v * v);
}

// ---------------------------------------------------------------------------------------------------
// Limited slopes (§3.1, fourth-order MC limiter of Colella 1985).
template <typename R>
__device__ __forceinline__ R mc2(R qm, R q0, R qp) {
  R dl = q0 - qm, dr = qp - q0, dc = (R)0.5 * (qp - qm);
  if (!(dl * dr > (R)0)) return (R)0;
  R dlim = (R)2 * M<R>::mn(M<R>::ab(dl), M<R>::ab(dr));
  R mag = M<R>::mn(M<R>::ab(dc), dlim);
  return dc >= (R)0 ? mag : -mag;
}

template <typename R>
__device__ __forceinline__ R slope(int limiter, R qm2, R qm1, R q0, R qp1, R qp2) {
  if (limiter == 0) return (R)0;
  if (limiter == 1) return mc2(qm1, q0, qp1);
  R dl = q0 - qm1, dr = qp1 - q0, dc = (R)0.5 * (qp1 - qm1);
  if (!(dl * dr > (R)0)) return (R)0;
  R dlim = (R)2 * M<R>::mn(M<R>::ab(dl), M<R>::ab(dr));
  R d4 = ((R)4 / (R)3) * dc - ((R)1 / (R)6) * (mc2(q0, qp1, qp2) + mc2(qm2, qm1, q0));
  R mag = M<R>::mn(M<R>::ab(d4), dlim);
  return d4 >= (R)0 ? mag : -mag;
}

// Flattening shock detector on one line (§3.2, Colella 1990): chi in [0, 1].
template <typename R>
__device__ __forceinline__ R flatten_chi(R pm2, R pm1, R pp1, R pp2, R um1, R up1, R small_pres) {
  const R z0 = (R)0.75, z1 = (R)0.85, delta = (R)0.33;
  R dp1 = pp1 - pm1;
  R dp2 = pp2 - pm2;
  R z = M<R>::dv(M<R>::ab(dp1), M<R>::mx(M<R>::ab(dp2), small_pres));
  bool compress = (um1 - up1) > (R)0;
  bool jump = M<R>::ab(dp1) > delta * M<R>::mn(pp1, pm1);
  if (!(compress && jump)) return (R)1;
  R chi = (R)1 - M<R>::dv(z - z0, z1 - z0);
  chi = chi < (R)0 ? (R)0 : chi;
  chi = chi > (R)1 ? (R)1 : chi;
  return chi;
}

// ---------------------------------------------------------------------------------------------------
// Characteristic tracing (§3.2, Eq. 13) in the face frame q = (rho, un, ut, p), slope dq, sigma = dt/dx.
// Eigenvalues (un - c, un, un, un + c) with the explicit left/right eigenvectors
//   l1 = (0, -rho/2c, 0, 1/2c^2), l2 = (1, 0, 0, -1/c^2), l3 = (0, 0, 1, 0), l4 = (0, rho/2c, 0, 1/2c^2)
//   r1 = (1, -c/rho, 0, c^2),     r2 = (1, 0, 0, 0),      r3 = (0, 0, 1, 0), r4 = (1, c/rho, 0, c^2).
// Left state at i+1/2: q + (1 - sigma lam4) dq/2 + sum over lam_nu >= 0 of (sigma/2)(lam4 - lam_nu) beta_nu r_nu.
// Right state at i-1/2: q - (1 + sigma lam1) dq/2 + sum over lam_nu <= 0 of (sigma/2)(lam1 - lam_nu) beta_nu r_nu.
// Only the non-zero eigenvector entries are multiplied out.
template <typename R>
__device__ __forceinline__ void trace(const SP<R>& s, R sigma, const R q[4], const R dq[4], R qL[4], R qR[4]) {
  const R rho = q[0], un = q[1], pres = q[3];
  const R c = M<R>::sq(M<R>::dv(s.gamma * pres, rho));
  const R lam1 = un - c, lam2 = un, lam4 = un + c;
  const R c2 = c * c;
  const R roc = M<R>::dv((R)0.5 * rho, c);  // rho / 2c
  const R ic2h = M<R>::dv((R)0.5, c2);      // 1 / 2c^2
  const R ic2 = M<R>::dv((R)1, c2);         // 1 / c^2
  const R cor = M<R>::dv(c, rho);           // c / rho
  const R b1 = -roc * dq[1] + ic2h * dq[3];
  const R b2 = dq[0] + (-ic2) * dq[3];
  const R b3 = dq[2];
  const R b4 = roc * dq[1] + ic2h * dq[3];
  const R hs = (R)0.5 * sigma;
  // left state: reference with lam4, waves moving right add (sigma/2)(lam4 - lam) beta r
  R aL = (R)0.5 * ((R)1 - sigma * lam4);
  R l0 = q[0] + aL * dq[0], l1 = q[1] + aL * dq[1], l2 = q[2] + aL * dq[2], l3 = q[3] + aL * dq[3];
  if (lam1 >= (R)0) {
    R w = hs * (lam4 - lam1) * b1;
    l0 += w;
    l1 += w * (-cor);
    l3 += w * c2;
  }
  if (lam2 >= (R)0) {
    R w2 = hs * (lam4 - lam2) * b2;
    l0 += w2;
    R w3 = hs * (lam4 - lam2) * b3;
    l2 += w3;
  }
  // right state: reference with lam1, waves moving left add (sigma/2)(lam1 - lam) beta r
  R aR = (R)0.5 * ((R)1 + sigma * lam1);
  R r0 = q[0] - aR * dq[0], r1 = q[1] - aR * dq[1], r2 = q[2] - aR * dq[2], r3 = q[3] - aR * dq[3];
  if (lam2 <= (R)0) {
    R w2 = hs * (lam1 - lam2) * b2;
    r0 += w2;
    R w3 = hs * (lam1 - lam2) * b3;
    r2 += w3;
  }
  if (lam4 <= (R)0) {
    R w = hs * (lam1 - lam4) * b4;
    r0 += w;
    r1 += w * cor;
    r3 += w * c2;
  }
  l0 = l0 < s.small_dens ? s.small_dens : l0;
  r0 = r0 < s.small_dens ? s.small_dens : r0;
  l3 = l3 < s.small_pres ? s.small_pres : l3;
  r3 = r3 < s.small_pres ? s.small_pres : r3;
  qL[0] = l0; qL[1] = l1; qL[2] = l2; qL[3] = l3;
  qR[0] = r0; qR[1] = r1; qR[2] = r2; qR[3] = r3;
}

// ---------------------------------------------------------------------------------------------------
// Two-shock Riemann solver (§3.2, "the Riemann solver described in almgren:2010").
// Face frame: (rho, un, ut, p).  Newton iteration on u*_L(p) = u*_R(p) with the shock mass fluxes
// W_K = C_K sqrt(1 + (gamma+1)/(2 gamma) (p/p_K - 1)), C_K = sqrt(gamma p_K rho_K), slopes
// Z_K = 2 W_K^3 / (W_K^2 + C_K^2); acoustic start unless guess > 0.  Sampling at x/t = 0 from the upwind
// side of the contact, Hugoniot star density, shock or linearly interpolated fan.  Returns the flux
// (mass, normal momentum, transverse momentum, energy); iters/conv report the iteration.
template <typename R>
__device__ __forceinline__ void riemann(const SP<R>& s, const R qL[4], const R qR[4], R guess, R F[4], int& iters,
                                        bool& conv) {
  const R g = s.gamma, g1 = s.g1;
  const R rl = qL[0], ul = qL[1], vl = qL[2], pl = qL[3];
  const R rr = qR[0], ur = qR[1], vr = qR[2], pr = qR[3];
  const R cl = M<R>::sq(g * pl * rl);
  const R cr = M<R>::sq(g * pr * rr);
  R pst = guess > (R)0 ? guess : M<R>::dv(cr * pl + cl * pr + cl * cr * (ul - ur), cl + cr);
  pst = pst < s.small_pres ? s.small_pres : pst;
  int it = 0;
  bool ok = false;
  while (it < s.maxiter) {
    R wl = cl * M<R>::sq((R)1 + g1 * (M<R>::dv(pst, pl) - (R)1));
    R wr = cr * M<R>::sq((R)1 + g1 * (M<R>::dv(pst, pr) - (R)1));
    R usl = ul - M<R>::dv(pst - pl, wl);
    R usr = ur + M<R>::dv(pst - pr, wr);
    R zl = M<R>::dv((R)2 * wl * wl * wl, wl * wl + cl * cl);
    R zr = M<R>::dv((R)2 * wr * wr * wr, wr * wr + cr * cr);
    R pnew = pst - M<R>::dv(zl * zr * (usr - usl), zl + zr);
    pnew = pnew < s.small_pres ? s.small_pres : pnew;
    R dp = M<R>::ab(pnew - pst);
    pst = pnew;
    ++it;
    if (dp <= s.tol * pst) {
      ok = true;
      break;
    }
  }
  iters = it;
  conv = ok;
  const R wl = cl * M<R>::sq((R)1 + g1 * (M<R>::dv(pst, pl) - (R)1));
  const R wr = cr * M<R>::sq((R)1 + g1 * (M<R>::dv(pst, pr) - (R)1));
  const R ust = M<R>::dv((wl * ul + wr * ur) + (pl - pr), wl + wr);

  R fr, fu, fv, fp;
  if (ust == (R)0) {
    fr = (R)0.5 * (rl + rr);
    fu = (R)0;
    fv = (R)0.5 * (vl + vr);
    fp = pst;
  } else {
    const bool left = ust > (R)0;
    const R sgn = left ? (R)1 : (R)-1;
    const R ro = left ? rl : rr, uo = left ? ul : ur, vo = left ? vl : vr, po = left ? pl : pr;
    const R wo = left ? wl : wr;
    const R rst = M<R>::dv((R)1, M<R>::dv((R)1, ro) - M<R>::dv(pst - po, wo * wo));
    fv = vo;
    if (pst > po) {
      const R S = uo - sgn * M<R>::dv(wo, ro);
      if (sgn * S >= (R)0) {
        fr = ro; fu = uo; fp = po;
      } else {
        fr = rst; fu = ust; fp = pst;
      }
    } else {
      const R co = M<R>::sq(M<R>::dv(g * po, ro));
      const R cst = M<R>::sq(M<R>::dv(g * pst, rst));
      const R SH = uo - sgn * co;
      const R ST = ust - sgn * cst;
      if (sgn * SH >= (R)0) {
        fr = ro; fu = uo; fp = po;
      } else if (sgn * ST <= (R)0) {
        fr = rst; fu = ust; fp = pst;
      } else {
        const R frac = M<R>::dv(SH, SH - ST);
        fr = ro + frac * (rst - ro);
        fu = uo + frac * (ust - uo);
        fp = po + frac * (pst - po);
      }
    }
  }
  const R rhoE = M<R>::dv(fp, s.gm1) + (R)0.5 * fr * (fu * fu + fv * fv);
  F[0] = fr * fu;
  F[1] = fr * fu * fu + fp;
  F[2] = fr * fu * fv;
  F[3] = fu * (rhoE + fp);
}

}  // namespace hydro
