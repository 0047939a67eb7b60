// Device-side building blocks of the unsplit CTU step (paper §3.2; CTU construction of §3.1), templated
// on the arithmetic type R (double for the FP64 path, float for the FP32 path).
//
// Each function states the passage it implements.  For R = double the operations follow the formulas
// left to right, so results differ from a plain evaluation only by FMA contraction.  For R = float the
// same quantities are formed from hardware reciprocal and reciprocal-square-root approximations
// (a few ulp), sharing one reciprocal wherever a formula divides twice by the same value, and the
// internal energy is recovered in double where the kinetic energy is within 0.1% of the total energy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace hydro {

// Parameters as the kernels see them (plain values, passed by value).
struct KParams {
  int nx, ny, ng, pitch;  // interior size, ghost width, row pitch (elements)
  int NX, NY;             // padded extents nx + 2 ng, ny + 2 ng
  int bc[4];              // xlo, xhi, ylo, yhi: 0 outflow, 1 periodic, 2 reflect, 3 hydrostatic
  double dx, dy;
  double gamma, gm1, g1;  // gamma, gamma - 1, (gamma + 1)/(2 gamma)
  double cfl;
  int limiter, use_flattening;
  double cvisc;
  int riemann_maxiter;
  double riemann_tol;
  double small_dens, small_pres;
  // float copies (filled on the host) so the FP32 kernels never convert from double
  float gamma_f, gm1_f, igm1_f, g1_f, small_dens_f, small_pres_f, tol_f, cvisc_f, dx_f, dy_f, idx_f, idy_f;
  // failure-path test of the bounded TMA wait (0, 0 in normal operation): tma_test_drop = 1 issues no tile
  // copy (the tile's mbarrier then waits for bytes that never come); tma_polls != 0 replaces the poll budget
  int tma_test_drop;
  unsigned int tma_polls;
  double grav;  // gravitational acceleration along y
  float grav_f;
  int use_grav;  // grav != 0: the step applies the gravity terms
  int riemann_solver;  // 0 two-shock iteration, 1 HLLC
  int reconstruction;  // 0 piecewise linear, 1 piecewise parabolic
  int bc_general;      // some side is reflecting or hydrostatic (ghost values are not plain copies)
  float rec_f;         // FP32: kinetic-energy fraction above which the pressure is recomputed in double
};

// Time-step dependent factors of one CTU step, computed once in double (host, or the last block of
// the dt reduction) so the kernels do no double division: sig = dt/dx, h = dt/(2dx), as in Eqs. 3-5.
struct StepScalars {
  double dt, sigx, sigy, hx, hy;
  double hdtg;  // dt g / 2: half-step gravity of the traced v, and the factor of the time-centred sources
  float sigx_f, sigy_f, hx_f, hy_f, hdtg_f;
};

__host__ __device__ inline StepScalars make_step_scalars(double dt, double dx, double dy, double grav) {
  StepScalars s;
  s.dt = dt;
  s.sigx = dt / dx;
  s.sigy = dt / dy;
  s.hx = 0.5 * dt / dx;
  s.hy = 0.5 * dt / dy;
  s.hdtg = 0.5 * dt * grav;
  s.sigx_f = (float)s.sigx;
  s.sigy_f = (float)s.sigy;
  s.hx_f = (float)s.hx;
  s.hy_f = (float)s.hy;
  s.hdtg_f = (float)s.hdtg;
  return s;
}

// Scratch words the kernels share with the host, one block per context (device memory).
struct DevScratch {
  unsigned long long dt_min_bits;  // running min of the per-cell CFL time (double bits, all positive)
  unsigned int dt_blocks_done;     // last-block detection of the dt reduction
  unsigned int tot_blocks_done;    // last-block detection of the totals reduction
  double dt;                       // last reduced (and clamped) time step
  StepScalars sc;                  // factors of that time step
  double t;                        // simulated time (device driver loop)
  long long nsteps;                // steps taken
  unsigned int status;             // bit flags, see STATUS_*
  unsigned int pad_;
  unsigned long long stats[3];     // riemann solves, iterations, unconverged solves
  double totals[4];                // last conserved totals
  // fused steps: factors of the current and of the next step (alternating), next-dt accumulator and
  // last-block detection of the step kernel
  StepScalars scf[2];
  unsigned long long dtn_min_bits;
  unsigned int step_blocks_done;
  unsigned int pad2_;
};

enum : unsigned int {
  STATUS_NONFINITE = 1u,
  STATUS_NEGATIVE = 2u,
  STATUS_NONCONV = 4u,
  STATUS_TIMEOUT = 8u,  // a bounded device-side wait ran out (a tile's TMA copy did not land)
  // the second, equally bounded wait of such a tile ran out too: the copy may still have been in flight when
  // the block left, and could then have landed in shared memory a later block uses
  STATUS_TIMEOUT_INFLIGHT = 16u,
};

template <typename R>
constexpr bool is_f32() {
  return std::is_same<R, float>::value;
}

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
  // arguments are strictly positive wherever sq / rs are used (floored pressures and densities)
  static __device__ __forceinline__ float sq(float x);
  static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
  static __device__ __forceinline__ float mn(float a, float b) { return fminf(a, b); }
  static __device__ __forceinline__ float mx(float a, float b) { return fmaxf(a, b); }
  static __device__ __forceinline__ float ab(float a) { return fabsf(a); }
};

// approximate reciprocal (MUFU.RCP) for the FP32 path
__device__ __forceinline__ float rcpa(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// approximate reciprocal square root, subnormals flushed (one MUFU.RSQ, no subnormal fix-up): every
// argument in the FP32 path is a product of floored densities and pressures (>= 1e-30), never subnormal
__device__ __forceinline__ float rsqa(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float M<float>::sq(float x) { return x * rsqa(x); }

// Packed FP32x2 arithmetic (sm_100 and later): one instruction applies the same operation to two values,
// each rounded as the scalar operation rounds it.  The FP32 path uses it wherever two components of a state,
// or the two sides of a face, go through the same arithmetic; it halves the issue slots of that arithmetic.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\tsub.rn.f32x2 z, x, y;\n\t"
      "mov.b64 {%0, %1}, z;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// Four-component helpers: d = a - b and y = y + c x, in the FP32 path as two packed operations each; the FP64
// path keeps one scalar operation per component in the same order.
template <typename R>
__device__ __forceinline__ void sub4(const R a[4], const R b[4], R d[4]) {
  if constexpr (is_f32<R>()) {
    const float2 lo = sub2(f2(a[0], a[1]), f2(b[0], b[1])), hi = sub2(f2(a[2], a[3]), f2(b[2], b[3]));
    d[0] = lo.x; d[1] = lo.y; d[2] = hi.x; d[3] = hi.y;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) d[k] = a[k] - b[k];
  }
}
template <typename R>
__device__ __forceinline__ void axpy4(R c, const R x[4], R y[4]) {
  if constexpr (is_f32<R>()) {
    const float2 lo = fma2(f2(c), f2(x[0], x[1]), f2(y[0], y[1])), hi = fma2(f2(c), f2(x[2], x[3]), f2(y[2], y[3]));
    y[0] = lo.x; y[1] = lo.y; y[2] = hi.x; y[3] = hi.y;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) y[k] = y[k] + c * x[k];
  }
}

// Per-precision copies of the scalar parameters used in the stencil.
template <typename R>
struct SP {
  R gamma, gm1, igm1, g1, small_dens, small_pres, tol, cvisc, dx, dy, idx, idy;
  R rec;  // FP32: energy-recovery threshold (kinetic over total energy)
  int maxiter, limiter, flatten;
  __device__ __forceinline__ void load(const KParams& P) {
    if constexpr (is_f32<R>()) {
      gamma = P.gamma_f; gm1 = P.gm1_f; igm1 = P.igm1_f; g1 = P.g1_f; small_dens = P.small_dens_f;
      small_pres = P.small_pres_f; tol = P.tol_f; cvisc = P.cvisc_f; dx = P.dx_f; dy = P.dy_f;
      idx = P.idx_f; idy = P.idy_f; rec = P.rec_f;
    } else {
      gamma = P.gamma; gm1 = P.gm1; igm1 = 0.0; g1 = P.g1; small_dens = P.small_dens; small_pres = P.small_pres;
      tol = P.riemann_tol; cvisc = P.cvisc; dx = P.dx; dy = P.dy; idx = 0.0; idy = 0.0; rec = 0.0;
    }
    maxiter = P.riemann_maxiter;
    limiter = P.limiter;
    flatten = P.use_flattening;
  }
};

template <typename R>
__device__ __forceinline__ bool finite4(R a, R b, R c, R d) {
  return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
}

// Ghost-cell source index along one axis (paper §2, CellCenterData2d ghost filling; Fig. 1): outflow and
// hydrostatic clamp to the nearest interior index, periodic wraps, reflect mirrors about the wall.
__device__ __forceinline__ int map_index(int i, int ng, int n, int lo_bc, int hi_bc) {
  if (i < ng) return lo_bc == 1 ? i + n : lo_bc == 2 ? 2 * ng - 1 - i : ng;
  if (i >= ng + n) return hi_bc == 1 ? i - n : hi_bc == 2 ? 2 * (ng + n) - 1 - i : ng + n - 1;
  return i;
}

// Boundary condition that fills padded index i along one axis (-1 inside the domain).
__device__ __forceinline__ int ghost_bc(int i, int ng, int n, int lo_bc, int hi_bc) {
  return i < ng ? lo_bc : i >= ng + n ? hi_bc : -1;
}

// Value of the padded cell (i, j) as the ghost fill defines it (an interior cell: its stored value).  The
// source is the interior cell (map_x(i), map_y(j)); a reflecting side negates the momentum normal to it (mx
// across x walls, my across y walls).  A hydrostatic y side keeps the edge row's density and momenta and
// integrates its pressure with dp/dy = rho g at constant rho: p = p_edge + rho g (y - y_edge),
// E = p/(gamma - 1) + kinetic.  Every source is an interior cell, so one pass fills edges and corners; a
// corner combines its x side's mapping with its y side's, as filling the x sides of the interior rows and
// then the y bands over the full width does.  The hydrostatic energy is computed in double with rounded
// operations only, in the order of the formula, for every state precision.
template <typename R>
__device__ __forceinline__ void bc_cell(const KParams& P, const R* U, int i, int j, size_t plane, R v[4]) {
  const int si = map_index(i, P.ng, P.nx, P.bc[0], P.bc[1]);
  const int sj = map_index(j, P.ng, P.ny, P.bc[2], P.bc[3]);
  const size_t s = (size_t)sj * P.pitch + si;
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = U[s + k * plane];
  if (ghost_bc(i, P.ng, P.nx, P.bc[0], P.bc[1]) == 2) v[1] = -v[1];
  const int ybc = ghost_bc(j, P.ng, P.ny, P.bc[2], P.bc[3]);
  if (ybc == 2) {
    v[2] = -v[2];
  } else if (ybc == 3) {
    const double rho = (double)v[0], mx = (double)v[1], my = (double)v[2];
    const double ke = __ddiv_rn(__dmul_rn(0.5, __dadd_rn(__dmul_rn(mx, mx), __dmul_rn(my, my))), rho);
    const double pe = __dmul_rn(P.gm1, __dsub_rn((double)v[3], ke));
    const double pg = __dadd_rn(pe, __dmul_rn(__dmul_rn(rho, P.grav), __dmul_rn((double)(j - sj), P.dy)));
    v[3] = (R)__dadd_rn(__ddiv_rn(pg, P.gm1), ke);
  }
}

// bc_cell of a padded index clamped into the padded array (a ragged tile's halo can reach past it).  Not
// inlined: only boundary tiles of problems with reflecting or hydrostatic sides call it from the fused step,
// whose register allocation then stays that of the plain path.
template <typename R>
__device__ __noinline__ void bc_cell_clamped(const KParams& P, const R* U, int gi, int gj, size_t plane, R v[4]) {
  gi = gi < 0 ? 0 : (gi >= P.NX ? P.NX - 1 : gi);
  gj = gj < 0 ? 0 : (gj >= P.NY ? P.NY - 1 : gj);
  bc_cell(P, U, gi, gj, plane, v);
}

// Writes the ghost cell (i, j) with its boundary value (bc_cell).
template <typename R>
__device__ __forceinline__ void fill_ghost_cell(const KParams& P, R* __restrict__ U, int i, int j, size_t plane) {
  R v[4];
  bc_cell(P, U, i, j, plane, v);
  const size_t d = (size_t)j * P.pitch + i;
#pragma unroll
  for (int k = 0; k < 4; ++k) U[d + k * plane] = v[k];
}

// ---------------------------------------------------------------------------------------------------
// EOS (Eqs. 11-12): conserved (rho, mx, my, E) -> primitive (rho, u, v, p), floors on the copy.
template <typename R>
__device__ __forceinline__ void cons_to_prim(const SP<R>& s, R U0, R U1, R U2, R U3, R& rho, R& u, R& v, R& p) {
  rho = U0 < s.small_dens ? s.small_dens : U0;
  if constexpr (is_f32<R>()) {
    const float ir = rcpa(rho);
    const float2 uv = mul2(f2(U1, U2), f2(ir));
    u = uv.x;
    v = uv.y;
    const float ke = 0.5f * rho * (u * u + v * v);
    if (ke > s.rec * U3) {
      // kinetic energy within 0.1% (by default) of the total: recover e = E - rho |u|^2 / 2 in double
      const double rd = (double)rho, ud = (double)U1 / rd, vd = (double)U2 / rd;
      const double ked = 0.5 * rd * (ud * ud + vd * vd);
      p = (float)(((double)s.gm1) * ((double)U3 - ked));
    } else {
      p = s.gm1 * (U3 - ke);
    }
  } else {
    u = U1 / rho;
    v = U2 / rho;
    const double ke = 0.5 * rho * (u * u + v * v);
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
  if constexpr (is_f32<R>())
    U3 = p * s.igm1 + 0.5f * rho * (u * u + v * v);
  else
    U3 = p / s.gm1 + 0.5 * rho * (u * u + v * v);
}

// Pressure of a transversely corrected FP32 face state formed in double (see correct_state): the state's
// conserved values from its traced primitives (rho, u, v, p), less h times the flux differences dF, all in
// double, and p = (gamma - 1)(E - |m|^2 / (2 rho)) from them (rho floored as in cons_to_prim).  Not inlined:
// only high-Mach states call it, and the face loops keep the registers of the plain path.
static __device__ __noinline__ float corrected_pressure_f64(float gm1, float igm1, float small_dens, float small_pres,
                                                           float rho, float u, float v, float p, float h, float dF0,
                                                           float dF1, float dF2, float dF3) {
  const double rd = (double)rho, ud = (double)u, vd = (double)v, hd = (double)h;
  const double r2 = rd - hd * (double)dF0;
  const double mx = rd * ud - hd * (double)dF1, my = rd * vd - hd * (double)dF2;
  const double E = ((double)p * (double)igm1 + 0.5 * rd * (ud * ud + vd * vd)) - hd * (double)dF3;
  const double rf = r2 < (double)small_dens ? (double)small_dens : r2;
  const float pf = (float)((double)gm1 * (E - 0.5 * (mx * mx + my * my) / rf));
  return pf < small_pres ? small_pres : pf;
}

// Transverse correction of one traced face state (§3.1 CTU, Eqs. 3-4; §3.2): its primitives (rho, u, v, p)
// go to conserved variables, lose h times the transverse flux difference dF, and come back to primitives.
// FP32: where the state's kinetic energy exceeds rec of its total energy, the corrected total energy and
// the pressure are formed in double from the float primitives and flux difference, so that the float
// round trip through E does not cancel the pressure away (high Mach).
template <typename R>
__device__ __forceinline__ void correct_state(const SP<R>& s, R rho, R u, R v, R p, const R dF[4], R h, R q[4]) {
  R U[4];
  if constexpr (is_f32<R>()) {
    // prim_to_cons, keeping the kinetic energy for the high-Mach test
    const float ke = 0.5f * rho * (u * u + v * v);
    U[0] = rho;
    U[1] = rho * u;
    U[2] = rho * v;
    U[3] = p * s.igm1 + ke;
    const bool high_mach = ke > s.rec * U[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k] = U[k] - h * dF[k];
    cons_to_prim(s, U[0], U[1], U[2], U[3], q[0], q[1], q[2], q[3]);
    if (high_mach)
      q[3] = corrected_pressure_f64(s.gm1, s.igm1, s.small_dens, s.small_pres, rho, u, v, p, h, dF[0], dF[1], dF[2],
                                    dF[3]);
  } else {
    prim_to_cons(s, rho, u, v, p, U[0], U[1], U[2], U[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k] = U[k] - h * dF[k];
    cons_to_prim(s, U[0], U[1], U[2], U[3], q[0], q[1], q[2], q[3]);
  }
}

// ---------------------------------------------------------------------------------------------------
// Limited slopes (§3.1, fourth-order MC limiter of Colella 1985).  Written without data-dependent branches
// (the zero-slope cases are selects) so that a warp whose cells disagree on the limiter's case does not
// run both paths; the arithmetic and its order are those of the definition.
template <typename R>
__device__ __forceinline__ R mc2(R qm, R q0, R qp) {
  const R dl = q0 - qm, dr = qp - q0, dc = (R)0.5 * (qp - qm);
  const R dlim = (R)2 * M<R>::mn(M<R>::ab(dl), M<R>::ab(dr));
  const R mag = M<R>::mn(M<R>::ab(dc), dlim);
  const R lim = dc >= (R)0 ? mag : -mag;
  return dl * dr > (R)0 ? lim : (R)0;
}

template <typename R>
__device__ __forceinline__ R slope(int limiter, R qm2, R qm1, R q0, R qp1, R qp2) {
  if (limiter == 0) return (R)0;  // uniform over the launch
  if (limiter == 1) return mc2(qm1, q0, qp1);
  const R dl = q0 - qm1, dr = qp1 - q0, dc = (R)0.5 * (qp1 - qm1);
  const R dlim = (R)2 * M<R>::mn(M<R>::ab(dl), M<R>::ab(dr));
  const R d4 = ((R)4 / (R)3) * dc - ((R)1 / (R)6) * (mc2(q0, qp1, qp2) + mc2(qm2, qm1, q0));
  const R mag = M<R>::mn(M<R>::ab(d4), dlim);
  const R lim = d4 >= (R)0 ? mag : -mag;
  return dl * dr > (R)0 ? lim : (R)0;
}

// The same limiter for two components at once (FP32 path): the differences and products as packed
// operations, the magnitudes, minima and sign cases per component.
__device__ __forceinline__ float2 mc2_pair(float2 qm, float2 q0, float2 qp) {
  const float2 dl = sub2(q0, qm), dr = sub2(qp, q0), dc = mul2(f2(0.5f), sub2(qp, qm));
  const float2 dlim = mul2(f2(2.0f), f2(fminf(fabsf(dl.x), fabsf(dr.x)), fminf(fabsf(dl.y), fabsf(dr.y))));
  const float2 pr = mul2(dl, dr);
  const float mx = fminf(fabsf(dc.x), dlim.x), my = fminf(fabsf(dc.y), dlim.y);
  return f2(pr.x > 0.f ? (dc.x >= 0.f ? mx : -mx) : 0.f, pr.y > 0.f ? (dc.y >= 0.f ? my : -my) : 0.f);
}

__device__ __forceinline__ float2 slope_pair(int limiter, float2 qm2, float2 qm1, float2 q0, float2 qp1, float2 qp2) {
  if (limiter == 0) return f2(0.f);  // uniform over the launch
  if (limiter == 1) return mc2_pair(qm1, q0, qp1);
  const float2 dl = sub2(q0, qm1), dr = sub2(qp1, q0), dc = mul2(f2(0.5f), sub2(qp1, qm1));
  const float2 dlim = mul2(f2(2.0f), f2(fminf(fabsf(dl.x), fabsf(dr.x)), fminf(fabsf(dl.y), fabsf(dr.y))));
  const float2 m = add2(mc2_pair(q0, qp1, qp2), mc2_pair(qm2, qm1, q0));
  const float2 d4 = fma2(f2(4.0f / 3.0f), dc, mul2(f2(-1.0f / 6.0f), m));
  const float2 pr = mul2(dl, dr);
  const float mx = fminf(fabsf(d4.x), dlim.x), my = fminf(fabsf(d4.y), dlim.y);
  return f2(pr.x > 0.f ? (d4.x >= 0.f ? mx : -mx) : 0.f, pr.y > 0.f ? (d4.y >= 0.f ? my : -my) : 0.f);
}

// Flattening shock detector on one line (§3.2, Colella 1990): chi in [0, 1].
template <typename R>
__device__ __forceinline__ R flatten_chi(R pm2, R pm1, R pp1, R pp2, R um1, R up1, R small_pres) {
  const R z0 = (R)0.75, z1 = (R)0.85, delta = (R)0.33;
  R dp1 = pp1 - pm1;
  bool compress = (um1 - up1) > (R)0;
  bool jump = M<R>::ab(dp1) > delta * M<R>::mn(pp1, pm1);
  if (!(compress && jump)) return (R)1;
  R dp2 = pp2 - pm2;
  R chi;
  if constexpr (is_f32<R>()) {
    const float z = M<float>::ab(dp1) * rcpa(M<float>::mx(M<float>::ab(dp2), small_pres));
    chi = 1.0f - (z - z0) * (1.0f / (0.85f - 0.75f));
  } else {
    R z = M<R>::ab(dp1) / M<R>::mx(M<R>::ab(dp2), small_pres);
    chi = (R)1 - (z - z0) / (z1 - z0);
  }
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
  R c, c2, roc, ic2h, ic2, cor;
  if constexpr (is_f32<R>()) {
    const float ir = rcpa(rho);
    const float x = s.gamma * pres * ir;  // c^2
    const float ic = rsqa(x);           // 1/c
    c = x * ic;
    c2 = c * c;
    roc = 0.5f * rho * ic;
    ic2 = ic * ic;
    ic2h = 0.5f * ic2;
    cor = c * ir;
  } else {
    c = sqrt(s.gamma * pres / rho);
    c2 = c * c;
    roc = (0.5 * rho) / c;
    ic2h = 0.5 / c2;
    ic2 = 1.0 / c2;
    cor = c / rho;
  }
  const R lam1 = un - c, lam2 = un, lam4 = un + c;
  const R b1 = -roc * dq[1] + ic2h * dq[3];
  const R b2 = dq[0] + (-ic2) * dq[3];
  const R b3 = dq[2];
  const R b4 = roc * dq[1] + ic2h * dq[3];
  const R hs = (R)0.5 * sigma;
  // eigenvalue gaps lam4 - lam1 = 2c and lam4 - lam2 = c: FP64 forms them as the differences the formula
  // writes (the rounding the plain C implementation does); FP32 takes c and 2c themselves, since at high
  // Mach the difference of two nearly equal speeds u + c and u - c loses ~Mach ulps
  R g41, g42;
  if constexpr (is_f32<R>()) {
    g41 = 2.0f * c;
    g42 = c;
  } else {
    g41 = lam4 - lam1;
    g42 = lam4 - lam2;
  }
  // left state: reference with lam4, waves moving right add (sigma/2)(lam4 - lam) beta r
  R aL = (R)0.5 * ((R)1 - sigma * lam4);
  R l0, l1, l2, l3;
  if constexpr (is_f32<R>()) {
    const float2 lo = fma2(f2(aL), f2(dq[0], dq[1]), f2(q[0], q[1])), hi = fma2(f2(aL), f2(dq[2], dq[3]), f2(q[2], q[3]));
    l0 = lo.x; l1 = lo.y; l2 = hi.x; l3 = hi.y;
  } else {
    l0 = q[0] + aL * dq[0]; l1 = q[1] + aL * dq[1]; l2 = q[2] + aL * dq[2]; l3 = q[3] + aL * dq[3];
  }
  if (lam1 >= (R)0) {
    R w = hs * g41 * b1;
    l0 += w;
    l1 += w * (-cor);
    l3 += w * c2;
  }
  if (lam2 >= (R)0) {
    R w2 = hs * g42 * b2;
    l0 += w2;
    R w3 = hs * g42 * b3;
    l2 += w3;
  }
  // right state: reference with lam1, waves moving left add (sigma/2)(lam1 - lam) beta r, with
  // lam1 - lam2 = -c and lam1 - lam4 = -2c
  R g12, g14;
  if constexpr (is_f32<R>()) {
    g12 = -c;
    g14 = -2.0f * c;
  } else {
    g12 = lam1 - lam2;
    g14 = lam1 - lam4;
  }
  R aR = (R)0.5 * ((R)1 + sigma * lam1);
  R r0, r1, r2, r3;
  if constexpr (is_f32<R>()) {
    const float2 lo = fma2(f2(-aR), f2(dq[0], dq[1]), f2(q[0], q[1])), hi = fma2(f2(-aR), f2(dq[2], dq[3]), f2(q[2], q[3]));
    r0 = lo.x; r1 = lo.y; r2 = hi.x; r3 = hi.y;
  } else {
    r0 = q[0] - aR * dq[0]; r1 = q[1] - aR * dq[1]; r2 = q[2] - aR * dq[2]; r3 = q[3] - aR * dq[3];
  }
  if (lam2 <= (R)0) {
    R w2 = hs * g12 * b2;
    r0 += w2;
    R w3 = hs * g12 * b3;
    r2 += w3;
  }
  if (lam4 <= (R)0) {
    R w = hs * g14 * b4;
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
// Piecewise-parabolic reconstruction (PPM, Colella & Woodward 1984; the upgrade §3.2 points to).  Edges of
// the middle cell of a0..a4 (one primitive variable along one direction): interface values
// a_{i+1/2} = a_i + (a_{i+1} - a_i)/2 - (da_{i+1} - da_i)/6 from MC-limited slopes da; a local extremum
// flattens the profile to the average; a parabola whose extremum falls inside the cell has it moved to the
// nearer edge (aL = 3 a_i - 2 aR or aR = 3 a_i - 2 aL); flattening blends the edges toward the average.
template <typename R>
__device__ __forceinline__ void ppm_edges(R a0, R a1, R a2, R a3, R a4, R xi, R& eL, R& eR) {
  const R dm = mc2(a0, a1, a2), d0 = mc2(a1, a2, a3), dp = mc2(a2, a3, a4);
  const R c = a2;
  R l, r;
  if constexpr (is_f32<R>()) {
    l = a1 + 0.5f * (a2 - a1) - (d0 - dm) * (1.0f / 6.0f);
    r = a2 + 0.5f * (a3 - a2) - (dp - d0) * (1.0f / 6.0f);
  } else {
    l = a1 + 0.5 * (a2 - a1) - (d0 - dm) / 6.0;
    r = a2 + 0.5 * (a3 - a2) - (dp - d0) / 6.0;
  }
  const bool flat = (r - c) * (c - l) <= (R)0;
  const R da = r - l, mid = c - (R)0.5 * (l + r);
  R d6;
  if constexpr (is_f32<R>())
    d6 = da * da * (1.0f / 6.0f);
  else
    d6 = da * da / 6.0;
  const bool left_ex = da * mid > d6;
  const bool right_ex = !left_ex && -(da * da) / (R)6 > da * mid;
  const R l2 = flat ? c : (left_ex ? (R)3 * c - (R)2 * r : l);
  const R r2 = flat ? c : (right_ex ? (R)3 * c - (R)2 * l : r);
  eL = xi * l2 + ((R)1 - xi) * c;
  eR = xi * r2 + ((R)1 - xi) * c;
}

// PPM characteristic tracing in the face frame.  The cell's profile is a(x) = aL + x (da + a6 (1 - x)) on
// [0, 1], da = aR - aL, a6 = 6 (q - (aL + aR)/2); its average over the fraction s of the cell next to the
// right edge is Ip(s) = aR - (s/2)(da - (1 - 2s/3) a6), next to the left edge Im(s) = aL + (s/2)(da + (1 - 2s/3) a6).
// Left state at i+1/2: ref = Ip(max(sigma lam4, 0)), minus, for each wave with lam_nu >= 0, its component
// (l_nu . (ref - Ip(sigma lam_nu))) r_nu; right state at i-1/2 with Im, ref = Im(max(-sigma lam1, 0)) and the
// waves with lam_nu <= 0.  Eigenvectors as in trace (only their non-zero entries multiplied out, in the
// order of the wave sums); floors on the results.
template <typename R>
__device__ __forceinline__ void trace_ppm(const SP<R>& s, R sigma, const R q[4], const R eL[4], const R eR[4],
                                          R qL[4], R qR[4]) {
  const R rho = q[0], un = q[1], pres = q[3];
  R c, c2, roc, ic2h, ic2, cor;
  if constexpr (is_f32<R>()) {
    const float ir = rcpa(rho);
    const float x = s.gamma * pres * ir;
    const float ic = rsqa(x);
    c = x * ic;
    c2 = c * c;
    roc = 0.5f * rho * ic;
    ic2 = ic * ic;
    ic2h = 0.5f * ic2;
    cor = c * ir;
  } else {
    c = sqrt(s.gamma * pres / rho);
    c2 = c * c;
    roc = (0.5 * rho) / c;
    ic2h = 0.5 / c2;
    ic2 = 1.0 / c2;
    cor = c / rho;
  }
  const R lam1 = un - c, lam2 = un, lam4 = un + c;
  R da[4], a6[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    da[m] = eR[m] - eL[m];
    a6[m] = (R)6 * (q[m] - (R)0.5 * (eL[m] + eR[m]));
  }
  const R two3 = (R)2 / (R)3;
  // ---- left state at i+1/2
  {
    const R s4 = sigma * lam4 > (R)0 ? sigma * lam4 : (R)0;
    R ref[4], o[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ref[m] = eR[m] - (R)0.5 * s4 * (da[m] - ((R)1 - two3 * s4) * a6[m]);
      o[m] = ref[m];
    }
    // ref - Ip(sn); FP32 in the factored form 0.5 (sn - s4)(da - a6 (1 - 2 (sn + s4) / 3)), with
    // sn - s4 = sigma (lam_nu - lam4) = gap taken as -2 sigma c, -sigma c or 0 (at high Mach the difference of
    // the two nearly equal products would lose ~Mach ulps)
    auto dif = [&](int m, R sn, R gap) {
      if constexpr (is_f32<R>())
        return 0.5f * gap * (da[m] - a6[m] * (1.0f - two3 * (sn + s4)));
      else
        return ref[m] - (eR[m] - (R)0.5 * sn * (da[m] - ((R)1 - two3 * sn) * a6[m]));
    };
    const R sc = sigma * c;
    if (lam1 >= (R)0) {
      const R sn = sigma * lam1;
      const R b = -roc * dif(1, sn, -2 * sc) + ic2h * dif(3, sn, -2 * sc);
      o[0] -= b;
      o[1] -= b * (-cor);
      o[3] -= b * c2;
    }
    if (lam2 >= (R)0) {
      const R sn = sigma * lam2;
      const R b2 = dif(0, sn, -sc) + (-ic2) * dif(3, sn, -sc);
      o[0] -= b2;
      const R b3 = dif(2, sn, -sc);
      o[2] -= b3;
    }
    if (lam4 >= (R)0) {
      const R sn = sigma * lam4;
      const R b = roc * dif(1, sn, (R)0) + ic2h * dif(3, sn, (R)0);
      o[0] -= b;
      o[1] -= b * cor;
      o[3] -= b * c2;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) qL[m] = o[m];
  }
  // ---- right state at i-1/2
  {
    const R s1 = -sigma * lam1 > (R)0 ? -sigma * lam1 : (R)0;
    R ref[4], o[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      ref[m] = eL[m] + (R)0.5 * s1 * (da[m] + ((R)1 - two3 * s1) * a6[m]);
      o[m] = ref[m];
    }
    // ref - Im(sn); FP32 in the factored form 0.5 (s1 - sn)(da + a6 (1 - 2 (sn + s1) / 3)), with
    // s1 - sn = sigma (lam_nu - lam1) = gap taken as 0, sigma c or 2 sigma c
    auto dif = [&](int m, R sn, R gap) {
      if constexpr (is_f32<R>())
        return 0.5f * gap * (da[m] + a6[m] * (1.0f - two3 * (sn + s1)));
      else
        return ref[m] - (eL[m] + (R)0.5 * sn * (da[m] + ((R)1 - two3 * sn) * a6[m]));
    };
    const R sc = sigma * c;
    if (lam1 <= (R)0) {
      const R sn = -sigma * lam1;
      const R b = -roc * dif(1, sn, (R)0) + ic2h * dif(3, sn, (R)0);
      o[0] -= b;
      o[1] -= b * (-cor);
      o[3] -= b * c2;
    }
    if (lam2 <= (R)0) {
      const R sn = -sigma * lam2;
      const R b2 = dif(0, sn, sc) + (-ic2) * dif(3, sn, sc);
      o[0] -= b2;
      const R b3 = dif(2, sn, sc);
      o[2] -= b3;
    }
    if (lam4 <= (R)0) {
      const R sn = -sigma * lam4;
      const R b = roc * dif(1, sn, 2 * sc) + ic2h * dif(3, sn, 2 * sc);
      o[0] -= b;
      o[1] -= b * cor;
      o[3] -= b * c2;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) qR[m] = o[m];
  }
  qL[0] = qL[0] < s.small_dens ? s.small_dens : qL[0];
  qR[0] = qR[0] < s.small_dens ? s.small_dens : qR[0];
  qL[3] = qL[3] < s.small_pres ? s.small_pres : qL[3];
  qR[3] = qR[3] < s.small_pres ? s.small_pres : qR[3];
}

// ---------------------------------------------------------------------------------------------------
// Euler flux (Eqs. 8-10, g = 0) of a face state (rho, un, ut, p): (rho un, rho un^2 + p, rho un ut, un (rho E + p)).
template <typename R>
__device__ __forceinline__ void face_flux(const SP<R>& s, R fr, R fu, R fv, R fp, R F[4]) {
  R rhoE;
  if constexpr (is_f32<R>())
    rhoE = fp * s.igm1 + 0.5f * fr * (fu * fu + fv * fv);
  else
    rhoE = fp / s.gm1 + 0.5 * fr * (fu * fu + fv * fv);
  F[0] = fr * fu;
  F[1] = fr * fu * fu + fp;
  F[2] = fr * fu * fv;
  F[3] = fu * (rhoE + fp);
}

// Two-shock Riemann solver (§3.2, "the Riemann solver described in almgren:2010").
// Face frame: (rho, un, ut, p).  Newton iteration on u*_L(p) = u*_R(p) with the shock mass fluxes
// W_K = C_K sqrt(1 + (gamma+1)/(2 gamma) (p/p_K - 1)), C_K = sqrt(gamma p_K rho_K), slopes
// Z_K = 2 W_K^3 / (W_K^2 + C_K^2); acoustic start unless guess > 0.  Sampling at x/t = 0 from the upwind
// side of the contact, Hugoniot star density, shock or linearly interpolated fan.  Returns the flux
// (mass, normal momentum, transverse momentum, energy); iters/conv report the iteration.
__device__ __forceinline__ void riemann(const SP<double>& s, const double qL[4], const double qR[4], double guess,
                                        double F[4], int& iters, bool& conv, double* pstar_out = nullptr) {
  const double g = s.gamma, g1 = s.g1;
  const double rl = qL[0], ul = qL[1], vl = qL[2], pl = qL[3];
  const double rr = qR[0], ur = qR[1], vr = qR[2], pr = qR[3];
  const double cl = sqrt(g * pl * rl);
  const double cr = sqrt(g * pr * rr);
  // stop also once the step's velocity mismatch |dp| (1/Z_L + 1/Z_R) is below tol times the velocity scale
  const double vscale = fabs(ul) + fabs(ur) + cl / rl + cr / rr;
  double pst = guess > 0.0 ? guess : (cr * pl + cl * pr + cl * cr * (ul - ur)) / (cl + cr);
  pst = pst < s.small_pres ? s.small_pres : pst;
  int it = 0;
  bool ok = false;
  while (it < s.maxiter) {
    double wl = cl * sqrt(1.0 + g1 * (pst / pl - 1.0));
    double wr = cr * sqrt(1.0 + g1 * (pst / pr - 1.0));
    double usl = ul - (pst - pl) / wl;
    double usr = ur + (pst - pr) / wr;
    double zl = 2.0 * wl * wl * wl / (wl * wl + cl * cl);
    double zr = 2.0 * wr * wr * wr / (wr * wr + cr * cr);
    double pnew = pst - zl * zr * (usr - usl) / (zl + zr);
    pnew = pnew < s.small_pres ? s.small_pres : pnew;
    double dp = fabs(pnew - pst);
    pst = pnew;
    ++it;
    if (dp <= s.tol * pst || dp * (zl + zr) / (zl * zr) <= s.tol * vscale) {
      ok = true;
      break;
    }
  }
  iters = it;
  conv = ok;
  const double wl = cl * sqrt(1.0 + g1 * (pst / pl - 1.0));
  const double wr = cr * sqrt(1.0 + g1 * (pst / pr - 1.0));
  const double ust = ((wl * ul + wr * ur) + (pl - pr)) / (wl + wr);

  double fr, fu, fv, fp;
  if (ust == 0.0) {
    fr = 0.5 * (rl + rr);
    fu = 0.0;
    fv = 0.5 * (vl + vr);
    fp = pst;
  } else {
    const bool left = ust > 0.0;
    const double sgn = left ? 1.0 : -1.0;
    const double ro = left ? rl : rr, uo = left ? ul : ur, vo = left ? vl : vr, po = left ? pl : pr;
    const double wo = left ? wl : wr;
    const double rst = 1.0 / (1.0 / ro - (pst - po) / (wo * wo));
    fv = vo;
    if (pst > po) {
      const double S = uo - sgn * (wo / ro);
      if (sgn * S >= 0.0) {
        fr = ro; fu = uo; fp = po;
      } else {
        fr = rst; fu = ust; fp = pst;
      }
    } else {
      const double co = sqrt(g * po / ro);
      const double cst = sqrt(g * pst / rst);
      const double SH = uo - sgn * co;
      const double ST = ust - sgn * cst;
      if (sgn * SH >= 0.0) {
        fr = ro; fu = uo; fp = po;
      } else if (sgn * ST <= 0.0) {
        fr = rst; fu = ust; fp = pst;
      } else {
        const double frac = SH / (SH - ST);
        fr = ro + frac * (rst - ro);
        fu = uo + frac * (ust - uo);
        fp = po + frac * (pst - po);
      }
    }
  }
  face_flux(s, fr, fu, fv, fp, F);
  if (pstar_out) *pstar_out = pst;
}

// FP32 form of the same solver.  With a_K = 1 + (gamma+1)/(2 gamma)(p/p_K - 1) and t_K = 1/sqrt(a_K):
// 1/W_K = t_K / C_K, W_K = C_K a_K t_K, and the Newton step -(u*_R - u*_L) / (1/Z_L + 1/Z_R) uses
// 1/Z_K = (a_K + 1) t_K^3 / (2 C_K); one rsqrt per side and one reciprocal per iteration.
__device__ __forceinline__ void riemann(const SP<float>& s, const float qL[4], const float qR[4], float guess,
                                        float F[4], int& iters, bool& conv, float* pstar_out = nullptr) {
  const float g = s.gamma, g1 = s.g1;
  const float rl = qL[0], ul = qL[1], vl = qL[2], pl = qL[3];
  const float rr = qR[0], ur = qR[1], vr = qR[2], pr = qR[3];
  // the two sides go through the same arithmetic: (left, right) pairs in packed operations
  const float2 P = f2(pl, pr), U = f2(ul, ur);
  const float2 X = mul2(mul2(f2(g), P), f2(rl, rr));  // C_K^2 = gamma p_K rho_K
  const float icl = rsqa(X.x), icr = rsqa(X.y);       // 1/C_K
  const float2 C = mul2(X, f2(icl, icr));
  const float cl = C.x, cr = C.y;
  // one MUFU reciprocal each costs fewer issue slots than forming 1/p_K from 1/C_K^2 = 1/(gamma p_K rho_K)
  const float2 IP = f2(rcpa(pl), rcpa(pr));
  // velocity scale of the problem: float rounding leaves u*_R - u*_L uncertain by ~2^-24 of it, which can
  // exceed tol * p* in pressure when p* << rho u^2, so the FP32 stopping rule also accepts a pressure
  // change smaller than the one a velocity mismatch of tol times this scale would produce
  const float2 PIC = mul2(P, f2(icl, icr));
  const float tolv = s.tol * (fabsf(ul) + fabsf(ur) + g * (PIC.x + PIC.y));
  // 1/C_K with the side's sign: u*_L falls and u*_R rises with the star pressure
  const float2 ICS = f2(-icl, icr);
  float pst = guess > 0.0f ? guess : (cr * pl + cl * pr + cl * cr * (ul - ur)) * rcpa(cl + cr);
  pst = pst < s.small_pres ? s.small_pres : pst;
  int it = 0;
  bool ok = false;
  while (it < s.maxiter) {
    const float2 A = fma2(f2(g1), fma2(f2(pst), IP, f2(-1.0f)), f2(1.0f));  // a_K
    const float2 T = f2(rsqa(A.x), rsqa(A.y));                             // t_K
    const float2 IWS = mul2(T, ICS);                                        // (-1/W_L, 1/W_R)
    const float2 US = fma2(sub2(f2(pst), P), IWS, U);                       // (u*_L, u*_R)
    // (a_K + 1) t_K^2 / 2 = (1 + 1/a_K) / 2 = (1 + t_K^2) / 2
    const float2 IZS = mul2(fma2(f2(0.5f), mul2(T, T), f2(0.5f)), IWS);    // (-1/Z_L, 1/Z_R)
    const float iz = IZS.y - IZS.x;  // 1 / (Z_L Z_R / (Z_L + Z_R))
    float pnew = pst - (US.y - US.x) * rcpa(iz);
    pnew = pnew < s.small_pres ? s.small_pres : pnew;
    const float dp = fabsf(pnew - pst);
    pst = pnew;
    ++it;
    if (dp <= s.tol * pst || dp * iz <= tolv) {
      ok = true;
      break;
    }
  }
  iters = it;
  conv = ok;
  const float2 A = fma2(f2(g1), fma2(f2(pst), IP, f2(-1.0f)), f2(1.0f));
  const float tl = rsqa(A.x), tr = rsqa(A.y);
  const float2 W = mul2(mul2(C, A), f2(tl, tr));
  const float wl = W.x, wr = W.y;
  const float2 WU = mul2(W, U);
  const float ust = ((WU.x + WU.y) + (pl - pr)) * rcpa(wl + wr);

  // sampling at x/t = 0 (the same cases as the FP64 solver).  A face on the contact (u* = 0; whole warps of
  // it in a fluid at rest) takes the mean state; otherwise the case (shock, fan head, fan tail, inside the
  // fan) is chosen by selects, since it varies within a warp and a branch per case would run every path.
  float fr, fu, fv, fp;
  if (ust == 0.0f) {
    fr = 0.5f * (rl + rr);
    fu = 0.0f;
    fv = 0.5f * (vl + vr);
    fp = pst;
  } else {
    const bool left = ust > 0.0f;
    const float sgn = left ? 1.0f : -1.0f;
    const float ro = left ? rl : rr, uo = left ? ul : ur, vo = left ? vl : vr, po = left ? pl : pr;
    const float wo = left ? wl : wr;
    const float ico = left ? icl : icr;
    const float iwo = (left ? tl : tr) * ico;
    const float iro = rcpa(ro);                       // 1/rho_o
    const float irst = iro - (pst - po) * iwo * iwo;  // 1/rho*, Hugoniot
    const float rst = rcpa(irst);
    const bool shock = pst > po;
    const float S = uo - sgn * wo * iro;                        // shock speed
    const float SH = uo - sgn * (g * po * ico);                 // fan head u_o -+ c_o
    const float ST = ust - sgn * M<float>::sq(g * pst * irst);  // fan tail u* -+ c*
    const bool take_o = shock ? sgn * S >= 0.0f : sgn * SH >= 0.0f;
    const bool take_star = shock ? !take_o : sgn * ST <= 0.0f;
    fr = take_o ? ro : rst;
    fu = take_o ? uo : ust;
    fp = take_o ? po : pst;
    fv = vo;
    // transonic fans are rare: the interpolation runs only in warps that have one
    const bool in_fan = !take_o && !take_star;
    if (__any_sync(__activemask(), in_fan)) {
      const float frac = SH * rcpa(SH - ST);
      if (in_fan) {
        fr = ro + frac * (rst - ro);
        fu = uo + frac * (ust - uo);
        fp = po + frac * (pst - po);
      }
    }
  }
  face_flux(s, fr, fu, fv, fp, F);
  if (pstar_out) *pstar_out = pst;
}

// HLLC approximate Riemann solver (§3.2's alternative solver, after Toro 1997) in the face frame
// (rho, un, ut, p).  Outer wave speeds: the direct (Davis) bounds of both sides' sound waves,
// S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R); contact speed
// S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R)) / (rho_L (S_L - u_L) - rho_R (S_R - u_R));
// star state of side K: rho_K (S_K - u_K)/(S_K - S*) (1, S*, v_K, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))).
// The flux is F(U_L) for 0 <= S_L, F_L + S_L (U*_L - U_L) for S_L < 0 <= S*, F_R + S_R (U*_R - U_R) for
// S* < 0 <= S_R, F(U_R) for S_R < 0: side o gives F(U_o), plus the jump across its outer wave when that
// wave has passed the face.  FP64 evaluates every expression in the order
// written; FP32 takes its divisions and square roots from reciprocal approximations.  The denominators do
// not vanish: S_L - u_L <= -c_L < 0 < c_R <= S_R - u_R, and S_o - S* is nonzero where the jump is applied.
template <typename R>
__device__ __forceinline__ void hllc(const SP<R>& s, const R qL[4], const R qR[4], R F[4]) {
  const R rl = qL[0], ul = qL[1], vl = qL[2], pl = qL[3];
  const R rr = qR[0], ur = qR[1], vr = qR[2], pr = qR[3];
  R cl, cr;
  if constexpr (is_f32<R>()) {
    cl = M<R>::sq(s.gamma * pl * rcpa(rl));
    cr = M<R>::sq(s.gamma * pr * rcpa(rr));
  } else {
    cl = sqrt(s.gamma * pl / rl);
    cr = sqrt(s.gamma * pr / rr);
  }
  const R SL = M<R>::mn(ul - cl, ur - cr);
  const R SR = M<R>::mx(ul + cl, ur + cr);
  const R num = pr - pl + rl * ul * (SL - ul) - rr * ur * (SR - ur);
  const R den = rl * (SL - ul) - rr * (SR - ur);
  R sst;
  if constexpr (is_f32<R>())
    sst = num * rcpa(den);
  else
    sst = num / den;
  // side whose flux the face takes (left when the whole fan is right of it, or the contact is), and whether
  // that side's outer wave has passed the face
  const bool left = (R)0 <= SL || (R)0 <= sst;
  const R ro = left ? rl : rr, uo = left ? ul : ur, vo = left ? vl : vr, po = left ? pl : pr;
  const R So = left ? SL : SR;
  const bool jump = left ? SL < (R)0 : (R)0 <= SR;
  face_flux(s, ro, uo, vo, po, F);
  if (jump) {
    R Eo, f, es;
    if constexpr (is_f32<R>()) {
      Eo = po * s.igm1 + 0.5f * ro * (uo * uo + vo * vo);
      const float a = ro * (So - uo);
      f = a * rcpa(So - sst);
      es = Eo * rcpa(ro) + (sst - uo) * (sst + po * rcpa(a));
    } else {
      Eo = po / s.gm1 + 0.5 * ro * (uo * uo + vo * vo);
      f = ro * (So - uo) / (So - sst);
      es = Eo / ro + (sst - uo) * (sst + po / (ro * (So - uo)));
    }
    const R Us[4] = {f, f * sst, f * vo, f * es};
    const R Uo[4] = {ro, ro * uo, ro * vo, Eo};
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = F[k] + So * (Us[k] - Uo[k]);
  }
}

// CFL constraint of one interior cell (Eq. 6 with |u|+c): min(dx/(|u|+c), dy/(|v|+c)), folded into rbest;
// non-finite and non-positive cells set status bits instead.  FP64 evaluates the formula as written (the
// order the exact-rounding FP64 kernels share with the plain C implementation).  FP32 forms the same
// minimum as the reciprocal of the larger signal rate max((|u|+c)/dx, (|v|+c)/dy), with c^2 = gamma p / rho
// from the reciprocal of rho already formed for the velocities: one reciprocal square root and two
// reciprocals per cell instead of four divisions.
template <typename R>
__device__ __forceinline__ void cfl_value(const SP<R>& s, R U0, R U1, R U2, R U3, R& rbest, unsigned int& flags) {
  if (!finite4(U0, U1, U2, U3)) {
    flags |= STATUS_NONFINITE;
    return;
  }
  if constexpr (is_f32<R>()) {
    // every product and sum rounds on its own (no multiply-add contraction, which the compiler would
    // choose differently in each kernel that inlines this), so the step kernels that fold in the CFL value
    // of their new state and the standalone reduction give the same time step
    const float rho = U0 < s.small_dens ? s.small_dens : U0;
    const float ir = rcpa(rho);
    const float u = __fmul_rn(U1, ir), v = __fmul_rn(U2, ir);
    const float ke = __fmul_rn(__fmul_rn(0.5f, rho), __fadd_rn(__fmul_rn(u, u), __fmul_rn(v, v)));
    const float e = __fsub_rn(U3, ke);
    if (!(U0 > 0.0f) || !(e > 0.0f)) flags |= STATUS_NEGATIVE;
    float p;
    if (ke > __fmul_rn(s.rec, U3)) {  // as cons_to_prim: recover e = E - rho |u|^2 / 2 in double
      const double rd = (double)rho, ud = __ddiv_rn((double)U1, rd), vd = __ddiv_rn((double)U2, rd);
      p = (float)__dmul_rn((double)s.gm1,
                           __dsub_rn((double)U3, __dmul_rn(__dmul_rn(0.5, rd), __dadd_rn(__dmul_rn(ud, ud),
                                                                                      __dmul_rn(vd, vd)))));
    } else {
      p = __fmul_rn(s.gm1, e);
    }
    p = p < s.small_pres ? s.small_pres : p;
    const float c2 = __fmul_rn(__fmul_rn(s.gamma, p), ir);
    const float cs = __fmul_rn(c2, rsqa(c2));
    const float rate = fmaxf(__fmul_rn(__fadd_rn(fabsf(u), cs), s.idx), __fmul_rn(__fadd_rn(fabsf(v), cs), s.idy));
    const float t = rcpa(rate);
    rbest = t < rbest ? t : rbest;
  } else {
    R rho, u, v, p;
    cons_to_prim(s, U0, U1, U2, U3, rho, u, v, p);
    {
      const R ke = (0.5 * (U1 * U1 + U2 * U2)) / U0;
      if (!(U0 > (R)0) || !(U3 - ke > (R)0)) flags |= STATUS_NEGATIVE;
    }
    const R cs = sqrt((s.gamma * p) / rho);
    const R tx = s.dx / (fabs(u) + cs);
    const R ty = s.dy / (fabs(v) + cs);
    const R t = fmin(tx, ty);
    rbest = t < rbest ? t : rbest;
  }
}

template <typename R>
__device__ __forceinline__ void cfl_cell(const SP<R>& s, const R* __restrict__ U, size_t o, size_t plane, R& rbest,
                                         unsigned int& flags) {
  cfl_value(s, U[o], U[o + plane], U[o + 2 * plane], U[o + 3 * plane], rbest, flags);
}

// Source cell of a tile cell at padded index (gi, gj).  BCMAP: ghost and out-of-array positions map to
// the interior cell the boundary conditions assign them (periodic wrap, outflow clamp), i.e. the value a
// ghost fill would have written; otherwise the padded array is read as is, clamped to its extent.
template <bool BCMAP>
__device__ __forceinline__ size_t cell_offset(const KParams& P, int gi, int gj) {
  if constexpr (BCMAP) {
    int ki = gi - P.ng, kj = gj - P.ng;
    if (ki < 0 || ki >= P.nx) ki = P.bc[0] == 1 ? ((ki % P.nx) + P.nx) % P.nx : (ki < 0 ? 0 : P.nx - 1);
    if (kj < 0 || kj >= P.ny) kj = P.bc[2] == 1 ? ((kj % P.ny) + P.ny) % P.ny : (kj < 0 ? 0 : P.ny - 1);
    return (size_t)(kj + P.ng) * P.pitch + (ki + P.ng);
  } else {
    gi = gi < P.NX - 1 ? gi : P.NX - 1;
    gj = gj < P.NY - 1 ? gj : P.NY - 1;
    return (size_t)gj * P.pitch + gi;
  }
}

}  // namespace hydro
