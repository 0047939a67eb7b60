// Dimensionally split variant of the step (paper §3.1: the fluxes of a directional update are built without
// the transverse flow, each directional update acts on the state the previous one left, and the order of the
// directions alternates from step to step).  One sweep applies the one-dimensional piecewise-linear Godunov
// method of §3.2 along x or y to every interior line of the state:
//   0. primitives of the tile's cells, in the face frame (rho, u_normal, u_transverse, p);
//   1. flattening along the line only, xi = min(chi_m, chi_{m-s});
//   2. limited slopes along the line times xi, characteristic tracing (Eq. 13) with sigma = dt / h;
//   3. Riemann solves at the faces, artificial viscosity from the divergence along the line;
//   4. conservative update U += sigma (F_{m-1/2} - F_{m+1/2}).
// Gravity (along y): every traced v gains dt g / 2 (transverse in the x sweep, normal in the y sweep), and
// the y sweep adds the time-centred sources (rho v) += dt g (rho^n + rho^{n+1}) / 2 and (rho E) +=
// dt g ((rho v)^n + (rho v)^{n+1}) / 2, n being the state it starts from.
// A CTA takes NL lines of LN cells along the sweep (plus the 4 halo cells each side the flattening needs).
// Halo cells outside the domain are read through the boundary conditions' map of the interior (bc_cell: the
// values a ghost fill would write), so neither sweep needs a ghost-fill pass.  FUSED (the second sweep of a
// step run by hydro_step_fused): the sweep also folds the CFL constraint of its new cells into a minimum,
// and its last block advances the time and writes the next step's factors, as the fused unsplit step does.
// Shared memory is laid out so that the load enumeration is also the storage order: along-the-line
// positions are fastest for x sweeps (rows), lines are fastest for y sweeps (columns), so both load
// consecutive x addresses with consecutive threads.  Instantiated for FP32 in k_split.cu and for FP64 in
// k_split_f64.cu, which is compiled without multiply-add contraction (each expression then rounds like the
// plain C implementation of the method).
#pragma once
#include <atomic>

#include "ctu_kernels.cuh"

namespace hydro {

template <typename R, int DIR, int LN, int NL>
struct SweepLayout {
  static constexpr int PQ = LN + 8;  // positions loaded along a line
  static constexpr int PC = LN + 2;  // traced cells along a line: positions [3, LN + 5)
  static constexpr int PF = LN + 1;  // faces along a line: positions [4, LN + 4]
  static constexpr int nQ = PQ * NL, nC = PC * NL, nF = PF * NL;
  // strides along the line and between lines, for the q arrays (Q) and the traced-cell arrays (C)
  static constexpr int QA = DIR == 0 ? 1 : NL, QL = DIR == 0 ? PQ : 1;
  static constexpr int CA = DIR == 0 ? 1 : NL, CL = DIR == 0 ? PC : 1;
  static constexpr int FA = DIR == 0 ? 1 : NL, FL = DIR == 0 ? PF : 1;
  // [4][nQ] primitives (stages 0-2), then [4][nF] fluxes (stages 3-4); [nC] xi; [nC] u_normal; [4][nC] x 2
  // traced states
  static constexpr int elems = 4 * nQ + 2 * nC + 8 * nC;
  static constexpr size_t bytes = sizeof(R) * (size_t)elems;
  static_assert(nF <= nQ, "the fluxes reuse the primitive area");
};

// item e of an enumeration over (position along, line) in storage order -> (along, line)
template <int DIR, int PA, int NL>
__device__ __forceinline__ void sweep_item(int e, int& a, int& l) {
  if constexpr (DIR == 0) {
    a = e % PA;
    l = e / PA;
  } else {
    l = e % NL;
    a = e / NL;
  }
}

// Threads of the FP32 sweep CTAs (overridable at compile time for sweeps of the launch shape).  Measured per
// split step, KH 1024^2 / Sedov 2048^2: 256 threads 77.9 / 225 us, 384 threads (36 warps per SM, 56
// registers) 70.3 / 206 us, 512 threads (two CTAs per SM) 77.3 / 245 us.
#ifndef HYDRO_SWEEP_F32_NT
#define HYDRO_SWEEP_F32_NT 384
#endif
constexpr int SWEEP_F32_NT = HYDRO_SWEEP_F32_NT;

// Resident CTAs per SM the register allocator must allow (shared memory admits three tiles of either
// precision's shapes).
#ifndef HYDRO_SWEEP_MINB
#define HYDRO_SWEEP_MINB 3
#endif

template <typename R, int DIR, int LN, int NL, int NT, bool FUSED, int MODE>
__global__ void __launch_bounds__(NT, HYDRO_SWEEP_MINB) sweep_kernel(KParams P, const R* __restrict__ Uin, R* __restrict__ Uout,
                                                   StepScalars sc_host, const StepScalars* __restrict__ sc_dev,
                                                   DevScratch* __restrict__ scr, int check_state,
                                                   StepScalars* __restrict__ sc_next, double tmax) {
  using L = SweepLayout<R, DIR, LN, NL>;
  constexpr int PQ = L::PQ, PC = L::PC, PF = L::PF, nQ = L::nQ, nC = L::nC, nF = L::nF;
  constexpr int kn = DIR == 0 ? 1 : 2, kt = DIR == 0 ? 2 : 1;  // normal / transverse momentum components
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R* sq = reinterpret_cast<R*>(smem_raw);  // [4][nQ] primitives, face frame
  R* sG = sq;                               // [4][nF] fluxes (conserved order), after stage 2
  R* sxi = sq + 4 * nQ;                     // [nC]
  R* sun = sxi + nC;                        // [nC] normal velocity of the traced cells
  R* sl = sun + nC;                         // [4][nC] left state at m+1/2 of cell m
  R* sr = sl + 4 * nC;                      // [4][nC] right state at m-1/2

  SP<R> s;
  s.load(P);
  const StepScalars& sc = sc_dev ? *sc_dev : sc_host;
  R sigma;
  if constexpr (is_f32<R>())
    sigma = DIR == 0 ? sc.sigx_f : sc.sigy_f;
  else
    sigma = DIR == 0 ? sc.sigx : sc.sigy;
  const R h = DIR == 0 ? s.dx : s.dy;
  R hdtg;  // dt g / 2
  if constexpr (is_f32<R>())
    hdtg = sc.hdtg_f;
  else
    hdtg = sc.hdtg;
  const int n = DIR == 0 ? P.nx : P.ny;      // interior cells along a line
  const int nlines = DIR == 0 ? P.ny : P.nx;
  const int bt = DIR == 0 ? blockIdx.x : blockIdx.y;  // tile along the sweep
  const int bl = DIR == 0 ? blockIdx.y : blockIdx.x;  // group of lines
  const int a0 = P.ng + bt * LN;                      // padded index of the tile's first cell along the sweep
  const int l0 = P.ng + bl * NL;                      // padded index of its first line
  const size_t plane = (size_t)P.NY * P.pitch;
  const int tid = threadIdx.x;
  // Lines past the domain (a ragged last group) and positions past the padded array (a ragged last tile)
  // are clamped to cells that exist; what is computed from them is never stored or counted.
  auto clamp_line = [&](int l) { return l < P.ng + nlines ? l : P.ng + nlines - 1; };
  auto clamp_along = [&](int a) { return a < n + 2 * P.ng ? a : n + 2 * P.ng - 1; };
  auto interior_offset = [&](int a, int l) -> size_t {
    const int i = DIR == 0 ? a : l, j = DIR == 0 ? l : a;
    return (size_t)j * P.pitch + i;
  };
  // cell (along a, line l) with ghost values from the boundary map
  auto load_cell = [&](int a, int l, R v[4]) {
    a = clamp_along(a);
    l = clamp_line(l);
    if (a >= P.ng && a < P.ng + n) {
      const size_t o = interior_offset(a, l);
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = __ldg(Uin + o + k * plane);
    } else {
      bc_cell(P, Uin, DIR == 0 ? a : l, DIR == 0 ? l : a, plane, v);
    }
  };
  auto store_prim = [&](int e, const R U[4]) {
    R q[4];
    cons_to_prim(s, U[0], U[1], U[2], U[3], q[0], q[1], q[2], q[3]);
    sq[e] = q[0];
    sq[nQ + e] = q[kn];
    sq[2 * nQ + e] = q[kt];
    sq[3 * nQ + e] = q[3];
  };

  // ---- 0. primitives of positions [0, LN + 8) of every line
  if (a0 - 4 >= P.ng && a0 + LN + 4 <= P.ng + n) {
    // the tile's positions are all interior: every load of a thread is issued before any conversion
    constexpr int NLD = (nQ + NT - 1) / NT;
    R Ul[NLD][4];
#pragma unroll
    for (int it = 0; it < NLD; ++it) {
      const int e = tid + it * NT;
      if (e < nQ) {
        int a, l;
        sweep_item<DIR, PQ, NL>(e, a, l);
        const size_t o = interior_offset(a0 - 4 + a, clamp_line(l0 + l));
#pragma unroll
        for (int k = 0; k < 4; ++k) Ul[it][k] = __ldg(Uin + o + k * plane);
      }
    }
#pragma unroll
    for (int it = 0; it < NLD; ++it) {
      const int e = tid + it * NT;
      if (e < nQ) store_prim(e, Ul[it]);
    }
  } else {
    for (int e = tid; e < nQ; e += NT) {
      int a, l;
      sweep_item<DIR, PQ, NL>(e, a, l);
      R U[4];
      load_cell(a0 - 4 + a, l0 + l, U);
      store_prim(e, U);
    }
  }
  __syncthreads();

  // ---- 1.-2. flattening, slopes and tracing of the cells at positions [3, LN + 5)
  for (int e = tid; e < nC; e += NT) {
    int c, l;
    sweep_item<DIR, PC, NL>(e, c, l);
    const int b = (c + 3) * L::QA + l * L::QL;  // the cell's index in the q arrays
    constexpr int st = L::QA;
    const R* qp = sq + 3 * nQ;
    const R* qn = sq + nQ;
    R xi = (R)1;
    if (s.flatten) {
      auto chi = [&](int m) {
        return flatten_chi<R>(qp[b + (m - 2) * st], qp[b + (m - 1) * st], qp[b + (m + 1) * st], qp[b + (m + 2) * st],
                              qn[b + (m - 1) * st], qn[b + (m + 1) * st], s.small_pres);
      };
      const int sgn = (qp[b + st] - qp[b - st]) >= (R)0 ? 1 : -1;
      xi = M<R>::mn(chi(0), chi(-sgn));
    }
    sxi[e] = xi;
    sun[e] = qn[b];
    R q[4], ql[4], qr[4];
    if constexpr ((MODE & RECON_PPM) != 0) {
      R eL[4], eR[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const R* a = sq + k * nQ + b;
        q[k] = a[0];
        ppm_edges<R>(a[-2 * st], a[-st], a[0], a[st], a[2 * st], xi, eL[k], eR[k]);
      }
      trace_ppm<R>(s, sigma, q, eL, eR, ql, qr);
    } else {
      R dq[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const R* a = sq + k * nQ + b;
        q[k] = a[0];
        dq[k] = xi * slope<R>(s.limiter, a[-2 * st], a[-st], a[0], a[st], a[2 * st]);
      }
      trace<R>(s, sigma, q, dq, ql, qr);
    }
    if (P.use_grav) {  // half-step gravity on v: transverse in the x sweep, normal in the y sweep
      constexpr int kv = DIR == 0 ? 2 : 1;
      ql[kv] = ql[kv] + hdtg;
      qr[kv] = qr[kv] + hdtg;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sl[k * nC + e] = ql[k];
      sr[k * nC + e] = qr[k];
    }
  }
  __syncthreads();

  // ---- 3. Riemann solves + artificial viscosity at faces [0, LN] of each line (face f between traced
  //         cells f and f + 1, i.e. padded positions a0 + f - 1 and a0 + f)
  TileCounters cnt;
  for (int e = tid; e < nF; e += NT) {
    int f, l;
    sweep_item<DIR, PF, NL>(e, f, l);
    const int fa = a0 + f;  // padded index of the cell right of the face
    const bool valid = l0 + l < P.ng + nlines && fa <= P.ng + n;
    const int cL = f * L::CA + l * L::CL, cR = cL + L::CA;
    R a[4], bq[4], F[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = sl[k * nC + cL];
      bq[k] = sr[k * nC + cR];
    }
    int it = 0;
    bool ok = true;
    if constexpr (face_kind(MODE) == FACE_HLLC) {
      hllc(s, a, bq, F);
    } else {
      R pst;
      riemann(s, a, bq, (R)0, F, it, ok, &pst);
    }
    if (valid && (f < LN || fa == P.ng + n)) {  // a face shared by two tiles counts once
      cnt.solves++;
      cnt.iters += it;
      cnt.nonconv += ok ? 0 : 1;
    }
    R G[4];
    G[0] = F[0];
    G[kn] = F[1];
    G[kt] = F[2];
    G[3] = F[3];
    if (s.cvisc > (R)0 && valid) {
      R av;
      if constexpr (is_f32<R>()) {
        av = s.cvisc * M<R>::mx(sun[cL] - sun[cR], (R)0);
      } else {
        const R div = (sun[cR] - sun[cL]) / h;
        av = s.cvisc * M<R>::mx(-div * h, (R)0);
      }
      R UL[4], UR[4];
      load_cell(fa - 1, l0 + l, UL);
      load_cell(fa, l0 + l, UR);
#pragma unroll
      for (int k = 0; k < 4; ++k) G[k] += av * (UL[k] - UR[k]);
    }
    const int g = f * L::FA + l * L::FL;
#pragma unroll
    for (int k = 0; k < 4; ++k) sG[k * nF + g] = G[k];
  }
  __syncthreads();

  // ---- 4. conservative update of the tile's interior cells
  constexpr int nU = LN * NL;
  R cmin = is_f32<R>() ? (R)FLT_MAX : (R)DBL_MAX;
  for (int e = tid; e < nU; e += NT) {
    int u, l;
    sweep_item<DIR, LN, NL>(e, u, l);
    if (l0 + l >= P.ng + nlines || a0 + u >= P.ng + n) continue;
    const size_t o = interior_offset(a0 + u, l0 + l);
    const int g = u * L::FA + l * L::FL;
    R Un[4], U0[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      U0[k] = __ldg(Uin + o + k * plane);
      Un[k] = U0[k] + sigma * (sG[k * nF + g] - sG[k * nF + g + L::FA]);
    }
    if (DIR == 1 && P.use_grav) {
      // the time-centred gravity sources, once per step, from the state this sweep starts from
      Un[2] = Un[2] + hdtg * (U0[0] + Un[0]);
      Un[3] = Un[3] + hdtg * (U0[2] + Un[2]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) Uout[o + k * plane] = Un[k];
    if constexpr (FUSED) {
      cfl_value(s, Un[0], Un[1], Un[2], Un[3], cmin, cnt.flags);  // the next step's constraint (Eq. 6)
    } else if (check_state) {
      if (!finite4(Un[0], Un[1], Un[2], Un[3])) {
        cnt.flags |= STATUS_NONFINITE;
      } else {
        const R ke = M<R>::dv((R)0.5 * (Un[1] * Un[1] + Un[2] * Un[2]), Un[0]);
        if (!(Un[0] > (R)0) || !(Un[3] - ke > (R)0)) cnt.flags |= STATUS_NEGATIVE;
      }
    }
  }
  flush_counters<NT>(cnt, scr);
  if constexpr (FUSED) {
    // block minimum of the CFL constraint; the last block to finish advances the time by this step's dt
    // and writes the next step's factors (dt = cfl * min, clamped to reach tmax when tmax > 0)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const R o = __shfl_xor_sync(0xffffffffu, cmin, off);
      cmin = o < cmin ? o : cmin;
    }
    __shared__ R wmin[NT / 32];
    __shared__ bool last;
    if ((tid & 31) == 0) wmin[tid >> 5] = cmin;
    __syncthreads();
    if (tid == 0) {
      R b = wmin[0];
      for (int k = 1; k < NT / 32; ++k) b = wmin[k] < b ? wmin[k] : b;
      atomicMin(&scr->dtn_min_bits, (unsigned long long)__double_as_longlong((double)b));
      __threadfence();
      last = atomicAdd(&scr->step_blocks_done, 1u) == gridDim.x * gridDim.y - 1u;
    }
    __syncthreads();
    if (last && tid == 0) {
      __threadfence();
      const unsigned long long bits =
          atomicExch(&scr->dtn_min_bits, (unsigned long long)__double_as_longlong(DBL_MAX));
      const double t = scr->t + sc.dt;
      scr->t = t;
      scr->nsteps = scr->nsteps + 1;
      double dt = P.cfl * __longlong_as_double((long long)bits);
      if (tmax > 0.0) {
        const double left = tmax - t;
        dt = dt > left ? left : dt;
        dt = dt < 0.0 ? 0.0 : dt;
      }
      scr->dt = dt;
      *sc_next = make_step_scalars(dt, P.dx, P.dy, P.grav);
      scr->step_blocks_done = 0u;
    }
  }
}

// Launch of one sweep with the tile shape of the precision (dynamic shared memory raised once per device).
// sc_next == NULL: a plain sweep; otherwise the fused second sweep of a step (FUSED instantiation).  MODE:
// FACE_PLAIN or FACE_HLLC, with RECON_PPM for piecewise-parabolic reconstruction (each its own instantiation,
// so the paper's configuration keeps its registers).
template <typename R, int DIR, int LN, int NL, int NT, int MODE>
struct Sweep {
  static cudaError_t launch(const KParams& P, const R* Uin, R* Uout, const StepScalars& sc_host,
                            const StepScalars* sc_dev, DevScratch* scr, int check_state, StepScalars* sc_next,
                            double tmax, cudaStream_t stream) {
    using L = SweepLayout<R, DIR, LN, NL>;
    static std::atomic<unsigned long long> done_plain{0}, done_fused{0};
    const int along = DIR == 0 ? P.nx : P.ny, lines = DIR == 0 ? P.ny : P.nx;
    const int ta = (along + LN - 1) / LN, tl = (lines + NL - 1) / NL;
    const dim3 grid(DIR == 0 ? ta : tl, DIR == 0 ? tl : ta);
    cudaError_t e;
    if (sc_next) {
      e = smem_attr_once(sweep_kernel<R, DIR, LN, NL, NT, true, MODE>, L::bytes, done_fused);
      if (e != cudaSuccess) return e;
      sweep_kernel<R, DIR, LN, NL, NT, true, MODE><<<grid, NT, L::bytes, stream>>>(P, Uin, Uout, sc_host, sc_dev, scr,
                                                                                  check_state, sc_next, tmax);
    } else {
      e = smem_attr_once(sweep_kernel<R, DIR, LN, NL, NT, false, MODE>, L::bytes, done_plain);
      if (e != cudaSuccess) return e;
      sweep_kernel<R, DIR, LN, NL, NT, false, MODE><<<grid, NT, L::bytes, stream>>>(P, Uin, Uout, sc_host, sc_dev, scr,
                                                                                   check_state, nullptr, 0.0);
    }
    return cudaGetLastError();
  }
};

}  // namespace hydro
