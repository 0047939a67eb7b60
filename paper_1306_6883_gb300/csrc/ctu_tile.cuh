// One tile of the fused CTU step (paper §3.2 algorithm; CTU construction §3.1, Eqs. 3-5), shared by the
// single-problem kernel (k_ctu.cu) and the batched persistent kernel (k_batch.cu).
//
// A CTA computes TX x TY interior cells.  It stages the (TX+8) x (TY+8) primitive tile (4-cell halo) in
// shared memory and runs every stage of the step on it without sending any intermediate to global memory:
//   0. load U (FP32 tiles inside the valid array: one TMA bulk tensor copy), convert to primitives (Eqs. 11-12)
//   1. flattening coefficient xi on (TX+2) x (TY+2) cells    (§3.2, Colella 1990)
//   2. limited slopes and characteristic tracing, x and y     (§3.1 limiter; Eq. 13)
//   3. Riemann solves on the traced (hat) states at all faces the transverse terms need
//   4. transverse correction + final Riemann solves + artificial viscosity at the tile's faces
//   5. conservative update (Eq. 5), written to the other state buffer
// Global traffic per cell is one read of U (plus the halo) and one write of U^{n+1}.  FP32 tiles keep U^n
// of the traced cells in shared memory for the viscosity term and the update; FP64 tiles (whose shared
// memory is twice as large per cell) re-read it through L1/L2.
//
// Shared memory is reused across stages: the hat fluxes of stage 3 overwrite the primitive tile (dead
// after stage 2; the velocities the viscosity needs are kept separately), and each final flux of stage 4
// overwrites the left traced state that only its own face reads.
#pragma once

#include "hydro_device.cuh"
#include "mlp.cuh"
#include "tma.cuh"

namespace hydro {

// Storage of a family of 4-component values per cell or face (traced states, fluxes, U^n copies) in shared
// memory.  FP32 keeps a cell's four components together, so that one 16-byte access moves them (the face
// loops then issue one load or store per state instead of four); FP64 keeps four planes of n values.
template <typename R, int n>
struct Quad {
  static __device__ __forceinline__ void ld(const R* base, int c, R v[4]) {
    if constexpr (is_f32<R>()) {
      const float4 t = reinterpret_cast<const float4*>(base)[c];
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = base[k * n + c];
    }
  }
  static __device__ __forceinline__ void st(R* base, int c, R v0, R v1, R v2, R v3) {
    if constexpr (is_f32<R>()) {
      reinterpret_cast<float4*>(base)[c] = make_float4(v0, v1, v2, v3);
    } else {
      base[c] = v0; base[n + c] = v1; base[2 * n + c] = v2; base[3 * n + c] = v3;
    }
  }
};

template <typename R, int TX, int TY>
struct TileLayout {
  static constexpr int QX = TX + 8, QY = TY + 8;  // primitive tile with a 4-cell halo
  static constexpr int SX = TX + 2, SY = TY + 2;  // cells whose face states are traced
  static constexpr int QP = QX;  // row pitch of the primitive tile
  // FP32 tiles keep the conserved values of the traced cells for the viscosity term (no global re-read);
  // FP64 tiles re-read them from L2 to keep 3 CTAs per SM
  static constexpr bool SMEM_U = sizeof(R) == 4;
  static constexpr int nC = SX * SY;
  static constexpr int nQ = 4 * QP * QY;
  static constexpr int nFXH = 4 * SY * (TX + 1);  // hat x fluxes: rows [3, TY+5), faces [4, TX+5)
  static constexpr int nFYH = 4 * (TY + 1) * SX;  // hat y fluxes: faces [4, TY+5), columns [3, TX+5)
  static constexpr int nA = (nQ + nC) > (nFXH + nFYH) ? (nQ + nC) : (nFXH + nFYH);  // region A
  static constexpr int nS = 4 * nC;               // one traced-state family
  static constexpr int nU = SMEM_U ? 4 * nC : 0;
  static constexpr int elems = nA + 4 * nS + 2 * nC + nU;
  static constexpr size_t bytes = sizeof(R) * (size_t)elems;
  // FP32 quads (Quad) are 16-byte accesses: every array of them starts on a 16-byte boundary
  static_assert(sizeof(R) != 4 || (nA % 4 == 0 && nC % 4 == 0 && nFXH % 4 == 0), "quad arrays must stay aligned");
};

// The four conserved values of padded cell (gi, gj) as the step sees them: through the boundary map for the
// fused step (bc_cell where a side is reflecting or hydrostatic), else from the ghost-filled array.
template <bool FUSED, typename R>
__device__ __forceinline__ void tile_cell(const KParams& P, const R* __restrict__ U, int gi, int gj, size_t plane,
                                          R v[4]) {
  if (FUSED && P.bc_general) {
    R w[4];
    bc_cell_clamped(P, U, gi, gj, plane, w);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = w[k];
  } else {
    const size_t o = cell_offset<FUSED>(P, gi, gj);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __ldg(U + o + k * plane);
  }
}

// Counters each thread accumulates over the tiles it works on.
struct TileCounters {
  unsigned int solves = 0, iters = 0, nonconv = 0, flags = 0;
};

// Time-step factors in the kernel's precision.
template <typename R>
struct StepFactors {
  R sigx, sigy, hx, hy, hdtg;
  __device__ __forceinline__ void load(const StepScalars& sc) {
    if constexpr (is_f32<R>()) {
      sigx = sc.sigx_f; sigy = sc.sigy_f; hx = sc.hx_f; hy = sc.hy_f; hdtg = sc.hdtg_f;
    } else {
      sigx = sc.sigx; sigy = sc.sigy; hx = sc.hx; hy = sc.hy; hdtg = sc.hdtg;
    }
  }
};

// Identity of a face within one step, for the harvest's sampling hash.
__device__ __forceinline__ unsigned int face_key(int bx, int by, int stage, int e) {
  return hash32((unsigned int)bx * 0x9E3779B1u ^ hash32((unsigned int)by * 0x85EBCA77u + (unsigned int)stage)) ^
         (unsigned int)e * 0xC2B2AE3Du;
}

// One Riemann solve of a face (every lane of the warp calls this; `active` lanes have a face).
//  FACE_PLAIN:   acoustic start.
//  FACE_HARVEST: acoustic start, and a hash-sampled subset of faces records inputs, p* and iterations.
//  FACE_HLLC:    the HLLC solver instead of the two-shock iteration (no iterations to count).
// (FACE_LEARNED tiles solve their ungated faces as FACE_PLAIN and their gated ones after the tile's network
// pass, see ctu_tile.)
template <typename R, int MODE>
__device__ __forceinline__ void face_solve(const SP<R>& s, const R a[4], const R b[4], bool active,
                                           const FaceHook& hook, unsigned int key, R F[4], TileCounters& cnt) {
  constexpr int K = face_kind(MODE);
  static_assert(K == FACE_PLAIN || K == FACE_HLLC || K == FACE_HARVEST, "face loops solve plain, harvest or HLLC");
  static_assert(K != FACE_HARVEST || is_f32<R>(), "the harvest is an FP32 path");
  if constexpr (K == FACE_HLLC) {
    if (!active) return;
    hllc(s, a, b, F);
    cnt.solves++;
    return;
  }
  if (!active) return;
  int it;
  bool ok;
  R pst;
  riemann(s, a, b, (R)0, F, it, ok, &pst);
  cnt.solves++;
  cnt.iters += it;
  cnt.nonconv += ok ? 0 : 1;
  if constexpr (K == FACE_HARVEST) {
    if (hash32(key ^ hook.hseed) < hook.hthresh ||
        (hook.hgate_ratio > 0.f && strong_face(a, b, hook.hgate_ratio, hook.hgate_u4))) {
      const unsigned long long k = atomicAdd(hook.hcount, 1ull);
      if (k < hook.hcap) {
        float* d = hook.hbuf + 8 * k;
        d[0] = a[0]; d[1] = a[1]; d[2] = a[3]; d[3] = b[0]; d[4] = b[1]; d[5] = b[3]; d[6] = pst;
        d[7] = (float)it;
      }
    }
  }
}

// The FP32 two-shock solve of a queued face, out of line for the single-problem step: there the pass over
// queued faces is rare, and a second inlined copy of the solver in the kernel made the code generated for the
// face loops slower (Sedov 4096^2 learned step 1.163 ms inline, 1.150 ms with this call).  Ensemble tiles,
// whose passes are frequent, keep the solver inline (the call made them 2.6 % slower).
static __device__ __noinline__ void riemann_out(float gamma, float g1, float igm1, float small_pres, float tol,
                                                int maxiter, float rl, float ul, float vl, float pl, float rr,
                                                float ur, float vr, float pr, float guess, float F[4], int& it,
                                                bool& ok) {
  SP<float> s{};
  s.gamma = gamma;
  s.g1 = g1;
  s.igm1 = igm1;
  s.small_pres = small_pres;
  s.tol = tol;
  s.maxiter = maxiter;
  const float a[4] = {rl, ul, vl, pl}, b[4] = {rr, ur, vr, pr};
  riemann(s, a, b, guess, F, it, ok);
}

// Gated faces a FACE_LEARNED tile holds per stage: 2 words each (face item, starting pressure).  A shared
// array of its own (1 KB), present only in the learned kernels.
constexpr int LEARNED_QUEUE = 128;
__device__ __forceinline__ float* learned_queue() {
  __shared__ float q[2 * LEARNED_QUEUE];
  return q;
}

// Whether tile (bx, by) loads its padded box by one TMA copy: the box must lie where the array holds the
// values the step needs (FUSED: the interior, so that no boundary map applies; otherwise the ghost-filled
// array), and the copy's shared-memory destination must be 128-byte aligned.
template <int TX, int TY, bool FUSED>
__device__ __forceinline__ bool tile_box_ok(const KParams& P, int bx, int by, const void* dst) {
  constexpr int QX = TX + 8, QY = TY + 8;
  if ((smem_addr(dst) & 127u) != 0) return false;
  const int x0 = P.ng + bx * TX - 4, y0 = P.ng + by * TY - 4;
  return FUSED ? (x0 >= P.ng && x0 + QX <= P.ng + P.nx && y0 >= P.ng && y0 + QY <= P.ng + P.ny)
               : (x0 + QX <= P.NX && y0 + QY <= P.NY);
}

// One TX x TY tile (tile indices bx, by) of one CTU step, executed by all NT threads of the block.
// smem_raw must hold TileLayout<R, TX, TY>::bytes.  Starts and ends with a block-wide barrier-free
// state, so consecutive calls by the same block need one __syncthreads() between them.  MODE selects
// the face-solve variant (face_solve) and, with RECON_PPM, piecewise-parabolic reconstruction in stage 2;
// wsm is the network's weights for FACE_LEARNED.  FUSED: ghost cells
// come from the boundary-condition map of the interior (no ghost fill needed) and the CFL constraint of
// every new cell is folded into *cfl_min (no separate dt pass needed).  PERSIST: the block runs several
// tiles in turn (a TMA tile load then first orders the previous tile's shared-memory accesses before it).
// tmap: TMA descriptor of Uin for FP32 tile loads (NULL: cell by cell).
template <typename R, int TX, int TY, int NT, int MODE = FACE_PLAIN, bool FUSED = false, bool PERSIST = false>
__device__ __forceinline__ void ctu_tile(const KParams& P, const SP<R>& s, const StepFactors<R>& f,
                                         const R* __restrict__ Uin, R* __restrict__ Uout, int bx, int by,
                                         unsigned char* smem_raw, TileCounters& cnt, const FaceHook& hook = FaceHook{},
                                         const MlpBlob* wsm = nullptr, R* cfl_min = nullptr,
                                         const CUtensorMap* tmap = nullptr) {
  using L = TileLayout<R, TX, TY>;
  constexpr int QX = L::QX, QP = L::QP, QY = L::QY, SX = L::SX, SY = L::SY, nC = L::nC;
  // row width of the y-face items of stage 4 and the cells of stage 5: SX when that makes every warp one
  // row (consecutive, conflict-free shared-memory addresses; lanes past TX idle), else TX
  constexpr int RW = SX % 32 == 0 ? SX : TX;
  R* sq = reinterpret_cast<R*>(smem_raw);  // region A, stages 0-2: [4][QY][QP] primitives (row pitch QP)
  R* sxi = sq + L::nQ;                      //                         [SY][SX] flattening
  R* sfxh = sq;                             // region A, stages 3-4: [4][SY][TX+1] hat x fluxes
  R* sfyh = sq + L::nFXH;                   //                         [4][TY+1][SX] hat y fluxes
  R* sxl = sq + L::nA;                      // [4][SY][SX] left state at i+1/2 of each cell (then final Fx)
  R* sxr = sxl + L::nS;                     // right state at i-1/2
  R* syl = sxr + L::nS;                     // lower state at j+1/2 (then final Fy)
  R* syr = syl + L::nS;                     // upper state at j-1/2
  R* su = syr + L::nS;                      // [SY][SX] cell velocities for the viscosity
  R* sv = su + nC;
  R* sU = sv + nC;                          // [4][SY][SX] conserved values of the traced cells (FP32)

  const R sigx = f.sigx, sigy = f.sigy, hx = f.hx, hy = f.hy;
  const R ux = sigx, uy = sigy;  // update factors dt/dx, dt/dy (Eq. 5)

  const int tid = threadIdx.x;
  const int x0 = P.ng + bx * TX;  // padded column of the first interior cell of the tile
  const int y0 = P.ng + by * TY;
  const size_t plane = (size_t)P.NY * P.pitch;

  // ---- 0. load the tile.  FUSED: ghost cells are taken from the interior cells the boundary conditions
  // map them to (the values a ghost fill would have written); otherwise the ghost cells are read as filled
  // and indices past the array are clamped (such cells only feed cells outside the grid)
  // FP32 tiles whose padded box lies where the array holds the values the step needs (FUSED: the interior,
  // so that no boundary map applies; otherwise the ghost-filled array) arrive by one TMA copy of the
  // [4][QY][QX] box into the primitive area and are converted there in place; other tiles are loaded cell
  // by cell.
  bool tma_tile = false;
  if constexpr (is_f32<R>()) {
    static_assert(QP == QX, "the TMA box is stored densely");
    tma_tile = tmap != nullptr && tile_box_ok<TX, TY, FUSED>(P, bx, by, sq);
  }
  if (tma_tile) {
    __shared__ unsigned long long tma_bar;
    const unsigned int bar = smem_addr(&tma_bar);
    if constexpr (PERSIST) {
      // a block that runs several tiles has read and written this shared memory through the generic
      // proxy; order those accesses before the copy's async-proxy writes
      fence_proxy_async_smem();
      __syncthreads();
    }
    const unsigned int polls = P.tma_polls ? P.tma_polls : TMA_WAIT_POLLS;
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_arrive_expect_tx(bar, 4u * QX * QY * sizeof(R));
      if (!P.tma_test_drop) tma_load_3d(smem_addr(sq), tmap, x0 - 4, y0 - 4, 0, bar);
    }
    __syncthreads();
    const bool landed = mbar_wait(bar, 0, polls);
    if (__syncthreads_or(!landed)) {
      // the copy did not complete within the poll budget: report it, give it one more budget to land
      // (the shared memory should not be released under it) and leave this tile.  If it has not landed after
      // that either, say so apart: the step's output is then to be discarded, and so is anything a later
      // block on this SM computed while the copy could still arrive
      cnt.flags |= STATUS_TIMEOUT;
      const bool late = !mbar_wait(bar, 0, polls);
      if (__syncthreads_or(late)) cnt.flags |= STATUS_TIMEOUT_INFLIGHT;
      if (tid == 0) mbar_inval(bar);
      return;
    }
    for (int e = tid; e < QX * QY; e += NT) {
      const int lx = e % QX, ly = e / QX;
      const int d = ly * QP + lx;
      const R U0 = sq[d], U1 = sq[QP * QY + d], U2 = sq[2 * QP * QY + d], U3 = sq[3 * QP * QY + d];
      R rho, u, v, p;
      cons_to_prim(s, U0, U1, U2, U3, rho, u, v, p);
      if (lx >= 3 && lx < SX + 3 && ly >= 3 && ly < SY + 3) {
        const int c = (ly - 3) * SX + (lx - 3);
        Quad<R, nC>::st(sU, c, U0, U1, U2, U3);
      }
      sq[d] = rho;
      sq[QP * QY + d] = u;
      sq[2 * QP * QY + d] = v;
      sq[3 * QP * QY + d] = p;
    }
    __syncthreads();
    if (tid == 0) mbar_inval(bar);  // every thread has passed the wait; the next tile initialises it again
  } else {
    // a thread's cells in groups of two: both cells' loads are issued before either is converted, so their
    // latencies overlap, while the values in flight stay few enough to keep the stages' registers free of
    // spills (all of a thread's cells at once held up to 16 loads)
    constexpr int NLD = (QX * QY + NT - 1) / NT, CH = 2;
#pragma unroll 1
    for (int c0 = 0; c0 < NLD; c0 += CH) {
      R Ul[CH][4];
#pragma unroll
      for (int it = 0; it < CH; ++it) {
        const int e = tid + (c0 + it) * NT;
        if (e < QX * QY) {
          const int gi = x0 - 4 + e % QX, gj = y0 - 4 + e / QX;
          if (FUSED && P.bc_general) {  // reflecting or hydrostatic sides: the ghost fill's values
            R v[4];
            bc_cell_clamped(P, Uin, gi, gj, plane, v);
#pragma unroll
            for (int k = 0; k < 4; ++k) Ul[it][k] = v[k];
          } else {
            const size_t o = cell_offset<FUSED>(P, gi, gj);
#pragma unroll
            for (int k = 0; k < 4; ++k) Ul[it][k] = __ldg(Uin + o + k * plane);
          }
        }
      }
#pragma unroll
      for (int it = 0; it < CH; ++it) {
        const int e = tid + (c0 + it) * NT;
        if (e < QX * QY) {
          const int lx = e % QX, ly = e / QX;
          R rho, u, v, p;
          cons_to_prim(s, Ul[it][0], Ul[it][1], Ul[it][2], Ul[it][3], rho, u, v, p);
          if constexpr (L::SMEM_U) {
            if (lx >= 3 && lx < SX + 3 && ly >= 3 && ly < SY + 3) {
              const int c = (ly - 3) * SX + (lx - 3);
              Quad<R, nC>::st(sU, c, Ul[it][0], Ul[it][1], Ul[it][2], Ul[it][3]);
            }
          }
          const int d = ly * QP + lx;
          sq[d] = rho;
          sq[QP * QY + d] = u;
          sq[2 * QP * QY + d] = v;
          sq[3 * QP * QY + d] = p;
        }
      }
    }
    __syncthreads();
  }

  __shared__ int queue_n[2];  // gated faces queued by a FACE_LEARNED tile in stages 3 and 4
  if (face_kind(MODE) == FACE_LEARNED && tid == 0) queue_n[0] = queue_n[1] = 0;
  const R* qu = sq + QP * QY;
  const R* qv = sq + 2 * QP * QY;
  const R* qp = sq + 3 * QP * QY;
  // ---- 1. flattening xi = min(xi_x, xi_y) on cells lx in [3, TX+5), ly in [3, TY+5); keep u, v there
  for (int e = tid; e < nC; e += NT) {
    const int cx = e % SX + 3, cy = e / SX + 3;
    const int b = cy * QP + cx;
    R xi = (R)1;
    if (s.flatten) {
      auto chix = [&](int m) {
        return flatten_chi<R>(qp[b + m - 2], qp[b + m - 1], qp[b + m + 1], qp[b + m + 2], qu[b + m - 1], qu[b + m + 1],
                              s.small_pres);
      };
      auto chiy = [&](int m) {
        return flatten_chi<R>(qp[b + (m - 2) * QP], qp[b + (m - 1) * QP], qp[b + (m + 1) * QP], qp[b + (m + 2) * QP],
                              qv[b + (m - 1) * QP], qv[b + (m + 1) * QP], s.small_pres);
      };
      const int sx = (qp[b + 1] - qp[b - 1]) >= (R)0 ? 1 : -1;
      const int sy = (qp[b + QP] - qp[b - QP]) >= (R)0 ? 1 : -1;
      const R xix = M<R>::mn(chix(0), chix(-sx));
      const R xiy = M<R>::mn(chiy(0), chiy(-sy));
      xi = M<R>::mn(xix, xiy);
    }
    sxi[e] = xi;
    su[e] = qu[b];
    sv[e] = qv[b];
  }
  __syncthreads();

  // ---- 2. slopes + tracing for the same cells; items [0, nC) trace in x, [nCa, nCa + nC) in y (the y
  // items start at a warp boundary, so the direction is uniform over a warp and each direction's code has
  // its shared-memory offsets as constants)
  {
    auto trace_cell = [&](auto ydir, int c) {
      constexpr bool YD = decltype(ydir)::value;
      constexpr int st = YD ? QP : 1;
      // face frame (rho, un, ut, p) -> planes of the (rho, u, v, p) arrays; in y un = v, ut = u
      constexpr int k1 = YD ? 2 : 1, k2 = YD ? 1 : 2;
      const int b = (c / SX + 3) * QP + c % SX + 3;
      const R xi = sxi[c];
      R q[4], ql[4], qrr[4];
      if constexpr ((MODE & RECON_PPM) != 0) {
        R eL[4], eR[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int k = m == 0 ? 0 : m == 1 ? k1 : m == 2 ? k2 : 3;
          const R* a = sq + k * QP * QY + b;
          q[m] = a[0];
          ppm_edges<R>(a[-2 * st], a[-st], a[0], a[st], a[2 * st], xi, eL[m], eR[m]);
        }
        trace_ppm<R>(s, YD ? sigy : sigx, q, eL, eR, ql, qrr);
      } else {
        R dq[4];
        if constexpr (is_f32<R>()) {
          // components in pairs (rho, un) and (ut, p), each pair's limiter in packed arithmetic
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const R* a = sq + (h == 0 ? 0 : k2) * QP * QY + b;
            const R* c = sq + (h == 0 ? k1 : 3) * QP * QY + b;
            q[2 * h] = a[0];
            q[2 * h + 1] = c[0];
            const float2 d = mul2(f2(xi), slope_pair(s.limiter, f2(a[-2 * st], c[-2 * st]), f2(a[-st], c[-st]),
                                                      f2(a[0], c[0]), f2(a[st], c[st]), f2(a[2 * st], c[2 * st])));
            dq[2 * h] = d.x;
            dq[2 * h + 1] = d.y;
          }
        } else {
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const int k = m == 0 ? 0 : m == 1 ? k1 : m == 2 ? k2 : 3;
            const R* a = sq + k * QP * QY + b;
            q[m] = a[0];
            dq[m] = xi * slope<R>(s.limiter, a[-2 * st], a[-st], a[0], a[st], a[2 * st]);
          }
        }
        trace<R>(s, YD ? sigy : sigx, q, dq, ql, qrr);
      }
      if (P.use_grav) {  // half-step gravity (the rho g source, §3.2) on v: normal in y, transverse in x
        constexpr int mg = YD ? 1 : 2;
        ql[mg] = ql[mg] + f.hdtg;
        qrr[mg] = qrr[mg] + f.hdtg;
      }
      // stored in (rho, u, v, p) order
      if constexpr (YD) {
        Quad<R, nC>::st(syl, c, ql[0], ql[2], ql[1], ql[3]);
        Quad<R, nC>::st(syr, c, qrr[0], qrr[2], qrr[1], qrr[3]);
      } else {
        Quad<R, nC>::st(sxl, c, ql[0], ql[1], ql[2], ql[3]);
        Quad<R, nC>::st(sxr, c, qrr[0], qrr[1], qrr[2], qrr[3]);
      }
    };
    constexpr int nCa = (nC + 31) / 32 * 32;
    for (int e = tid; e < nCa + nC; e += NT) {
      if (e < nCa) {
        if (e < nC) trace_cell(std::false_type{}, e);
      } else {
        trace_cell(std::true_type{}, e - nCa);
      }
    }
  }
  __syncthreads();

  // FACE_LEARNED: faces past the network's gate are not solved in the face loops.  Each is queued in a small
  // shared array of its own (face item and, later, starting pressure; LEARNED_QUEUE entries), the other faces
  // are solved at once from the acoustic start, and after the stage's barrier the network proposes the
  // starting pressures of the queued faces, 32 per warp, which are then solved from them (a tile with no
  // gated face skips this, and its barriers are those of the plain kernel).  The face loops thus carry no
  // call and keep the registers of the plain kernel, and a warp evaluates the network on 32 gated faces
  // rather than on the 31 others of a warp that holds one.  The queued faces' states are rebuilt from the
  // traced states, which stay in place until each face's own flux replaces them.  A full queue leaves
  // further gated faces to the acoustic start.
  constexpr bool LEARNED = face_kind(MODE) == FACE_LEARNED;
  float* queue = nullptr;
  float gate_ratio = 0.f, gate_u4 = 0.f;
  if constexpr (LEARNED) {
    queue = learned_queue();
    gate_ratio = wsm->gate_ratio;
    gate_u4 = wsm->gate_u4;
  }
  // queue the face of item e of stage st (0: 3, 1: 4) if it is past the gate; false if it is solved in the loop
  auto defer = [&](int st, int e, const R a[4], const R b[4]) -> bool {
    if constexpr (LEARNED) {
      if (!strong_face(a, b, gate_ratio, gate_u4)) return false;
      const int k = atomicAdd(&queue_n[st], 1);
      if (k >= LEARNED_QUEUE) return false;
      queue[2 * k] = __int_as_float(e);
      return true;
    } else {
      return false;
    }
  };
  // the network's starting pressures for the queued faces, then their solves (block-wide, called only when
  // the queue, filled before a barrier, holds a face); states(e, isx, a, b) rebuilds an item's face states,
  // finish(e, isx, F) stores its flux
  auto learned_pass = [&](int st, int nXIa, auto&& states, auto&& finish) {
    if constexpr (LEARNED) {
      const int n = queue_n[st] < LEARNED_QUEUE ? queue_n[st] : LEARNED_QUEUE;
      for (int b0 = tid - (tid & 31); b0 < n; b0 += NT) {  // warp-uniform: the forward pass is warp-collective
        const int k = b0 + (tid & 31);
        float x[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float pref = 0.f;
        if (k < n) {
          const int e = __float_as_int(queue[2 * k]);
          R a[4], b[4];
          states(e, e < nXIa, a, b);
          pref = mlp_features(a[0], a[1], a[3], b[0], b[1], b[3], x);
        }
        float y = mlp_warp_forward(x, wsm, n - b0);
        y = fminf(fmaxf(y, -40.f), 40.f);
        if (k < n) queue[2 * k + 1] = pref * __expf(y);
      }
      __syncthreads();
      for (int k = tid; k < n; k += NT) {
        const int e = __float_as_int(queue[2 * k]);
        const bool isx = e < nXIa;
        R a[4], b[4], F[4];
        states(e, isx, a, b);
        int it;
        bool ok;
        if constexpr (PERSIST)  // ensembles: passes are frequent (quadrant interfaces), the call would cost more
          riemann(s, a, b, queue[2 * k + 1], F, it, ok);
        else
          riemann_out(s.gamma, s.g1, s.igm1, s.small_pres, s.tol, s.maxiter, a[0], a[1], a[2], a[3], b[0], b[1], b[2],
                      b[3], queue[2 * k + 1], F, it, ok);
        cnt.solves++;
        cnt.iters += it;
        cnt.nonconv += ok ? 0 : 1;
        finish(e, isx, F);
      }
    }
  };
  constexpr int FACE_LOOP_MODE = LEARNED ? (MODE & ~3) | FACE_PLAIN : MODE;

  // ---- 3. hat Riemann solves.  x faces: lx in [4, TX+5) between cells lx-1 and lx, rows [3, TY+5).
  //         y faces: ly in [4, TY+5), columns [3, TX+5).  Results overwrite region A.
  {
    // x-face items run over rows of SX (the last item of each row idle) so a warp's shared-memory reads
    // stay on consecutive addresses of the SX-wide arrays; y-face items start at a warp boundary
    constexpr int nXI = SX * SY, nXIa = (nXI + 31) / 32 * 32, nYF = (TY + 1) * SX;
    auto states = [&](int e, bool isx, R a[4], R bq[4]) {
      if (isx) {
        // face fx = e % SX (0..TX) <-> lx = fx + 4 in row ly = e / SX + 3; cell lx-1 has s index e
        const int cL = e;
        const int cR = cL + 1;
        Quad<R, nC>::ld(sxl, cL, a);
        Quad<R, nC>::ld(sxr, cR, bq);
      } else {
        const int f = e - nXIa;                // = fy * SX + column s index; face 0..TY <-> ly = fy + 4
        const int cL = f;                      // cell ly-1 = fy + 3
        const int cR = cL + SX;
        R l[4], r[4];
        Quad<R, nC>::ld(syl, cL, l);
        Quad<R, nC>::ld(syr, cR, r);
        a[0] = l[0]; a[1] = l[2]; a[2] = l[1]; a[3] = l[3];
        bq[0] = r[0]; bq[1] = r[2]; bq[2] = r[1]; bq[3] = r[3];
      }
    };
    auto finish = [&](int e, bool isx, const R F[4]) {
      if (isx) {
        const int fx = e % SX, ry = e / SX;
        Quad<R, SY * (TX + 1)>::st(sfxh, ry * (TX + 1) + fx, F[0], F[1], F[2], F[3]);
      } else {
        Quad<R, (TY + 1) * SX>::st(sfyh, e - nXIa, F[0], F[2], F[1], F[3]);
      }
    };
    // warp-uniform trip count: every lane of a warp runs the same iterations (the harvest's gated faces and
    // the solver's fan test are warp-collective); lanes without a face only take part in them
    for (int e0 = tid - (tid & 31); e0 < nXIa + nYF; e0 += NT) {
      const int e = e0 + (tid & 31);
      const bool isx = e < nXIa;
      bool active = isx ? (e < nXI && e % SX <= TX) : (e - nXIa < nYF);
      R a[4] = {(R)1, (R)0, (R)0, (R)1}, bq[4] = {(R)1, (R)0, (R)0, (R)1}, F[4];
      if (active) {
        states(e, isx, a, bq);
        if (defer(0, e, a, bq)) active = false;
      }
      face_solve<R, FACE_LOOP_MODE>(s, a, bq, active, hook, face_key(bx, by, 0, e), F, cnt);
      if (active) finish(e, isx, F);
    }
    __syncthreads();
    // the queued faces, if the tile has any, after the stage's own barrier (one more barrier only then)
    if constexpr (LEARNED) {
      if (queue_n[0] > 0) {  // block-uniform: read after the barrier
        learned_pass(0, nXIa, states, finish);
        __syncthreads();
      }
    }
  }

  // ---- 4. transverse correction + final solves + artificial viscosity at the tile's faces
  {
    // as in stage 3: x-face items over rows of SX, y-face items from a warp boundary, over rows of RW
    constexpr int nXI = SX * TY, nXIa = (nXI + 31) / 32 * 32, nYF = (TY + 1) * RW;
    auto states = [&](int e, bool isx, R a[4], R bq[4]) {
      if (isx) {
        const int fx = e % SX, ty = e / SX;  // face lx = fx + 4, row ly = ty + 4
        const int cL = (ty + 1) * SX + fx, cR = cL + 1;  // s indices of cells lx-1 and lx
        // hat y fluxes of columns lx-1 and lx at faces ly (j-1/2) and ly+1 (j+1/2): index fy = ly - 4
        const int fL = ty * SX + fx, fR = fL + 1;
        using FY = Quad<R, (TY + 1) * SX>;
        R dL[4], dR[4], t0[4], t1[4], l[4], r[4];
        FY::ld(sfyh, fL + SX, t1);
        FY::ld(sfyh, fL, t0);
        sub4(t1, t0, dL);
        FY::ld(sfyh, fR + SX, t1);
        FY::ld(sfyh, fR, t0);
        sub4(t1, t0, dR);
        Quad<R, nC>::ld(sxl, cL, l);
        Quad<R, nC>::ld(sxr, cR, r);
        correct_state(s, l[0], l[1], l[2], l[3], dL, hy, a);
        correct_state(s, r[0], r[1], r[2], r[3], dR, hy, bq);
      } else {
        const int f = e - nXIa;
        const int tx = f % RW, fy = f / RW;  // column lx = tx + 4, face ly = fy + 4
        const int cL = fy * SX + tx + 1, cR = cL + SX;  // cells ly-1 and ly of column lx
        // hat x fluxes of rows ly-1 and ly at faces lx (i-1/2) and lx+1 (i+1/2): row index ry = ly - 3
        const int fL = fy * (TX + 1) + tx, fR = fL + (TX + 1);
        using FX = Quad<R, SY * (TX + 1)>;
        R dL[4], dR[4], t0[4], t1[4], l[4], r[4];
        FX::ld(sfxh, fL + 1, t1);
        FX::ld(sfxh, fL, t0);
        sub4(t1, t0, dL);
        FX::ld(sfxh, fR + 1, t1);
        FX::ld(sfxh, fR, t0);
        sub4(t1, t0, dR);
        R ql[4], qrr[4];
        Quad<R, nC>::ld(syl, cL, l);
        Quad<R, nC>::ld(syr, cR, r);
        correct_state(s, l[0], l[1], l[2], l[3], dL, hx, ql);
        correct_state(s, r[0], r[1], r[2], r[3], dR, hx, qrr);
        a[0] = ql[0]; a[1] = ql[2]; a[2] = ql[1]; a[3] = ql[3];
        bq[0] = qrr[0]; bq[1] = qrr[2]; bq[2] = qrr[1]; bq[3] = qrr[3];
      }
    };
    auto finish = [&](int e, bool isx, const R F[4]) {
      if (isx) {
        const int fx = e % SX, ty = e / SX;
        const int cL = (ty + 1) * SX + fx, cR = cL + 1;
        R G[4] = {F[0], F[1], F[2], F[3]};
        // artificial viscosity from the cell-centred velocities of the time-n state
        if (s.cvisc > (R)0) {
          R div;
          const R dvy = sv[cR + SX] + sv[cL + SX] - sv[cR - SX] - sv[cL - SX];
          if constexpr (is_f32<R>())
            div = (su[cR] - su[cL]) * s.idx + dvy * (0.25f * s.idy);
          else
            div = (su[cR] - su[cL]) / s.dx + dvy / (4.0 * s.dy);
          const R av = s.cvisc * M<R>::mx(-div * s.dx, (R)0);
          if constexpr (L::SMEM_U) {
            R uL[4], uR[4], du[4];
            Quad<R, nC>::ld(sU, cL, uL);
            Quad<R, nC>::ld(sU, cR, uR);
            sub4(uL, uR, du);
            axpy4(av, du, G);
          } else {
            const int gi = x0 + fx, gj = y0 + ty;  // padded index of cell lx
            R uL[4], uR[4];
            tile_cell<FUSED>(P, Uin, gi - 1, gj, plane, uL);
            tile_cell<FUSED>(P, Uin, gi, gj, plane, uR);
#pragma unroll
            for (int k = 0; k < 4; ++k) G[k] += av * (uL[k] - uR[k]);
          }
        }
        Quad<R, nC>::st(sxl, cL, G[0], G[1], G[2], G[3]);  // only this face read sxl[cL]
      } else {
        const int f = e - nXIa;
        const int tx = f % RW, fy = f / RW;  // column lx = tx + 4, face ly = fy + 4
        const int cL = fy * SX + tx + 1, cR = cL + SX;  // cells ly-1 and ly of column lx
        R G[4] = {F[0], F[2], F[1], F[3]};
        if (s.cvisc > (R)0) {
          R div;
          const R dux = (su[cR + 1] + su[cL + 1] - su[cR - 1] - su[cL - 1]);
          if constexpr (is_f32<R>())
            div = (sv[cR] - sv[cL]) * s.idy + dux * (0.25f * s.idx);
          else
            div = (sv[cR] - sv[cL]) / s.dy + dux / (4.0 * s.dx);
          const R av = s.cvisc * M<R>::mx(-div * s.dy, (R)0);
          if constexpr (L::SMEM_U) {
            R uL[4], uR[4], du[4];
            Quad<R, nC>::ld(sU, cL, uL);
            Quad<R, nC>::ld(sU, cR, uR);
            sub4(uL, uR, du);
            axpy4(av, du, G);
          } else {
            const int gi = x0 + tx, gj = y0 + fy;  // padded index of cell (lx, ly)
            R uL[4], uR[4];
            tile_cell<FUSED>(P, Uin, gi, gj - 1, plane, uL);
            tile_cell<FUSED>(P, Uin, gi, gj, plane, uR);
#pragma unroll
            for (int k = 0; k < 4; ++k) G[k] += av * (uL[k] - uR[k]);
          }
        }
        Quad<R, nC>::st(syl, cL, G[0], G[1], G[2], G[3]);  // only this face read syl[cL]
      }
    };
    for (int e0 = tid - (tid & 31); e0 < nXIa + nYF; e0 += NT) {
      const int e = e0 + (tid & 31);
      const bool isx = e < nXIa;
      bool active = isx ? (e < nXI && e % SX <= TX) : (e - nXIa < nYF && (e - nXIa) % RW < TX);
      R a[4] = {(R)1, (R)0, (R)0, (R)1}, bq[4] = {(R)1, (R)0, (R)0, (R)1}, F[4];
      if (active) {
        states(e, isx, a, bq);
        if (defer(1, e, a, bq)) active = false;
      }
      face_solve<R, FACE_LOOP_MODE>(s, a, bq, active, hook, face_key(bx, by, 1, e), F, cnt);
      if (active) finish(e, isx, F);
    }
    __syncthreads();
    // the queued faces, if the tile has any, after the stage's own barrier (one more barrier only then)
    if constexpr (LEARNED) {
      if (queue_n[1] > 0) {  // block-uniform: read after the barrier
        learned_pass(1, nXIa, states, finish);
        __syncthreads();
      }
    }
  }

  // ---- 5. conservative update of the tile's valid cells
  unsigned int& flags = cnt.flags;
  for (int e = tid; e < RW * TY; e += NT) {
    const int tx = e % RW, ty = e / RW;
    const int gi = x0 + tx, gj = y0 + ty;
    if (tx >= TX || gi >= P.ng + P.nx || gj >= P.ng + P.ny) continue;
    const size_t o = (size_t)gj * P.pitch + gi;
    const int cx = (ty + 1) * SX + tx;  // final x flux of face tx (left of cell) lives in sxl[cx]
    const int cy = ty * SX + tx + 1;    // final y flux of face ty (below the cell) lives in syl[cy]
    R Un[4], rho_n, my_n, fx0[4], fx1[4], fy0[4], fy1[4], un[4];
    Quad<R, nC>::ld(sxl, cx, fx0);
    Quad<R, nC>::ld(sxl, cx + 1, fx1);
    Quad<R, nC>::ld(syl, cy, fy0);
    Quad<R, nC>::ld(syl, cy + SX, fy1);
    if constexpr (L::SMEM_U) {
      Quad<R, nC>::ld(sU, cy + SX, un);  // the cell's own U^n, s index (ty + 1) * SX + tx + 1
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) un[k] = __ldg(Uin + o + k * plane);
    }
    rho_n = un[0];
    my_n = un[2];
    if constexpr (is_f32<R>()) {
      // (rho, rho u) and (rho v, E) in packed arithmetic
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 dx = sub2(f2(fx0[2 * h], fx0[2 * h + 1]), f2(fx1[2 * h], fx1[2 * h + 1]));
        const float2 dy = sub2(f2(fy0[2 * h], fy0[2 * h + 1]), f2(fy1[2 * h], fy1[2 * h + 1]));
        const float2 d = fma2(f2(ux), dx, mul2(f2(uy), dy));
        const float2 n = add2(f2(un[2 * h], un[2 * h + 1]), d);
        Un[2 * h] = n.x;
        Un[2 * h + 1] = n.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const R d = ux * (fx0[k] - fx1[k]) + uy * (fy0[k] - fy1[k]);
        Un[k] = un[k] + d;
      }
    }
    if (P.use_grav) {
      // time-centred gravity sources (§3.2): rho v gains dt g (rho^n + rho^{n+1}) / 2, then rho E gains
      // dt g ((rho v)^n + (rho v)^{n+1}) / 2 with the updated momentum
      Un[2] = Un[2] + f.hdtg * (rho_n + Un[0]);
      Un[3] = Un[3] + f.hdtg * (my_n + Un[2]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) Uout[o + k * plane] = Un[k];
    if constexpr (FUSED) {
      // the CFL constraint of the new state (Eq. 6), for the next step's time step
      cfl_value(s, Un[0], Un[1], Un[2], Un[3], *cfl_min, flags);
    } else if (!finite4(Un[0], Un[1], Un[2], Un[3])) {
      flags |= STATUS_NONFINITE;
    } else {
      const R ke = M<R>::dv((R)0.5 * (Un[1] * Un[1] + Un[2] * Un[2]), Un[0]);
      if (!(Un[0] > (R)0) || !(Un[3] - ke > (R)0)) flags |= STATUS_NEGATIVE;
    }
  }
}

}  // namespace hydro
