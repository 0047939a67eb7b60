// Single-problem CTU step kernels and their launch templates: one CTA per tile (the tile itself is in
// ctu_tile.cuh).  Instantiated for FP32 in k_ctu.cu and for FP64 in k_ctu_f64.cu, which is compiled without
// multiply-add contraction.
#pragma once
#include <float.h>

#include <atomic>

#include "ctu_tile.cuh"
#include "hydro_kernels.h"

namespace hydro {

// Per-block reduction of the tile counters into the context's scratch: warp shuffles, then one thread adds
// the block's sums (one atomic per counter and block; per-warp atomics on the same words cost ~4 % of a
// KH 1024^2 step).  Called by every thread of the block.
template <int NT>
__device__ __forceinline__ void flush_counters(TileCounters& cnt, DevScratch* scr) {
  if (cnt.nonconv) cnt.flags |= STATUS_NONCONV;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    cnt.solves += __shfl_xor_sync(0xffffffffu, cnt.solves, off);
    cnt.iters += __shfl_xor_sync(0xffffffffu, cnt.iters, off);
    cnt.nonconv += __shfl_xor_sync(0xffffffffu, cnt.nonconv, off);
    cnt.flags |= __shfl_xor_sync(0xffffffffu, cnt.flags, off);
  }
  __shared__ unsigned int part[NT / 32][4];
  if ((threadIdx.x & 31) == 0) {
    const int w = threadIdx.x >> 5;
    part[w][0] = cnt.solves;
    part[w][1] = cnt.iters;
    part[w][2] = cnt.nonconv;
    part[w][3] = cnt.flags;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long solves = 0, iters = 0, nonconv = 0;
    unsigned int flags = 0;
    for (int w = 0; w < NT / 32; ++w) {
      solves += part[w][0];
      iters += part[w][1];
      nonconv += part[w][2];
      flags |= part[w][3];
    }
    atomicAdd(&scr->stats[0], solves);
    atomicAdd(&scr->stats[1], iters);
    if (nonconv) atomicAdd(&scr->stats[2], nonconv);
    if (flags) atomicOr(&scr->status, flags);
  }
}

// Tile of the single-problem FP32 kernels (overridable at compile time for tile sweeps; the TMA box of the
// state buffers is encoded for it).  Measured on KH
// 1024^2 and Sedov 2048^2 at 256 threads: 32x16 (3 CTAs per SM) beats 30x16 (warp-aligned rows but a ragged
// last tile on power-of-two grids), 30x8 and 14x16 by 1-2%, and 30x24/384, 62x8 and 30x32/512 (fewer warps
// per SM) by 4-40%.  With 384 threads (36 warps per SM at 56 registers) 32x16 gains another 6-8%; more
// threads per tile force spills or fewer tiles per SM and lose.
#ifndef HYDRO_F32_TX
#define HYDRO_F32_TX 32
#endif
#ifndef HYDRO_F32_TY
#define HYDRO_F32_TY 16
#endif
#ifndef HYDRO_F32_NT
#define HYDRO_F32_NT 384
#endif
constexpr int F32_TX = HYDRO_F32_TX, F32_TY = HYDRO_F32_TY, F32_NT = HYDRO_F32_NT;

#ifndef HYDRO_F32_MINB
#define HYDRO_F32_MINB 3
#endif
// Resident blocks per SM the register allocator must allow: shared memory admits three tiles per SM in
// both precisions, and three blocks of 384 (FP32) or 256 (FP64) threads need <= 56 or <= 85 registers.
template <typename R>
constexpr int min_blocks() {
  return is_f32<R>() ? HYDRO_F32_MINB : 3;
}

template <typename R, int TX, int TY, int NT, int MODE>
__global__ void __launch_bounds__(NT, min_blocks<R>()) ctu_step_kernel(KParams P, const R* __restrict__ Uin, R* __restrict__ Uout,
                                                      StepScalars sc_host, const StepScalars* __restrict__ sc_dev,
                                                      DevScratch* __restrict__ scr, FaceHook hook,
                                                      const __grid_constant__ CUtensorMap tmap, int use_tma) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the network's weights are read from global memory (L1/L2-resident) only by warps whose gate opens,
  // which is rare in smooth flow, so no CTA pays to stage them
  const MlpBlob* wsm = face_kind(MODE) == FACE_LEARNED ? hook.mlp : nullptr;
  SP<R> s;
  s.load(P);
  StepFactors<R> f;
  f.load(sc_dev ? *sc_dev : sc_host);
  TileCounters cnt;
  ctu_tile<R, TX, TY, NT, MODE>(P, s, f, Uin, Uout, blockIdx.x, blockIdx.y, smem_raw, cnt, hook, wsm, nullptr,
                                use_tma ? &tmap : nullptr);
  flush_counters<NT>(cnt, scr);
}

// Raises a kernel's dynamic shared-memory limit once per device (function attributes belong to the device's
// context); later calls on the same device only test a bit.  Devices beyond 63 set it on every call.
template <typename K>
cudaError_t smem_attr_once(K kernel, size_t smem, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_relaxed);
  return e;
}

template <typename R, int TX, int TY, int NT, int MODE>
cudaError_t launch_ctu_step(const KParams& P, const R* Uin, R* Uout, const StepScalars& sc_host,
                            const StepScalars* sc_dev, DevScratch* scr, const FaceHook& hook, const CUtensorMap* tmap,
                            cudaStream_t stream) {
  const size_t smem = TileLayout<R, TX, TY>::bytes;
  static std::atomic<unsigned long long> attr_done{0};
  cudaError_t e = smem_attr_once(ctu_step_kernel<R, TX, TY, NT, MODE>, smem, attr_done);
  if (e != cudaSuccess) return e;
  dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
  ctu_step_kernel<R, TX, TY, NT, MODE><<<grid, NT, smem, stream>>>(P, Uin, Uout, sc_host, sc_dev, scr, hook,
                                                                    tmap ? *tmap : CUtensorMap{}, tmap ? 1 : 0);
  return cudaGetLastError();
}

// Fused step: the tile reads ghost cells through the boundary map and folds the CFL constraint of its new
// cells into a block minimum; the last block to finish advances the time by this step's dt and writes
// the next step's factors, so a run needs one launch per step and no ghost-fill or dt pass.  A step may be
// split into launches over bands of tile rows (by0: the band's first tile row; nblocks: the tiles of the
// whole step), which run concurrently; the last block of all of them finishes the step.
template <typename R, int TX, int TY, int NT, int MODE = FACE_PLAIN>
__global__ void __launch_bounds__(NT, min_blocks<R>()) ctu_step_fused_kernel(KParams P, const R* __restrict__ Uin,
                                                            R* __restrict__ Uout, const StepScalars* __restrict__ sc_cur,
                                                            StepScalars* __restrict__ sc_next,
                                                            DevScratch* __restrict__ scr, double tmax,
                                                            const __grid_constant__ CUtensorMap tmap, int use_tma,
                                                            int by0, unsigned int nblocks,
                                                            const MlpBlob* __restrict__ mlp) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // FACE_LEARNED: the network's weights (read from global memory by the warps whose gate opens)
  const MlpBlob* wsm = face_kind(MODE) == FACE_LEARNED ? mlp : nullptr;
  SP<R> s;
  s.load(P);
  StepFactors<R> f;
  f.load(*sc_cur);
  TileCounters cnt;
  R cmin = is_f32<R>() ? (R)FLT_MAX : (R)DBL_MAX;
  const int by = by0 + (int)blockIdx.y;
  if (sc_cur->dt == 0.0) {
    // a step of length zero (the run has reached tmax) leaves the state as it is: copy the tile's interior
    // cells and take their CFL constraint as a step would (the next dt is then clamped to 0 again)
    const size_t plane = (size_t)P.NY * P.pitch;
    for (int e = threadIdx.x; e < TX * TY; e += NT) {
      const int gi = P.ng + blockIdx.x * TX + e % TX, gj = P.ng + by * TY + e / TX;
      if (gi >= P.ng + P.nx || gj >= P.ng + P.ny) continue;
      const size_t o = (size_t)gj * P.pitch + gi;
      R u[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) Uout[o + k * plane] = u[k] = Uin[o + k * plane];
      cfl_value(s, u[0], u[1], u[2], u[3], cmin, cnt.flags);
    }
  } else {
    ctu_tile<R, TX, TY, NT, MODE, true>(P, s, f, Uin, Uout, blockIdx.x, by, smem_raw, cnt, FaceHook{}, wsm,
                                        &cmin, use_tma ? &tmap : nullptr);
  }
  flush_counters<NT>(cnt, scr);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const R o = __shfl_xor_sync(0xffffffffu, cmin, off);
    cmin = o < cmin ? o : cmin;
  }
  __shared__ R wmin[NT / 32];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = cmin;
  __syncthreads();
  if (threadIdx.x == 0) {
    R b = wmin[0];
    for (int k = 1; k < NT / 32; ++k) b = wmin[k] < b ? wmin[k] : b;
    atomicMin(&scr->dtn_min_bits, (unsigned long long)__double_as_longlong((double)b));
    __threadfence();
    last = atomicAdd(&scr->step_blocks_done, 1u) == nblocks - 1u;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const unsigned long long bits =
        atomicExch(&scr->dtn_min_bits, (unsigned long long)__double_as_longlong(DBL_MAX));
    const double t = scr->t + sc_cur->dt;
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

// band: tile rows [band.x, band.x + band.y) of the step (band.y <= 0: all of them).  mlp: the network of
// MODE FACE_LEARNED (device).
template <typename R, int TX, int TY, int NT, int MODE = FACE_PLAIN>
cudaError_t launch_ctu_step_fused(const KParams& P, const R* Uin, R* Uout, const StepScalars* sc_cur,
                                  StepScalars* sc_next, DevScratch* scr, double tmax, const CUtensorMap* tmap,
                                  cudaStream_t stream, int2 band = make_int2(0, 0), const MlpBlob* mlp = nullptr) {
  const size_t smem = TileLayout<R, TX, TY>::bytes;
  static std::atomic<unsigned long long> attr_done{0};
  cudaError_t e = smem_attr_once(ctu_step_fused_kernel<R, TX, TY, NT, MODE>, smem, attr_done);
  if (e != cudaSuccess) return e;
  const int tx = (P.nx + TX - 1) / TX, ty = (P.ny + TY - 1) / TY;
  const int y0 = band.y > 0 ? band.x : 0, ny = band.y > 0 ? band.y : ty;
  if (y0 < 0 || ny <= 0 || y0 + ny > ty) return cudaErrorInvalidValue;
  dim3 grid(tx, ny);
  ctu_step_fused_kernel<R, TX, TY, NT, MODE><<<grid, NT, smem, stream>>>(
      P, Uin, Uout, sc_cur, sc_next, scr, tmax, tmap ? *tmap : CUtensorMap{}, tmap ? 1 : 0, y0,
      (unsigned int)tx * (unsigned int)ty, mlp);
  return cudaGetLastError();
}

}  // namespace hydro
