// Batched kernels for ensembles of independent problems on uneven grids (one problem per member, each with
// its own CFL time step): a dt reduction over all members at once, and a persistent fused CTU
// step kernel whose CTAs pull tiles of any member from a work queue.  The step reads cells outside each
// member's domain through its boundary map and folds the CFL constraint of its new cells into the member's
// accumulator; the member's last tile advances its time and writes its next step's factors, so a run needs
// one dt pass at its start and then one launch per step and tile shape.  Instantiated for FP32 in k_batch.cu and for
// FP64 in k_batch_f64.cu, which is compiled without multiply-add contraction.
#pragma once
#include <float.h>

#include <atomic>

#include "ctu_tile.cuh"
#include "hydro_batch_internal.h"

namespace hydro {

// ---------------------------------------------------------------------------------------------------
// CFL dt of every member.  Block b reduces BATCH_DT_CELLS cells of member tab[b].x from cell tab[b].y;
// tab[b].z is the member's block count, so the member's last block finalises its dt, step factors and
// time, and resets the member's accumulator.
template <typename R>
__global__ void __launch_bounds__(256) batch_dt_kernel(const BatchMember* __restrict__ mem, const int4* __restrict__ tab,
                                                      int parity, int advance) {
  const int4 t = tab[blockIdx.x];
  const BatchMember& m = mem[t.x];
  const KParams& P = m.P;
  const R* U = (const R*)m.U[parity];
  DevScratch* scr = m.scr;
  SP<R> s;
  s.load(P);
  const size_t plane = (size_t)P.NY * P.pitch;
  const int ncell = P.nx * P.ny;
  R rbest = is_f32<R>() ? (R)FLT_MAX : (R)DBL_MAX;
  unsigned int flags = 0;
  const int end = min(t.y + BATCH_DT_CELLS, ncell);
  for (int e = t.y + threadIdx.x; e < end; e += 256) {
    const int j = e / P.nx, i = e % P.nx;
    cfl_cell(s, U, (size_t)(j + P.ng) * P.pitch + (i + P.ng), plane, rbest, flags);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const R o = __shfl_xor_sync(0xffffffffu, rbest, off);
    rbest = o < rbest ? o : rbest;
    flags |= __shfl_xor_sync(0xffffffffu, flags, off);
  }
  __shared__ R wmin[8];
  __shared__ unsigned int wflags[8];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) {
    wmin[threadIdx.x >> 5] = rbest;
    wflags[threadIdx.x >> 5] = flags;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    R b = wmin[0];
    unsigned int f = wflags[0];
    for (int k = 1; k < 8; ++k) {
      b = wmin[k] < b ? wmin[k] : b;
      f |= wflags[k];
    }
    atomicMin(&scr->dt_min_bits, (unsigned long long)__double_as_longlong((double)b));
    if (f) atomicOr(&scr->status, f);
    __threadfence();
    last = (atomicAdd(&scr->dt_blocks_done, 1u) == (unsigned int)t.z - 1u);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const unsigned long long bits = atomicExch(&scr->dt_min_bits, (unsigned long long)__double_as_longlong(DBL_MAX));
    const double dt = P.cfl * __longlong_as_double((long long)bits);
    scr->dt = dt;
    scr->sc = make_step_scalars(dt, P.dx, P.dy, P.grav);
    scr->scf[parity] = scr->sc;  // the factors the fused step at this parity reads
    if (advance) {
      scr->t = scr->t + dt;
      scr->nsteps = scr->nsteps + 1;
    }
    scr->dt_blocks_done = 0u;
  }
}

// ---------------------------------------------------------------------------------------------------
// One tile of a member is done: fold its CFL minimum into the member's accumulator; the member's last tile
// (of `ntiles`) turns the minimum into the next step's factors scf[1 - parity] and, if advance, adds this
// step to the member's time.  Not inlined: one thread per tile calls it, and the step loop's registers stay
// those of the tile.
static __device__ __noinline__ void member_tile_done(const BatchMember& m, double tile_min, int ntiles, int parity,
                                              int advance) {
  DevScratch* scr = m.scr;
  atomicMin(&scr->dtn_min_bits, (unsigned long long)__double_as_longlong(tile_min));
  __threadfence();
  if (atomicAdd(&scr->step_blocks_done, 1u) != (unsigned int)ntiles - 1u) return;
  __threadfence();
  const unsigned long long bits = atomicExch(&scr->dtn_min_bits, (unsigned long long)__double_as_longlong(DBL_MAX));
  if (advance) {
    scr->t = scr->t + scr->scf[parity].dt;
    scr->nsteps = scr->nsteps + 1;
  }
  const double dt = m.P.cfl * __longlong_as_double((long long)bits);
  scr->dt = dt;
  scr->sc = make_step_scalars(dt, m.P.dx, m.P.dy, m.P.grav);
  scr->scf[1 - parity] = scr->sc;
  scr->step_blocks_done = 0u;
}

// ---------------------------------------------------------------------------------------------------
// Persistent fused CTU step over a tile list (member, tile x, tile y, the member's tile count), largest
// members first: each CTA takes the next tile from an atomic queue until the list is exhausted.  A tile
// reads the member's factors scf[parity], folds its cells' CFL minimum into the member's accumulator, and
// the member's last tile sets its next factors scf[1 - parity] (and, if advance, its time and step count).
// MODE FACE_LEARNED: every member's Riemann iterations start from the learned proposal of the weights mlp,
// which the warps whose gate opens read from global memory (L1-resident; a shared-memory copy per CTA would
// cost the third CTA per SM).
template <typename R, int TX, int TY, int NT, int MODE = FACE_PLAIN>
__global__ void __launch_bounds__(NT, is_f32<R>() ? 3 : 2) batch_step_kernel(const BatchMember* __restrict__ mem,
                                                       const int4* __restrict__ tiles, int ntiles,
                                                       unsigned int* __restrict__ queue, int parity,
                                                       DevScratch* __restrict__ agg,
                                                       const CUtensorMap* __restrict__ tmaps, int advance,
                                                       const MlpBlob* __restrict__ mlp) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int cur;
  __shared__ R wmin[NT / 32];
  TileCounters cnt;
  while (true) {
    if (threadIdx.x == 0) cur = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int k = cur;
    if (k >= ntiles) break;
    const int4 t = tiles[k];
    const BatchMember& m = mem[t.x];
    SP<R> s;
    s.load(m.P);
    StepFactors<R> f;
    f.load(m.scr->scf[parity]);
    const CUtensorMap* tm = (tmaps != nullptr && m.tma) ? tmaps + 2 * t.x + parity : nullptr;
    R cmin = is_f32<R>() ? (R)FLT_MAX : (R)DBL_MAX;
    ctu_tile<R, TX, TY, NT, MODE, true, true>(m.P, s, f, (const R*)m.U[parity], (R*)m.U[1 - parity], t.y, t.z,
                                              smem_raw, cnt, FaceHook{}, face_kind(MODE) == FACE_LEARNED ? mlp : nullptr,
                                              &cmin, tm);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const R o = __shfl_xor_sync(0xffffffffu, cmin, off);
      cmin = o < cmin ? o : cmin;
    }
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = cmin;
    __syncthreads();
    if (threadIdx.x == 0) {
      R b = wmin[0];
      for (int w = 1; w < NT / 32; ++w) b = wmin[w] < b ? wmin[w] : b;
      member_tile_done(m, (double)b, t.w, parity, advance);
    }
    __syncthreads();  // the tile's last shared-memory reads finish before the next tile's loads
  }
  if (cnt.nonconv) cnt.flags |= STATUS_NONCONV;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    cnt.solves += __shfl_xor_sync(0xffffffffu, cnt.solves, off);
    cnt.iters += __shfl_xor_sync(0xffffffffu, cnt.iters, off);
    cnt.nonconv += __shfl_xor_sync(0xffffffffu, cnt.nonconv, off);
    cnt.flags |= __shfl_xor_sync(0xffffffffu, cnt.flags, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&agg->stats[0], (unsigned long long)cnt.solves);
    atomicAdd(&agg->stats[1], (unsigned long long)cnt.iters);
    if (cnt.nonconv) atomicAdd(&agg->stats[2], (unsigned long long)cnt.nonconv);
    if (cnt.flags) atomicOr(&agg->status, cnt.flags);
  }
}

template <typename R, int TX, int TY, int NT, int MODE = FACE_PLAIN>
struct BatchStep {
  // per device (function attributes and occupancy belong to the device's context): set by prepare()
  static std::atomic<int> blocks_per_sm[64];
  static cudaError_t prepare() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (blocks_per_sm[dev].load(std::memory_order_relaxed) > 0) return cudaSuccess;
    const size_t smem = TileLayout<R, TX, TY>::bytes;
    e = cudaFuncSetAttribute(batch_step_kernel<R, TX, TY, NT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    int b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_step_kernel<R, TX, TY, NT, MODE>, NT, smem);
    if (e != cudaSuccess) return e;
    blocks_per_sm[dev].store(b > 0 ? b : 1, std::memory_order_relaxed);
    return cudaSuccess;
  }
  static cudaError_t launch(const BatchMember* mem, const int4* tiles, int ntiles, unsigned int* queue, int parity,
                            DevScratch* agg, cudaStream_t stream, int* grid_out, const CUtensorMap* tmaps,
                            int advance, const MlpBlob* mlp = nullptr) {
    cudaError_t e = prepare();
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int grid = nsm * blocks_per_sm[dev].load(std::memory_order_relaxed);
    if (grid > ntiles) grid = ntiles;
    if (grid_out) *grid_out = grid;
    if (grid <= 0) return cudaSuccess;
    e = cudaMemsetAsync(queue, 0, sizeof(unsigned int), stream);
    if (e != cudaSuccess) return e;
    batch_step_kernel<R, TX, TY, NT, MODE><<<grid, NT, TileLayout<R, TX, TY>::bytes, stream>>>(
        mem, tiles, ntiles, queue, parity, agg, tmaps, advance, mlp);
    return cudaGetLastError();
  }
};
template <typename R, int TX, int TY, int NT, int MODE>
std::atomic<int> BatchStep<R, TX, TY, NT, MODE>::blocks_per_sm[64] = {};

}  // namespace hydro
