// Ghost-cell fill, CFL time-step reduction and conserved-total reduction kernels.
#include <float.h>

#include "hydro_device.cuh"
#include "hydro_kernels.h"

namespace hydro {

// ---------------------------------------------------------------------------------------------------
// Ghost cells (paper §2, CellCenterData2d ghost filling; Fig. 1): ghost (i, j) takes interior cell
// (map_x(i), map_y(j)) through fill_ghost_cell (outflow, periodic, reflecting and hydrostatic sides).
// All sources are interior cells, so one pass over the ghost frame fills edges and corners.
template <typename R>
__global__ void fill_ghost_kernel(KParams P, R* __restrict__ U) {
  // ghost frame enumerated as: bottom band ng x NX, top band ng x NX, then left/right bands ny x ng each
  const int band = P.ng * P.NX;
  const int side = P.ny * P.ng;
  const int n = 2 * band + 2 * side;
  const size_t plane = (size_t)P.NY * P.pitch;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int i, j;
    if (e < band) {
      j = e / P.NX; i = e % P.NX;
    } else if (e < 2 * band) {
      const int f = e - band;
      j = P.ng + P.ny + f / P.NX; i = f % P.NX;
    } else if (e < 2 * band + side) {
      const int f = e - 2 * band;
      j = P.ng + f / P.ng; i = f % P.ng;
    } else {
      const int f = e - 2 * band - side;
      j = P.ng + f / P.ng; i = P.ng + P.nx + f % P.ng;
    }
    fill_ghost_cell(P, U, i, j, plane);
  }
}

cudaError_t fill_ghost(int precision, const KParams& P, void* U, cudaStream_t stream) {
  const int n = 2 * P.ng * P.NX + 2 * P.ny * P.ng;
  const int threads = 256;
  int blocks = (n + threads - 1) / threads;
  if (blocks > 1024) blocks = 1024;
  if (precision == 0)
    fill_ghost_kernel<double><<<blocks, threads, 0, stream>>>(P, (double*)U);
  else
    fill_ghost_kernel<float><<<blocks, threads, 0, stream>>>(P, (float*)U);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------
// CFL time step (Eq. 6 with signal speeds |u|+c, |v|+c): per-cell min(dx/(|u|+c), dy/(|v|+c)) in the
// state's precision, promoted to double; warp-shuffle min, block min, one atomicMin per block on the
// bit pattern (positive doubles order like their bits); the last block to finish scales by cfl, clamps
// to tmax - t and resets the accumulator for the next call.
// Grid cap of the dt reduction (overridable at compile time for sweeps).  Measured on KH 1024^2 FP32, 200
// back-to-back launches: 152 blocks 13.6 us, 304 and 608 blocks 10.3 us, 1216 blocks 12.3 us (more blocks
// than that spend their time in the per-block atomics on the two shared words).
#ifndef HYDRO_DT_MAX_BLOCKS
#define HYDRO_DT_MAX_BLOCKS (4 * 152)
#endif
constexpr int DT_THREADS = 256;
constexpr int DT_MAX_BLOCKS = HYDRO_DT_MAX_BLOCKS;

template <typename R>
__global__ void __launch_bounds__(DT_THREADS) cfl_dt_kernel(KParams P, const R* __restrict__ U,
                                                           DevScratch* __restrict__ scr, double tmax, int advance,
                                                           StepScalars* __restrict__ sc_out) {
  SP<R> s;
  s.load(P);
  const size_t plane = (size_t)P.NY * P.pitch;
  R rbest = is_f32<R>() ? (R)FLT_MAX : (R)DBL_MAX;
  unsigned int flags = 0;
  // a block takes whole interior rows; a thread takes every DT_THREADS-th cell of a row, four at a time with
  // all their loads issued before any arithmetic
  for (int j = blockIdx.x; j < P.ny; j += gridDim.x) {
    const R* row = U + (size_t)(j + P.ng) * P.pitch + P.ng;
    for (int i0 = threadIdx.x; i0 < P.nx; i0 += 4 * DT_THREADS) {
      R v[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * DT_THREADS;
        if (i < P.nx) {
#pragma unroll
          for (int k = 0; k < 4; ++k) v[u][k] = __ldg(row + i + k * plane);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u * DT_THREADS < P.nx) cfl_value(s, v[u][0], v[u][1], v[u][2], v[u][3], rbest, flags);
    }
  }
  // the minimum of the per-cell values is exact in their own precision; promote once
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const R o = __shfl_xor_sync(0xffffffffu, rbest, off);
    rbest = o < rbest ? o : rbest;
    flags |= __shfl_xor_sync(0xffffffffu, flags, off);
  }
  const double best = (double)rbest;
  __shared__ double wmin[DT_THREADS / 32];
  __shared__ unsigned int wflags[DT_THREADS / 32];
  __shared__ bool last;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    wmin[w] = best;
    wflags[w] = flags;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = wmin[0];
    unsigned int f = wflags[0];
    for (int k = 1; k < DT_THREADS / 32; ++k) {
      b = wmin[k] < b ? wmin[k] : b;
      f |= wflags[k];
    }
    atomicMin(&scr->dt_min_bits, (unsigned long long)__double_as_longlong(b));
    if (f) atomicOr(&scr->status, f);
    __threadfence();
    const unsigned int done = atomicAdd(&scr->dt_blocks_done, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const unsigned long long bits = atomicExch(&scr->dt_min_bits, (unsigned long long)__double_as_longlong(DBL_MAX));
    double dt = P.cfl * __longlong_as_double((long long)bits);
    if (tmax > 0.0) {
      const double left = tmax - scr->t;
      dt = dt > left ? left : dt;
      dt = dt < 0.0 ? 0.0 : dt;
    }
    scr->dt = dt;
    scr->sc = make_step_scalars(dt, P.dx, P.dy, P.grav);
    if (sc_out) *sc_out = scr->sc;
    if (advance) {
      scr->t = scr->t + dt;
      scr->nsteps = scr->nsteps + 1;
    }
    scr->dt_blocks_done = 0u;
  }
}

cudaError_t cfl_dt(int precision, const KParams& P, const void* U, DevScratch* scr, double tmax, int advance_time,
                   StepScalars* sc_out, cudaStream_t stream) {
  const int blocks = P.ny < DT_MAX_BLOCKS ? P.ny : DT_MAX_BLOCKS;
  if (precision == 0)
    cfl_dt_kernel<double><<<blocks, DT_THREADS, 0, stream>>>(P, (const double*)U, scr, tmax, advance_time, sc_out);
  else
    cfl_dt_kernel<float><<<blocks, DT_THREADS, 0, stream>>>(P, (const float*)U, scr, tmax, advance_time, sc_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------
// Conserved totals: sum_ij U_k dx dy in double.  Each block owns a fixed set of rows (grid-stride over
// rows), each thread a fixed set of columns; block partials are combined by a fixed-shape tree, and the
// last block adds the per-block partials in block order.  Deterministic for a given grid size.
constexpr int TOT_THREADS = 256;
constexpr int TOT_MAX_BLOCKS = 2 * 152;

int totals_max_blocks() { return TOT_MAX_BLOCKS; }

template <typename R>
__global__ void __launch_bounds__(TOT_THREADS) totals_kernel(KParams P, const R* __restrict__ U,
                                                            double* __restrict__ partials, DevScratch* __restrict__ scr) {
  const size_t plane = (size_t)P.NY * P.pitch;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = blockIdx.x; j < P.ny; j += gridDim.x) {
    const size_t row = (size_t)(j + P.ng) * P.pitch + P.ng;
    for (int i = threadIdx.x; i < P.nx; i += TOT_THREADS) {
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += (double)U[row + i + k * plane];
    }
  }
  __shared__ double red[4][TOT_THREADS];
  __shared__ bool last;
#pragma unroll
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = TOT_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) partials[blockIdx.x * 4 + k] = red[k][0];
    __threadfence();
    const unsigned int done = atomicAdd(&scr->tot_blocks_done, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const double area = P.dx * P.dy;
    for (int k = 0; k < 4; ++k) {
      double sum = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) sum += ((volatile double*)partials)[b * 4 + k];
      scr->totals[k] = sum * area;
    }
    scr->tot_blocks_done = 0u;
  }
}

cudaError_t conserved_totals(int precision, const KParams& P, const void* U, double* partials, DevScratch* scr,
                             cudaStream_t stream) {
  const int blocks = P.ny < TOT_MAX_BLOCKS ? P.ny : TOT_MAX_BLOCKS;
  if (precision == 0)
    totals_kernel<double><<<blocks, TOT_THREADS, 0, stream>>>(P, (const double*)U, partials, scr);
  else
    totals_kernel<float><<<blocks, TOT_THREADS, 0, stream>>>(P, (const float*)U, partials, scr);
  return cudaGetLastError();
}

__global__ void init_scratch_kernel(DevScratch* scr) {
  scr->dt_min_bits = (unsigned long long)__double_as_longlong(DBL_MAX);
  scr->dt_blocks_done = 0u;
  scr->tot_blocks_done = 0u;
  scr->dt = 0.0;
  scr->t = 0.0;
  scr->nsteps = 0;
  scr->status = 0u;
  scr->stats[0] = scr->stats[1] = scr->stats[2] = 0ull;
  for (int k = 0; k < 4; ++k) scr->totals[k] = 0.0;
  scr->dtn_min_bits = (unsigned long long)__double_as_longlong(DBL_MAX);
  scr->step_blocks_done = 0u;
}

cudaError_t init_scratch(DevScratch* scr, cudaStream_t stream) {
  init_scratch_kernel<<<1, 1, 0, stream>>>(scr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------
// Upload of a dense host array [rows][width bytes] that the device can address (pinned, mapped) into the
// pitched state: the SMs read the host memory directly over the chip-to-chip link, which on this system
// moves a pitched copy faster than the copy engine does.  W: 16-byte vectors when every row start is
// 16-byte aligned on both sides, else 4-byte words (row widths are whole elements of 4 or 8 bytes).
template <typename W>
__global__ void __launch_bounds__(256) upload_rows_kernel(const W* __restrict__ src, W* __restrict__ dst,
                                                         size_t src_pitch, size_t dst_pitch, int width, int rows) {
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const W* s = src + (size_t)r * src_pitch;
    W* d = dst + (size_t)r * dst_pitch;
    for (int i = threadIdx.x; i < width; i += blockDim.x) d[i] = s[i];
  }
}

cudaError_t upload_rows(const void* host_dev, void* dst, size_t row_bytes, size_t dst_pitch_bytes, int rows,
                        cudaStream_t stream) {
  if (rows <= 0 || row_bytes == 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = rows < 8 * nsm ? rows : 8 * nsm;
  if (((uintptr_t)host_dev | (uintptr_t)dst | row_bytes | dst_pitch_bytes) % 16 == 0)
    upload_rows_kernel<uint4><<<grid, 256, 0, stream>>>((const uint4*)host_dev, (uint4*)dst, row_bytes / 16,
                                                        dst_pitch_bytes / 16, (int)(row_bytes / 16), rows);
  else
    upload_rows_kernel<unsigned int><<<grid, 256, 0, stream>>>((const unsigned int*)host_dev, (unsigned int*)dst,
                                                               row_bytes / 4, dst_pitch_bytes / 4,
                                                               (int)(row_bytes / 4), rows);
  return cudaGetLastError();
}

}  // namespace hydro
