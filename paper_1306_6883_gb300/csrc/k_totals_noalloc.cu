// Conserved totals without any allocation: hydro_conserved_totals_noalloc (declared in include/hydro.h).
//
// Some callers cannot allocate device memory at the point where they need the totals: code that runs
// while another allocator owns the device memory (a framework's caching allocator or a fixed pool,
// where a stray cudaMalloc would fragment or overrun the budget), and diagnostics taken after an
// out-of-memory error, when cudaMalloc itself fails.  This entry point needs no context and allocates
// nothing: its reduction scratch is the file-scope device array below, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/hydro.h"
#include "hydro_device.cuh"

namespace {

constexpr int kMaxRows = HYDRO_NOALLOC_MAX_ROWS;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 2 * 152;
// layout: per-row partial sums [kMaxRows][4], then the 4 totals, then one slot holding the block counter
constexpr int kScratchDoubles = 4 * kMaxRows + 4 + 4;

static __device__ __align__(256) double g_totals_scratch[kScratchDoubles];

// One partial per grid row (fixed-shape tree over the row), then the last block to finish adds the row
// partials: thread t sums rows t, t + 256, t + 512, ... in order, and a fixed-shape tree over the 256
// threads combines those sums.  The same per-cell double accumulation as the allocating totals kernel,
// with results that depend only on the grid (not on which block finishes last).
template <typename R>
__global__ void __launch_bounds__(kThreads) totals_rows_kernel(hydro::KParams P, const R* __restrict__ U,
                                                              double* __restrict__ scratch) {
  double* partials = scratch;
  double* totals = scratch + 4 * kMaxRows;
  unsigned int* done = reinterpret_cast<unsigned int*>(scratch + 4 * kMaxRows + 4);
  const size_t plane = (size_t)P.NY * P.pitch;
  __shared__ double red[4][kThreads];
  __shared__ bool last;
  for (int j = blockIdx.x; j < P.ny; j += gridDim.x) {
    const size_t row = (size_t)(j + P.ng) * P.pitch + P.ng;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < P.nx; i += kThreads) {
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += (double)U[row + i + k * plane];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
#pragma unroll
        for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) partials[4 * j + k] = red[k][0];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < P.ny; j += kThreads) {
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += ((volatile double*)partials)[4 * j + k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double area = P.dx * P.dy;
#pragma unroll
    for (int k = 0; k < 4; ++k) totals[k] = red[k][0] * area;
    *done = 0u;
  }
}

// Device address of g_totals_scratch per device ordinal, looked up once with that device current and kept
// for the life of the process.  A cudaDeviceReset of that device ends the context the address belongs to,
// so the entry point does not support being called after one.
std::mutex g_mu;
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};

hydro_status scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return HYDRO_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_totals_scratch) != cudaSuccess || !ptr) return HYDRO_ECUDA;
    g_scratch_addr[device] = static_cast<double*>(ptr);
  }
  *out = g_scratch_addr[device];
  return HYDRO_OK;
}

}  // namespace

extern "C" hydro_status hydro_conserved_totals_noalloc(const hydro_params* p, const void* d_state, void* cuda_stream,
                                                       double out[4]) {
  if (!p || !d_state || !out) return HYDRO_EINVAL;
  const size_t pitch = hydro_state_pitch(p);  // 0 when the parameters are invalid
  if (pitch == 0) return HYDRO_EINVAL;
  if (p->ny > kMaxRows) return HYDRO_ERANGE;
  hydro::KParams k{};
  k.nx = p->nx;
  k.ny = p->ny;
  k.ng = p->ng;
  k.pitch = (int)pitch;
  k.NX = p->nx + 2 * p->ng;
  k.NY = p->ny + 2 * p->ng;
  k.dx = (p->xmax - p->xmin) / p->nx;
  k.dy = (p->ymax - p->ymin) / p->ny;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return HYDRO_ECUDA;
  double* scratch = nullptr;
  hydro_status st = scratch_address(device, &scratch);
  if (st != HYDRO_OK) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // the block counter must start at zero; the partials of rows [0, ny) are all rewritten before use
  cudaError_t e = cudaMemsetAsync(scratch + 4 * kMaxRows + 4, 0, sizeof(double), stream);
  const int blocks = p->ny < kMaxBlocks ? p->ny : kMaxBlocks;
  if (e == cudaSuccess) {
    if (p->precision == HYDRO_FP32)
      totals_rows_kernel<float><<<blocks, kThreads, 0, stream>>>(k, (const float*)d_state, scratch);
    else
      totals_rows_kernel<double><<<blocks, kThreads, 0, stream>>>(k, (const double*)d_state, scratch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, scratch + 4 * kMaxRows, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}
