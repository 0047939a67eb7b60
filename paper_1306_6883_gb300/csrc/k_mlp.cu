// Training and packing of the learned star-pressure proposal (mlp.cuh), and its C ABI (hydro_mlp_*).
//
// Training data: samples harvested from CTU steps (8 floats each: rho_L, u_L, p_L, rho_R, u_R, p_R, p*,
// iterations).  Loss: mean squared error of y = ln(p*/p_ref) over a minibatch.  One training step is two
// launches: mlp_grad_kernel (each block takes 64 samples through forward and backward passes in shared
// memory and writes its partial gradient), then mlp_reduce_kernel (sums the block partials in block order
// -- deterministic -- and applies Adam, or just stores the gradient).  All arithmetic FP32.
#include <atomic>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/hydro.h"
#include "hydro_kernels.h"
#include "mlp.cuh"

namespace hydro {

constexpr int MLP_BS = 64;        // samples per block
constexpr int MLP_THREADS = 256;
constexpr int HP = 65;            // padded row stride of 64-wide shared arrays (bank-conflict free)

struct MlpSmem {
  float W[MLP_NPARAM];
  float X[MLP_BS][6];
  float T[MLP_BS];
  float M[MLP_BS];                // 1 for a real sample, 0 for padding
  float H1[MLP_BS * HP];          // h1, later dz1
  float H2[MLP_BS * HP];          // h2, later dz2
  float W2p[MLP_NH * HP];         // W2 with padded rows
  float DY[MLP_BS];
  float red[MLP_THREADS];
};

__device__ __forceinline__ unsigned int sample_index(unsigned long long seed, unsigned long long k, unsigned long long n) {
  // counter-based draw of a sample index: two rounds of the 32-bit avalanche on (seed, k)
  const unsigned int lo = hash32((unsigned int)k ^ (unsigned int)seed);
  const unsigned int hi = hash32((unsigned int)(k >> 32) ^ (unsigned int)(seed >> 32) ^ lo * 0x9E3779B1u);
  const unsigned long long r = ((unsigned long long)hi << 32) | lo;
  return (unsigned int)(r % n);
}

// Forward + backward of 64 samples per block.  samples: [n][8].  If batch_seed != 0 the block's samples
// are drawn with sample_index(batch_seed, blockIdx.x * 64 + s, n); otherwise they are rows
// blockIdx.x * 64 + s (those >= n are padding).  partial: [gridDim.x][MLP_NPARAM + 1] (gradient of the mean
// over `count` samples, then the block's sum of squared errors).
__global__ void __launch_bounds__(MLP_THREADS) mlp_grad_kernel(const float* __restrict__ theta,
                                                              const float* __restrict__ samples,
                                                              unsigned long long n, unsigned long long batch_seed,
                                                              float inv_count, float* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(raw);
  const int tid = threadIdx.x;
  for (int i = tid; i < MLP_NPARAM; i += MLP_THREADS) S.W[i] = theta[i];
  for (int i = tid; i < MLP_NH * MLP_NH; i += MLP_THREADS) S.W2p[(i / MLP_NH) * HP + i % MLP_NH] = theta[MLP_OFF_W2 + i];
  if (tid < MLP_BS) {
    unsigned long long row;
    bool real;
    if (batch_seed) {
      row = sample_index(batch_seed, (unsigned long long)blockIdx.x * MLP_BS + tid, n);
      real = true;
    } else {
      row = (unsigned long long)blockIdx.x * MLP_BS + tid;
      real = row < n;
      if (!real) row = 0;
    }
    const float* d = samples + 8 * row;
    float x[6];
    const float pref = mlp_features(d[0], d[1], d[2], d[3], d[4], d[5], x);
    for (int k = 0; k < 6; ++k) S.X[tid][k] = real ? x[k] : 0.f;
    S.T[tid] = real ? __logf(__fdividef(d[6], pref)) : 0.f;
    S.M[tid] = real ? 1.f : 0.f;
  }
  __syncthreads();
  const float* W1 = S.W + MLP_OFF_W1;
  const float* b1 = S.W + MLP_OFF_B1;
  const float* b2 = S.W + MLP_OFF_B2;
  const float* W3 = S.W + MLP_OFF_W3;
  const float b3 = S.W[MLP_OFF_B3];
  // layer 1: h1[s][j] = relu(b1[j] + sum_k W1[j][k] x[s][k])
  for (int q = tid; q < MLP_BS * MLP_NH; q += MLP_THREADS) {
    const int s = q / MLP_NH, j = q % MLP_NH;
    float z = b1[j];
#pragma unroll
    for (int k = 0; k < 6; ++k) z += W1[j * 6 + k] * S.X[s][k];
    S.H1[s * HP + j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  // layer 2: h2[s][i] = relu(b2[i] + sum_j W2[i][j] h1[s][j])
  for (int q = tid; q < MLP_BS * MLP_NH; q += MLP_THREADS) {
    const int s = q / MLP_NH, i = q % MLP_NH;
    float z = b2[i];
#pragma unroll 16
    for (int j = 0; j < MLP_NH; ++j) z += S.W2p[i * HP + j] * S.H1[s * HP + j];
    S.H2[s * HP + i] = fmaxf(z, 0.f);
  }
  __syncthreads();
  // output and its error: y[s] = b3 + W3 . h2[s]; dy = 2 (y - t) / count
  if (tid < MLP_BS) {
    float y = b3;
    for (int i = 0; i < MLP_NH; ++i) y += W3[i] * S.H2[tid * HP + i];
    const float err = (y - S.T[tid]) * S.M[tid];
    S.DY[tid] = 2.f * err * inv_count;
    S.red[tid] = err * err;
  } else {
    S.red[tid] = 0.f;
  }
  __syncthreads();
  float* out = partial + (size_t)blockIdx.x * (MLP_NPARAM + 1);
  // dW3[i] = sum_s dy[s] h2[s][i]; db3 = sum_s dy[s]
  if (tid < MLP_NH) {
    float g = 0.f;
    for (int s = 0; s < MLP_BS; ++s) g += S.DY[s] * S.H2[s * HP + tid];
    out[MLP_OFF_W3 + tid] = g;
  } else if (tid == MLP_NH) {
    float g = 0.f;
    for (int s = 0; s < MLP_BS; ++s) g += S.DY[s];
    out[MLP_OFF_B3] = g;
  }
  __syncthreads();
  // dz2[s][i] = dy[s] W3[i] 1[h2 > 0] (in place of h2)
  for (int q = tid; q < MLP_BS * MLP_NH; q += MLP_THREADS) {
    const int s = q / MLP_NH, i = q % MLP_NH;
    const float h = S.H2[s * HP + i];
    S.H2[s * HP + i] = h > 0.f ? S.DY[s] * W3[i] : 0.f;
  }
  __syncthreads();
  // dW2[i][j] = sum_s dz2[s][i] h1[s][j]; db2[i] = sum_s dz2[s][i]
  for (int q = tid; q < MLP_NH * MLP_NH; q += MLP_THREADS) {
    const int i = q / MLP_NH, j = q % MLP_NH;
    float g = 0.f;
#pragma unroll 16
    for (int s = 0; s < MLP_BS; ++s) g += S.H2[s * HP + i] * S.H1[s * HP + j];
    out[MLP_OFF_W2 + q] = g;
  }
  if (tid < MLP_NH) {
    float g = 0.f;
    for (int s = 0; s < MLP_BS; ++s) g += S.H2[s * HP + tid];
    out[MLP_OFF_B2 + tid] = g;
  }
  __syncthreads();
  // dz1[s][j] = (sum_i dz2[s][i] W2[i][j]) 1[h1 > 0]; write into a register first, then in place
  float dz1[MLP_BS * MLP_NH / MLP_THREADS];
  {
    int r = 0;
    for (int q = tid; q < MLP_BS * MLP_NH; q += MLP_THREADS, ++r) {
      const int s = q / MLP_NH, j = q % MLP_NH;
      float g = 0.f;
#pragma unroll 16
      for (int i = 0; i < MLP_NH; ++i) g += S.H2[s * HP + i] * S.W2p[i * HP + j];
      dz1[r] = S.H1[s * HP + j] > 0.f ? g : 0.f;
    }
  }
  __syncthreads();
  {
    int r = 0;
    for (int q = tid; q < MLP_BS * MLP_NH; q += MLP_THREADS, ++r) S.H1[(q / MLP_NH) * HP + q % MLP_NH] = dz1[r];
  }
  __syncthreads();
  // dW1[j][k] = sum_s dz1[s][j] x[s][k]; db1[j] = sum_s dz1[s][j]
  for (int q = tid; q < MLP_NH * 6; q += MLP_THREADS) {
    const int j = q / 6, k = q % 6;
    float g = 0.f;
    for (int s = 0; s < MLP_BS; ++s) g += S.H1[s * HP + j] * S.X[s][k];
    out[MLP_OFF_W1 + q] = g;
  }
  if (tid < MLP_NH) {
    float g = 0.f;
    for (int s = 0; s < MLP_BS; ++s) g += S.H1[s * HP + tid];
    out[MLP_OFF_B1 + tid] = g;
  }
  // block sum of squared errors (fixed tree)
  for (int w = MLP_THREADS / 2; w > 0; w >>= 1) {
    __syncthreads();
    if (tid < w) S.red[tid] += S.red[tid + w];
  }
  if (tid == 0) out[MLP_NPARAM] = S.red[0];
}

// Sum the block partials in block order; then either store the gradient (and loss) or take an Adam step.
__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int nblocks, float* __restrict__ grad_out,
                                  float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v, int adam,
                                  float lr, float b1, float b2, float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > MLP_NPARAM) return;
  float g = 0.f;
  for (int b = 0; b < nblocks; ++b) g += partial[(size_t)b * (MLP_NPARAM + 1) + p];
  if (grad_out) grad_out[p] = g;
  if (adam && p < MLP_NPARAM) {
    const float mi = b1 * m[p] + (1.f - b1) * g;
    const float vi = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mi;
    v[p] = vi;
    theta[p] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// He-normal initial weights from a counter-based generator (Box-Muller on hashed uniforms).
__global__ void mlp_init_kernel(float* theta, unsigned long long seed) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAM) return;
  float stdv = 0.f;
  if (p < MLP_OFF_B1) stdv = sqrtf(2.f / 6.f);
  else if (p >= MLP_OFF_W2 && p < MLP_OFF_B2) stdv = sqrtf(2.f / 64.f);
  else if (p >= MLP_OFF_W3 && p < MLP_OFF_B3) stdv = sqrtf(1.f / 64.f);
  const unsigned int h1 = hash32((unsigned int)p * 2u + 1u ^ (unsigned int)seed);
  const unsigned int h2 = hash32((unsigned int)p * 2u + 2u ^ (unsigned int)(seed >> 32) ^ 0x5bd1e995u);
  const float u1 = ((h1 >> 8) + 1) * (1.f / 16777217.f), u2 = (h2 >> 8) * (1.f / 16777216.f);
  theta[p] = stdv * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// BF16 fragment layout of the weights for the tensor-core inference (mlp.cuh, MlpBlob).
__global__ void mlp_pack_kernel(const float* __restrict__ theta, MlpBlob* __restrict__ blob, float gate_ratio,
                                float gate_u4) {
  const int tid = threadIdx.x;  // one block of 256 threads
  const float* W1 = theta + MLP_OFF_W1;
  const float* W2 = theta + MLP_OFF_W2;
  for (int q = tid; q < 8 * 32; q += blockDim.x) {
    const int nt = q / 32, lane = q % 32, g = lane >> 2, t = lane & 3;
    const int n = 8 * nt + g, k0 = 2 * t;
    const float lo = k0 < 6 ? W1[n * 6 + k0] : 0.f, hi = k0 + 1 < 6 ? W1[n * 6 + k0 + 1] : 0.f;
    blob->w1f[nt][lane] = pack_bf16(lo, hi);
  }
  for (int q = tid; q < 4 * 8 * 32; q += blockDim.x) {
    const int kt = q / 256, nt = (q / 32) % 8, lane = q % 32, g = lane >> 2, t = lane & 3;
    const int n = 8 * nt + g, k0 = 16 * kt + 2 * t;
    blob->w2f[kt][nt][lane][0] = pack_bf16(W2[n * 64 + k0], W2[n * 64 + k0 + 1]);
    blob->w2f[kt][nt][lane][1] = pack_bf16(W2[n * 64 + k0 + 8], W2[n * 64 + k0 + 9]);
  }
  for (int i = tid; i < 64; i += blockDim.x) {
    blob->b1[i] = theta[MLP_OFF_B1 + i];
    blob->b2[i] = theta[MLP_OFF_B2 + i];
    blob->w3[i] = theta[MLP_OFF_W3 + i];
  }
  if (tid == 0) {
    blob->b3 = theta[MLP_OFF_B3];
    blob->gate_ratio = gate_ratio;
    blob->gate_u4 = gate_u4;
    blob->pad_[0] = 0.f;
  }
}

// Network output for every sample: FP32 master weights (tc = 0) or the BF16 tensor-core path (tc = 1).
__global__ void mlp_predict_kernel(const float* __restrict__ theta, const MlpBlob* __restrict__ blob,
                                   const float* __restrict__ samples, unsigned long long n, int tc,
                                   float* __restrict__ y_out) {
  const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i < n;
  float x[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (act) {
    const float* d = samples + 8 * i;
    mlp_features(d[0], d[1], d[2], d[3], d[4], d[5], x);
  }
  if (tc) {  // every lane of the warp takes part
    const float y = mlp_warp_forward(x, blob);
    if (act) y_out[i] = y;
    return;
  }
  if (!act) return;
  float h1[64];
  for (int j = 0; j < 64; ++j) {
    float z = theta[MLP_OFF_B1 + j];
    for (int k = 0; k < 6; ++k) z += theta[MLP_OFF_W1 + j * 6 + k] * x[k];
    h1[j] = fmaxf(z, 0.f);
  }
  float y = theta[MLP_OFF_B3];
  for (int i2 = 0; i2 < 64; ++i2) {
    float z = theta[MLP_OFF_B2 + i2];
    for (int j = 0; j < 64; ++j) z += theta[MLP_OFF_W2 + i2 * 64 + j] * h1[j];
    y += theta[MLP_OFF_W3 + i2] * fmaxf(z, 0.f);
  }
  y_out[i] = y;
}

// FP32 two-shock iterations each sample needs at tolerance tol from the acoustic start (learned = 0) or
// from the network's start (learned = 1, tensor-core inference, no gate); sums[0] += iterations,
// sums[1] += unconverged solves, sums[2] += solves.  Grid-stride over warps of 32 samples (the network is
// warp-collective), counts kept per thread and added once per block, so that the time is the solves' own.
__global__ void __launch_bounds__(256) riemann_iters_kernel(const MlpBlob* __restrict__ blob,
                                                            const float* __restrict__ samples, unsigned long long n,
                                                            int learned, float gamma, float tol, int maxiter,
                                                            unsigned long long* __restrict__ sums) {
  SP<float> s{};
  s.gamma = gamma;
  s.gm1 = gamma - 1.f;
  s.igm1 = 1.f / (gamma - 1.f);
  s.g1 = (gamma + 1.f) / (2.f * gamma);
  s.small_dens = 1e-10f;
  s.small_pres = 1e-20f;
  s.tol = tol;
  s.maxiter = maxiter;
  unsigned long long it = 0, nc = 0, ns = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n;
       base += stride) {  // warp-uniform
    const unsigned long long i = base + (threadIdx.x & 31u);
    const bool act = i < n;
    float a[4] = {1.f, 0.f, 0.f, 1.f}, b[4] = {1.f, 0.f, 0.f, 1.f};
    if (act) {
      const float* d = samples + 8 * i;
      a[0] = d[0]; a[1] = d[1]; a[3] = d[2];
      b[0] = d[3]; b[1] = d[4]; b[3] = d[5];
    }
    float guess = 0.f;
    if (learned) {  // warp-collective
      float x[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      float pref = 0.f;
      if (act) pref = mlp_features(a[0], a[1], a[3], b[0], b[1], b[3], x);
      const float y = fminf(fmaxf(mlp_warp_forward(x, blob), -40.f), 40.f);
      guess = act ? pref * __expf(y) : 0.f;
    }
    if (act) {
      float F[4];
      int k;
      bool ok;
      riemann(s, a, b, guess, F, k, ok);
      it += (unsigned int)k;
      nc += ok ? 0u : 1u;
      ns += 1u;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    it += __shfl_xor_sync(0xffffffffu, it, off);
    nc += __shfl_xor_sync(0xffffffffu, nc, off);
    ns += __shfl_xor_sync(0xffffffffu, ns, off);
  }
  __shared__ unsigned long long part[8][3];
  if ((threadIdx.x & 31) == 0) {
    part[threadIdx.x >> 5][0] = it;
    part[threadIdx.x >> 5][1] = nc;
    part[threadIdx.x >> 5][2] = ns;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w][threadIdx.x];
    if (t) atomicAdd(&sums[threadIdx.x], t);
  }
}

}  // namespace hydro

// ------------------------------------------------------------------------------------------------ C ABI
using hydro::MLP_NPARAM;

struct hydro_mlp {
  cudaStream_t stream = nullptr;
  float* theta = nullptr;    // FP32 master weights
  float* m = nullptr;        // Adam moments
  float* v = nullptr;
  float* partial = nullptr;  // block partial gradients
  int partial_blocks = 0;
  float* grad = nullptr;     // last gradient + loss
  hydro::MlpBlob* blob = nullptr;
  float gate_dp = 0.35f, gate_du = 1.0f;
  long long adam_t = 0;
  char err[256] = {0};
};

static hydro_status mlp_fail(hydro_mlp* m, cudaError_t e, const char* where) {
  if (m) snprintf(m->err, sizeof m->err, "%s: %s", where, cudaGetErrorString(e));
  return HYDRO_ECUDA;
}

static cudaError_t ensure_partial(hydro_mlp* m, int blocks) {
  if (blocks <= m->partial_blocks) return cudaSuccess;
  if (m->partial) cudaFree(m->partial);
  m->partial = nullptr;
  cudaError_t e = cudaMalloc((void**)&m->partial, sizeof(float) * (size_t)blocks * (MLP_NPARAM + 1));
  m->partial_blocks = e == cudaSuccess ? blocks : 0;
  return e;
}

static cudaError_t repack(hydro_mlp* m) {
  const double du2 = (double)m->gate_du * m->gate_du;
  hydro::mlp_pack_kernel<<<1, 256, 0, m->stream>>>(m->theta, m->blob, (float)exp(2.0 * m->gate_dp), (float)(du2 * du2));
  return cudaGetLastError();
}

static cudaError_t grad_launch(hydro_mlp* m, const float* samples, unsigned long long n, unsigned long long seed,
                               int blocks, float inv_count) {
  // the attribute belongs to the device's context: set it once per device
  static std::atomic<unsigned long long> attr_done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (!bit || !(attr_done.load(std::memory_order_relaxed) & bit)) {
    e = cudaFuncSetAttribute(hydro::mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(hydro::MlpSmem));
    if (e != cudaSuccess) return e;
    if (bit) attr_done.fetch_or(bit, std::memory_order_relaxed);
  }
  hydro::mlp_grad_kernel<<<blocks, hydro::MLP_THREADS, sizeof(hydro::MlpSmem), m->stream>>>(m->theta, samples, n, seed,
                                                                                           inv_count, m->partial);
  return cudaGetLastError();
}

extern "C" {

hydro_status hydro_mlp_create(unsigned long long seed, void* cuda_stream, hydro_mlp** out) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  hydro_mlp* m = new (std::nothrow) hydro_mlp();
  if (!m) return HYDRO_ENOMEM;
  m->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMalloc((void**)&m->theta, sizeof(float) * MLP_NPARAM);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->m, sizeof(float) * MLP_NPARAM);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->v, sizeof(float) * MLP_NPARAM);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->grad, sizeof(float) * (MLP_NPARAM + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->blob, sizeof(hydro::MlpBlob));
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, sizeof(float) * MLP_NPARAM, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, sizeof(float) * MLP_NPARAM, m->stream);
  if (e == cudaSuccess) {
    hydro::mlp_init_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, m->stream>>>(m->theta, seed);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = repack(m);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    hydro_mlp_destroy(m);
    return e == cudaErrorMemoryAllocation ? HYDRO_ENOMEM : HYDRO_ECUDA;
  }
  *out = m;
  return HYDRO_OK;
}

void hydro_mlp_destroy(hydro_mlp* m) {
  if (!m) return;
  cudaFree(m->theta);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->grad);
  cudaFree(m->blob);
  if (m->partial) cudaFree(m->partial);
  delete m;
}

hydro_status hydro_mlp_set_weights(hydro_mlp* m, const float* host_theta) {
  if (!m || !host_theta) return HYDRO_EINVAL;
  cudaError_t e = cudaMemcpyAsync(m->theta, host_theta, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = repack(m);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? HYDRO_OK : mlp_fail(m, e, "set_weights");
}

hydro_status hydro_mlp_get_weights(hydro_mlp* m, float* host_theta) {
  if (!m || !host_theta) return HYDRO_EINVAL;
  cudaError_t e = cudaMemcpyAsync(host_theta, m->theta, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? HYDRO_OK : mlp_fail(m, e, "get_weights");
}

hydro_status hydro_mlp_set_gate(hydro_mlp* m, double gate_dp, double gate_du) {
  if (!m || !(gate_dp >= 0.0) || !(gate_du >= 0.0)) return HYDRO_EINVAL;
  m->gate_dp = (float)gate_dp;
  m->gate_du = (float)gate_du;
  cudaError_t e = repack(m);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? HYDRO_OK : mlp_fail(m, e, "set_gate");
}

hydro_status hydro_mlp_gradient(hydro_mlp* m, const float* d_samples, long long n, float* host_grad, double* loss) {
  if (!m || !d_samples || n < 1 || n > (1ll << 31)) return HYDRO_EINVAL;
  const int blocks = (int)((n + hydro::MLP_BS - 1) / hydro::MLP_BS);
  cudaError_t e = ensure_partial(m, blocks);
  if (e == cudaSuccess) e = grad_launch(m, d_samples, (unsigned long long)n, 0ull, blocks, 1.f / (float)n);
  if (e == cudaSuccess) {
    hydro::mlp_reduce_kernel<<<(MLP_NPARAM + 256) / 256, 256, 0, m->stream>>>(m->partial, blocks, m->grad, m->theta,
                                                                              m->m, m->v, 0, 0.f, 0.f, 0.f, 0.f,
                                                                              0.f, 0.f);
    e = cudaGetLastError();
  }
  std::vector<float> g(MLP_NPARAM + 1);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.data(), m->grad, sizeof(float) * (MLP_NPARAM + 1), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mlp_fail(m, e, "gradient");
  if (host_grad) memcpy(host_grad, g.data(), sizeof(float) * MLP_NPARAM);
  if (loss) *loss = g[MLP_NPARAM] / (double)n;
  return HYDRO_OK;
}

hydro_status hydro_mlp_train(hydro_mlp* m, const float* d_samples, long long n, int steps, int batch, double lr,
                             unsigned long long seed, double* last_loss) {
  if (!m || !d_samples || n < 1 || steps < 0 || batch < hydro::MLP_BS || batch % hydro::MLP_BS || !(lr > 0.0))
    return HYDRO_EINVAL;
  const int blocks = batch / hydro::MLP_BS;
  cudaError_t e = ensure_partial(m, blocks);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int s = 0; s < steps && e == cudaSuccess; ++s) {
    ++m->adam_t;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)m->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)m->adam_t)));
    const unsigned long long bseed = (seed * 0x9E3779B97F4A7C15ull) ^ (unsigned long long)m->adam_t | 1ull;
    e = grad_launch(m, d_samples, (unsigned long long)n, bseed, blocks, 1.f / (float)batch);
    if (e != cudaSuccess) break;
    hydro::mlp_reduce_kernel<<<(MLP_NPARAM + 256) / 256, 256, 0, m->stream>>>(
        m->partial, blocks, s + 1 == steps ? m->grad : nullptr, m->theta, m->m, m->v, 1, (float)lr, b1, b2, eps, c1, c2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = repack(m);
  float l = 0.f;
  if (e == cudaSuccess && steps > 0 && last_loss)
    e = cudaMemcpyAsync(&l, m->grad + MLP_NPARAM, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mlp_fail(m, e, "train");
  if (last_loss) *last_loss = steps > 0 ? l / (double)batch : 0.0;
  return HYDRO_OK;
}

hydro_status hydro_mlp_predict(hydro_mlp* m, const float* d_samples, long long n, int use_tensor_cores, float* d_out) {
  if (!m || !d_samples || !d_out || n < 1) return HYDRO_EINVAL;
  const unsigned long long blocks = ((unsigned long long)n + 127) / 128;
  hydro::mlp_predict_kernel<<<(unsigned int)blocks, 128, 0, m->stream>>>(m->theta, m->blob, d_samples,
                                                                          (unsigned long long)n, use_tensor_cores ? 1 : 0,
                                                                          d_out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  return e == cudaSuccess ? HYDRO_OK : mlp_fail(m, e, "predict");
}

hydro_status hydro_mlp_iterations(hydro_mlp* m, const float* d_samples, long long n, int learned, double gamma,
                                  double tol, int maxiter, double* mean_iters, long long* nonconv) {
  if (!m || !d_samples || n < 1 || !(gamma > 1.0) || !(tol > 0.0) || maxiter < 1) return HYDRO_EINVAL;
  unsigned long long* d_sums = nullptr;
  unsigned long long h[3] = {0, 0, 0};
  cudaError_t e = cudaMalloc((void**)&d_sums, sizeof h);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_sums, 0, sizeof h, m->stream);
  if (e == cudaSuccess) {
    // enough blocks to fill the GPU several times over; each takes a share of the samples
    int dev = 0, nsm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    unsigned long long blocks = ((unsigned long long)n + 255) / 256;
    const unsigned long long cap = 8ull * (unsigned long long)(nsm > 0 ? nsm : 1);
    if (blocks > cap) blocks = cap;
    if (e == cudaSuccess)
      hydro::riemann_iters_kernel<<<(unsigned int)blocks, 256, 0, m->stream>>>(
          m->blob, d_samples, (unsigned long long)n, learned ? 1 : 0, (float)gamma, (float)tol, maxiter, d_sums);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_sums, sizeof h, cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (d_sums) cudaFree(d_sums);
  if (e != cudaSuccess) return mlp_fail(m, e, "iterations");
  if (mean_iters) *mean_iters = h[2] ? (double)h[0] / (double)h[2] : 0.0;
  if (nonconv) *nonconv = (long long)h[1];
  return HYDRO_OK;
}

const void* hydro_mlp_device_blob(const hydro_mlp* m) { return m ? m->blob : nullptr; }

const char* hydro_mlp_last_error(const hydro_mlp* m) { return m ? m->err : "no model"; }

}  // extern "C"
