// Learned star-pressure proposal for the two-shock Riemann iteration (not in the paper: it only chooses
// where the §3.2 Newton iteration starts; the iteration still runs to the same tolerance and decides the
// answer).  MLP 6 -> 64 -> 64 -> 1, ReLU hidden layers, on reference-unit inputs that use the scaling
// symmetry of the Euler equations:
//   rho_ref = sqrt(rho_L rho_R), p_ref = sqrt(p_L p_R), c_ref = sqrt(p_ref/rho_ref), u_mean = (u_L+u_R)/2
//   x = (ln(rho_L/rho_ref), (u_L-u_mean)/c_ref, ln(p_L/p_ref), ln(rho_R/rho_ref), (u_R-u_mean)/c_ref, ln(p_R/p_ref))
//   y = ln(p*/p_ref), proposal p0 = p_ref exp(y).
// Master weights are FP32 (layout W1[64][6], b1[64], W2[64][64], b2[64], W3[64], b3); inference uses BF16
// weights and activations with FP32 accumulation on the tensor cores (mma.sync m16n8k16), 32 faces per
// warp, in a pass of each CTU tile over its gated faces.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace hydro {

constexpr int MLP_NIN = 6, MLP_NH = 64;
constexpr int MLP_OFF_W1 = 0, MLP_OFF_B1 = 384, MLP_OFF_W2 = 448, MLP_OFF_B2 = 4544, MLP_OFF_W3 = 4608,
              MLP_OFF_B3 = 4672, MLP_NPARAM = 4673;

// Inference weights in the register layout of the mma fragments (built by the packing kernel).
struct MlpBlob {
  uint32_t w1f[8][32];        // layer 1 B fragment per (n tile, lane): bf16 pair (W1[n][2t], W1[n][2t+1])
  uint32_t w2f[4][8][32][2];  // layer 2 B fragments per (k tile, n tile, lane)
  float b1[64], b2[64], w3[64];
  float b3;
  // gate: a face starts from the network's proposal if max(pL,pR) >= gate_ratio min(pL,pR) or
  // (uL-uR)^4 rho_L rho_R >= gate_u4 p_L p_R, i.e. |ln(pL/pR)|/2 >= gate_dp or |uL-uR|/c_ref >= gate_du with
  // gate_ratio = exp(2 gate_dp), gate_u4 = gate_du^4; otherwise from the acoustic guess
  float gate_ratio, gate_u4;
  float pad_[1];
};

// Device-side options of one CTU step beyond the method itself.
struct FaceHook {
  // harvest of Riemann inputs and converged star pressures (8 floats per sample:
  // rho_L, u_L, p_L, rho_R, u_R, p_R, p*, iterations)
  float* hbuf;
  unsigned long long* hcount;
  unsigned long long hcap;
  unsigned int hthresh;  // a face is sampled when its hash is below this
  unsigned int hseed;
  // faces past this gate (as MlpBlob::gate_ratio / gate_u4) are recorded whatever their hash; 0 = off
  float hgate_ratio, hgate_u4;
  const MlpBlob* mlp;    // learned proposal weights (device), or null
};

// Tile modes: the face-solve variant in the low two bits, and RECON_PPM for piecewise-parabolic
// reconstruction instead of piecewise-linear.
enum { FACE_PLAIN = 0, FACE_HARVEST = 1, FACE_LEARNED = 2, FACE_HLLC = 3, RECON_PPM = 4 };
constexpr int face_kind(int mode) { return mode & 3; }

__device__ __forceinline__ unsigned int hash32(unsigned int x) {
  // integer avalanche (xorshift-multiply)
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Reference-unit inputs of one face; returns p_ref.
__device__ __forceinline__ float mlp_features(float rl, float ul, float pl, float rr, float ur, float pr, float x[6]) {
  const float lr = 0.5f * __logf(__fdividef(rl, rr));  // ln(rho_L / rho_ref)
  const float lp = 0.5f * __logf(__fdividef(pl, pr));  // ln(p_L / p_ref)
  const float pp = pl * pr, pref = pp * rsqrtf(pp);    // sqrt(p_L p_R)
  const float icref = rsqrtf(pref * rsqrtf(rl * rr));  // 1 / sqrt(p_ref / rho_ref)
  const float du = 0.5f * (ul - ur) * icref;
  x[0] = lr;
  x[1] = du;
  x[2] = lp;
  x[3] = -lr;
  x[4] = -du;
  x[5] = -lp;
  return pref;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Network output y for the face of every lane of the warp (all 32 lanes must call it).  Not inlined: the
// CTU tiles call it only in their pass over the gated faces, after the face loops, and keeping its unrolled
// tensor-core code and registers apart leaves the loops' register allocation as in the plain kernel.
// rows (warp-uniform): the lanes whose outputs are used are 0 .. rows-1; with rows <= 16 only the first 16-row
// tile is evaluated (lanes 16-31 then return 0).  A tile's pass over one to sixteen gated faces, the common
// case, then waits on half the network's latency.
static __device__ __noinline__ float mlp_warp_forward(const float x[6], const MlpBlob* __restrict__ w, int rows = 32) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float yv[2][2] = {{0.f, 0.f}, {0.f, 0.f}};  // [m tile][row half] partial outputs of rows 16 mt + g + 8 half
  const int nmt = rows > 16 ? 2 : 1;
  // one m tile at a time keeps the live fragments to ~40 registers (weights are re-read from shared memory)
#pragma unroll 1
  for (int mt = 0; mt < nmt; ++mt) {
    // A fragment of layer 1: rows 16 mt + g and + 8, columns 2t, 2t+1 (columns >= 6 are zero padding)
    float xa[6], xb[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      xa[k] = __shfl_sync(0xffffffffu, x[k], 16 * mt + g);
      xb[k] = __shfl_sync(0xffffffffu, x[k], 16 * mt + g + 8);
    }
    const float a0 = t == 0 ? xa[0] : t == 1 ? xa[2] : t == 2 ? xa[4] : 0.f;
    const float a1 = t == 0 ? xa[1] : t == 1 ? xa[3] : t == 2 ? xa[5] : 0.f;
    const float b0 = t == 0 ? xb[0] : t == 1 ? xb[2] : t == 2 ? xb[4] : 0.f;
    const float b1 = t == 0 ? xb[1] : t == 1 ? xb[3] : t == 2 ? xb[5] : 0.f;
    const uint32_t A1[4] = {pack_bf16(a0, a1), pack_bf16(b0, b1), 0u, 0u};
    // layer 1 -> ReLU -> bf16 A fragments of layer 2 (n tiles 2kt, 2kt+1 form k tile kt)
    uint32_t A2[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int nt = 2 * kt + h;
        const float bl = w->b1[8 * nt + 2 * t], bh = w->b1[8 * nt + 2 * t + 1];
        float c[4] = {bl, bh, bl, bh};
        mma_bf16(c, A1, w->w1f[nt][lane], 0u);
        A2[kt][2 * h] = pack_bf16(fmaxf(c[0], 0.f), fmaxf(c[1], 0.f));
        A2[kt][2 * h + 1] = pack_bf16(fmaxf(c[2], 0.f), fmaxf(c[3], 0.f));
      }
    }
    // layer 2 -> ReLU -> dot with W3 (FP32 on the FMA pipe)
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float bl = w->b2[8 * nt + 2 * t], bh = w->b2[8 * nt + 2 * t + 1];
      float c[4] = {bl, bh, bl, bh};
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        const uint32_t a[4] = {A2[kt][0], A2[kt][1], A2[kt][2], A2[kt][3]};
        const uint2 bb = *reinterpret_cast<const uint2*>(&w->w2f[kt][nt][lane][0]);
        mma_bf16(c, a, bb.x, bb.y);
      }
      const float wl = w->w3[8 * nt + 2 * t], wh = w->w3[8 * nt + 2 * t + 1];
      s0 += fmaxf(c[0], 0.f) * wl + fmaxf(c[1], 0.f) * wh;
      s1 += fmaxf(c[2], 0.f) * wl + fmaxf(c[3], 0.f) * wh;
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    yv[mt][0] = s0 + w->b3;
    yv[mt][1] = s1 + w->b3;
  }
  // lane L owns row L = 16 mt + 8 half + r: its value sits in lanes 4 r .. 4 r + 3
  const int src = 4 * (lane & 7);
  const float v00 = __shfl_sync(0xffffffffu, yv[0][0], src), v01 = __shfl_sync(0xffffffffu, yv[0][1], src);
  const float v10 = __shfl_sync(0xffffffffu, yv[1][0], src), v11 = __shfl_sync(0xffffffffu, yv[1][1], src);
  const int mt = lane >> 4, half = (lane >> 3) & 1;
  return mt == 0 ? (half == 0 ? v00 : v01) : (half == 0 ? v10 : v11);
}

// The strong-face test of the gate: max(pL,pR) >= ratio min(pL,pR) or (uL-uR)^4 rho_L rho_R >= u4 p_L p_R
// (no transcendental functions).
__device__ __forceinline__ bool strong_face(const float a[4], const float b[4], float ratio, float u4) {
  const float du = a[1] - b[1], du2 = du * du;
  return fmaxf(a[3], b[3]) >= ratio * fminf(a[3], b[3]) || du2 * du2 * (a[0] * b[0]) >= u4 * (a[3] * b[3]);
}

}  // namespace hydro
