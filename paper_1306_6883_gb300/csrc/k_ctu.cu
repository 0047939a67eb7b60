// Single-problem CTU step: the FP32 instantiations and the precision dispatch (FP64 in k_ctu_f64.cu).
#include "ctu_kernels.cuh"

namespace hydro {

// Tile of the single-problem FP32 kernels (overridable at compile time for tile sweeps).  Measured on KH
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

int f32_tile_x() { return F32_TX; }
int f32_tile_y() { return F32_TY; }

cudaError_t ctu_step_fused(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars* sc_cur,
                           StepScalars* sc_next, DevScratch* scr, double tmax, const CUtensorMap* tmap,
                           cudaStream_t stream) {
  if (precision == 0) return ctu_step_fused_f64(P, (const double*)Uin, (double*)Uout, sc_cur, sc_next, scr, tmax, stream);
  return launch_ctu_step_fused<float, F32_TX, F32_TY, F32_NT>(P, (const float*)Uin, (float*)Uout, sc_cur, sc_next, scr,
                                                              tmax, tmap, stream);
}

cudaError_t ctu_step(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars& sc_host,
                     const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream, int mode, const FaceHook* hook,
                     const CUtensorMap* tmap) {
  if (precision == 0) return ctu_step_f64(P, (const double*)Uin, (double*)Uout, sc_host, sc_dev, scr, stream);
  const FaceHook h = hook ? *hook : FaceHook{};
  const float* in = (const float*)Uin;
  float* out = (float*)Uout;
  switch (mode) {
    case FACE_HARVEST:
      return launch_ctu_step<float, F32_TX, F32_TY, F32_NT, FACE_HARVEST>(P, in, out, sc_host, sc_dev, scr, h, tmap,
                                                                           stream);
    case FACE_LEARNED:
      // 256 threads: the network's warp-collective forward pass needs more than 56 registers
      return launch_ctu_step<float, F32_TX, F32_TY, 256, FACE_LEARNED>(P, in, out, sc_host, sc_dev, scr, h, tmap,
                                                                        stream);
    default:
      return launch_ctu_step<float, F32_TX, F32_TY, F32_NT, FACE_PLAIN>(P, in, out, sc_host, sc_dev, scr, h, tmap, stream);
  }
}

}  // namespace hydro
