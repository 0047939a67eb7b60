// Single-problem CTU step: the FP32 instantiations and the precision dispatch (FP64 in k_ctu_f64.cu).
#include "ctu_kernels.cuh"

namespace hydro {

int f32_tile_x() { return F32_TX; }
int f32_tile_y() { return F32_TY; }

cudaError_t ctu_step_fused(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars* sc_cur,
                           StepScalars* sc_next, DevScratch* scr, double tmax, const CUtensorMap* tmap,
                           cudaStream_t stream, int2 band, const MlpBlob* mlp) {
  if (mlp != nullptr) {
    // 320 threads (64 registers at 3 CTAs per SM): at 384 threads (56 registers) the gate test in the face
    // loops, together with the pass over the queued faces, makes the allocator spill inside the loops
    if (precision == 0 || P.reconstruction == 1 || P.riemann_solver == 1) return cudaErrorInvalidValue;
    return launch_ctu_step_fused<float, F32_TX, F32_TY, 320, FACE_LEARNED>(
        P, (const float*)Uin, (float*)Uout, sc_cur, sc_next, scr, tmax, tmap, stream, band, mlp);
  }
  if (P.reconstruction == 1)
    return ctu_step_fused_ppm(precision, P, Uin, Uout, sc_cur, sc_next, scr, tmax, tmap, stream, band);
  if (P.riemann_solver == 1)
    return ctu_step_fused_hllc(precision, P, Uin, Uout, sc_cur, sc_next, scr, tmax, tmap, stream, band);
  if (precision == 0)
    return ctu_step_fused_f64(P, (const double*)Uin, (double*)Uout, sc_cur, sc_next, scr, tmax, stream, band);
  return launch_ctu_step_fused<float, F32_TX, F32_TY, F32_NT>(P, (const float*)Uin, (float*)Uout, sc_cur, sc_next, scr,
                                                              tmax, tmap, stream, band);
}

int fused_tile_height(int precision) { return precision == 0 ? 16 : F32_TY; }  // FP64 tiles are 16 x 16

int fused_tile_rows(int precision, const KParams& P) {
  const int th = fused_tile_height(precision);
  return (P.ny + th - 1) / th;
}

cudaError_t ctu_step(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars& sc_host,
                     const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream, int mode, const FaceHook* hook,
                     const CUtensorMap* tmap) {
  if (P.reconstruction == 1) return ctu_step_ppm(precision, P, Uin, Uout, sc_host, sc_dev, scr, stream, tmap);
  if (P.riemann_solver == 1) return ctu_step_hllc(precision, P, Uin, Uout, sc_host, sc_dev, scr, stream, tmap);
  if (precision == 0) return ctu_step_f64(P, (const double*)Uin, (double*)Uout, sc_host, sc_dev, scr, stream);
  const FaceHook h = hook ? *hook : FaceHook{};
  const float* in = (const float*)Uin;
  float* out = (float*)Uout;
  switch (mode) {
    case FACE_HARVEST:
      return launch_ctu_step<float, F32_TX, F32_TY, F32_NT, FACE_HARVEST>(P, in, out, sc_host, sc_dev, scr, h, tmap,
                                                                           stream);
    case FACE_LEARNED:
      return launch_ctu_step<float, F32_TX, F32_TY, F32_NT, FACE_LEARNED>(P, in, out, sc_host, sc_dev, scr, h, tmap,
                                                                           stream);
    default:
      return launch_ctu_step<float, F32_TX, F32_TY, F32_NT, FACE_PLAIN>(P, in, out, sc_host, sc_dev, scr, h, tmap, stream);
  }
}

}  // namespace hydro
