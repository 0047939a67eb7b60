// Single-problem CTU step with piecewise-parabolic reconstruction (RECON_PPM), with either Riemann solver:
// the FP32 instantiations and the precision dispatch (FP64 in k_ctu_ppm_f64.cu).
#include "ctu_kernels.cuh"

namespace hydro {

cudaError_t ctu_step_ppm(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars& sc_host,
                         const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream, const CUtensorMap* tmap) {
  if (precision == 0) return ctu_step_ppm_f64(P, (const double*)Uin, (double*)Uout, sc_host, sc_dev, scr, stream);
  const float* in = (const float*)Uin;
  float* out = (float*)Uout;
  if (P.riemann_solver == 1)
    return launch_ctu_step<float, F32_TX, F32_TY, F32_NT, RECON_PPM | FACE_HLLC>(P, in, out, sc_host, sc_dev, scr,
                                                                                 FaceHook{}, tmap, stream);
  return launch_ctu_step<float, F32_TX, F32_TY, F32_NT, RECON_PPM | FACE_PLAIN>(P, in, out, sc_host, sc_dev, scr,
                                                                                FaceHook{}, tmap, stream);
}

cudaError_t ctu_step_fused_ppm(int precision, const KParams& P, const void* Uin, void* Uout,
                               const StepScalars* sc_cur, StepScalars* sc_next, DevScratch* scr, double tmax,
                               const CUtensorMap* tmap, cudaStream_t stream, int2 band) {
  if (precision == 0)
    return ctu_step_fused_ppm_f64(P, (const double*)Uin, (double*)Uout, sc_cur, sc_next, scr, tmax, stream, band);
  const float* in = (const float*)Uin;
  float* out = (float*)Uout;
  if (P.riemann_solver == 1)
    return launch_ctu_step_fused<float, F32_TX, F32_TY, F32_NT, RECON_PPM | FACE_HLLC>(P, in, out, sc_cur, sc_next,
                                                                                       scr, tmax, tmap, stream, band);
  return launch_ctu_step_fused<float, F32_TX, F32_TY, F32_NT, RECON_PPM | FACE_PLAIN>(P, in, out, sc_cur, sc_next,
                                                                                      scr, tmax, tmap, stream, band);
}

}  // namespace hydro
