// FP64 instantiations of the single-problem CTU step with piecewise-parabolic reconstruction.  Compiled with
// -fmad=false: every multiply and add rounds on its own, in source order, like the plain C implementation of
// the method.
#include "ctu_kernels.cuh"

namespace hydro {

cudaError_t ctu_step_ppm_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars& sc_host,
                             const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream) {
  if (P.riemann_solver == 1)
    return launch_ctu_step<double, 16, 16, 256, RECON_PPM | FACE_HLLC>(P, Uin, Uout, sc_host, sc_dev, scr, FaceHook{},
                                                                       nullptr, stream);
  return launch_ctu_step<double, 16, 16, 256, RECON_PPM | FACE_PLAIN>(P, Uin, Uout, sc_host, sc_dev, scr, FaceHook{},
                                                                      nullptr, stream);
}

cudaError_t ctu_step_fused_ppm_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars* sc_cur,
                                   StepScalars* sc_next, DevScratch* scr, double tmax, cudaStream_t stream,
                                   int2 band) {
  if (P.riemann_solver == 1)
    return launch_ctu_step_fused<double, 16, 16, 256, RECON_PPM | FACE_HLLC>(P, Uin, Uout, sc_cur, sc_next, scr, tmax,
                                                                             nullptr, stream, band);
  return launch_ctu_step_fused<double, 16, 16, 256, RECON_PPM | FACE_PLAIN>(P, Uin, Uout, sc_cur, sc_next, scr, tmax,
                                                                            nullptr, stream, band);
}

}  // namespace hydro
