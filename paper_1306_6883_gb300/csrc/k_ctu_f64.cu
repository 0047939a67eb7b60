// FP64 instantiations of the single-problem CTU step.  This file is compiled with -fmad=false: every
// multiply and add rounds on its own, in the order the source gives, so the FP64 step rounds exactly like
// the plain C implementation of the method it is tested against, and every FP64 kernel rounds alike.
#include "ctu_kernels.cuh"

namespace hydro {

cudaError_t ctu_step_fused_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars* sc_cur,
                               StepScalars* sc_next, DevScratch* scr, double tmax, cudaStream_t stream, int2 band) {
  return launch_ctu_step_fused<double, 16, 16, 256>(P, Uin, Uout, sc_cur, sc_next, scr, tmax, nullptr, stream, band);
}

cudaError_t ctu_step_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars& sc_host,
                         const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream) {
  return launch_ctu_step<double, 16, 16, 256, FACE_PLAIN>(P, Uin, Uout, sc_host, sc_dev, scr, FaceHook{}, nullptr,
                                                          stream);
}

}  // namespace hydro
