// Single-problem CTU step with the HLLC solver at every face (FACE_HLLC): the FP32 instantiations and the
// precision dispatch (FP64 in k_ctu_hllc_f64.cu).  A translation unit of its own so that it compiles in
// parallel with the two-shock kernels.
#include "ctu_kernels.cuh"

namespace hydro {

cudaError_t ctu_step_hllc(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars& sc_host,
                          const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream, const CUtensorMap* tmap) {
  if (precision == 0) return ctu_step_hllc_f64(P, (const double*)Uin, (double*)Uout, sc_host, sc_dev, scr, stream);
  return launch_ctu_step<float, F32_TX, F32_TY, F32_NT, FACE_HLLC>(P, (const float*)Uin, (float*)Uout, sc_host,
                                                                    sc_dev, scr, FaceHook{}, tmap, stream);
}

cudaError_t ctu_step_fused_hllc(int precision, const KParams& P, const void* Uin, void* Uout,
                                const StepScalars* sc_cur, StepScalars* sc_next, DevScratch* scr, double tmax,
                                const CUtensorMap* tmap, cudaStream_t stream, int2 band) {
  if (precision == 0)
    return ctu_step_fused_hllc_f64(P, (const double*)Uin, (double*)Uout, sc_cur, sc_next, scr, tmax, stream, band);
  return launch_ctu_step_fused<float, F32_TX, F32_TY, F32_NT, FACE_HLLC>(P, (const float*)Uin, (float*)Uout, sc_cur,
                                                                          sc_next, scr, tmax, tmap, stream, band);
}

}  // namespace hydro
