// FP32 sweeps of the dimensionally split variant with piecewise-parabolic reconstruction, and the precision
// dispatch (FP64 in k_split_ppm_f64.cu).
#include "sweep_kernels.cuh"

namespace hydro {

template <int MODE>
static cudaError_t sweep_ppm_f32(const KParams& P, const float* in, float* out, int dir, const StepScalars& sc_host,
                                 const StepScalars* sc_dev, DevScratch* scr, int check_state, StepScalars* sc_next,
                                 double tmax, cudaStream_t stream) {
  if (dir == 0)
    return Sweep<float, 0, 64, 16, SWEEP_F32_NT, MODE>::launch(P, in, out, sc_host, sc_dev, scr, check_state, sc_next, tmax,
                                                      stream);
  return Sweep<float, 1, 32, 32, SWEEP_F32_NT, MODE>::launch(P, in, out, sc_host, sc_dev, scr, check_state, sc_next, tmax,
                                                    stream);
}

cudaError_t split_sweep_ppm(int precision, const KParams& P, const void* Uin, void* Uout, int dir,
                            const StepScalars& sc_host, const StepScalars* sc_dev, DevScratch* scr, int check_state,
                            StepScalars* sc_next, double tmax, cudaStream_t stream) {
  if (precision == 0)
    return split_sweep_ppm_f64(P, (const double*)Uin, (double*)Uout, dir, sc_host, sc_dev, scr, check_state, sc_next,
                               tmax, stream);
  const float* in = (const float*)Uin;
  float* out = (float*)Uout;
  if (P.riemann_solver == 1)
    return sweep_ppm_f32<RECON_PPM | FACE_HLLC>(P, in, out, dir, sc_host, sc_dev, scr, check_state, sc_next, tmax,
                                                stream);
  return sweep_ppm_f32<RECON_PPM | FACE_PLAIN>(P, in, out, dir, sc_host, sc_dev, scr, check_state, sc_next, tmax,
                                               stream);
}

}  // namespace hydro
