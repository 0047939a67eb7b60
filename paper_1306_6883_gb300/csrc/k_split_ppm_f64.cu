// FP64 sweeps of the dimensionally split variant with piecewise-parabolic reconstruction.  Compiled with
// -fmad=false: every multiply and add rounds on its own, in source order, like the plain C implementation of
// the method.
#include "sweep_kernels.cuh"

namespace hydro {

template <int MODE>
static cudaError_t sweep_ppm_f64(const KParams& P, const double* in, double* out, int dir, const StepScalars& sc_host,
                                 const StepScalars* sc_dev, DevScratch* scr, int check_state, StepScalars* sc_next,
                                 double tmax, cudaStream_t stream) {
  if (dir == 0)
    return Sweep<double, 0, 32, 8, 128, MODE>::launch(P, in, out, sc_host, sc_dev, scr, check_state, sc_next, tmax,
                                                      stream);
  return Sweep<double, 1, 16, 32, 256, MODE>::launch(P, in, out, sc_host, sc_dev, scr, check_state, sc_next, tmax,
                                                     stream);
}

cudaError_t split_sweep_ppm_f64(const KParams& P, const double* Uin, double* Uout, int dir,
                                const StepScalars& sc_host, const StepScalars* sc_dev, DevScratch* scr,
                                int check_state, StepScalars* sc_next, double tmax, cudaStream_t stream) {
  if (P.riemann_solver == 1)
    return sweep_ppm_f64<RECON_PPM | FACE_HLLC>(P, Uin, Uout, dir, sc_host, sc_dev, scr, check_state, sc_next, tmax,
                                                stream);
  return sweep_ppm_f64<RECON_PPM | FACE_PLAIN>(P, Uin, Uout, dir, sc_host, sc_dev, scr, check_state, sc_next, tmax,
                                               stream);
}

}  // namespace hydro
