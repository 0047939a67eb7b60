// FP64 sweeps of the dimensionally split variant.  Compiled with -fmad=false: every multiply and add rounds
// on its own, in source order, like the plain C implementation of the method.
#include "sweep_kernels.cuh"

namespace hydro {

cudaError_t split_sweep_f64(const KParams& P, const double* Uin, double* Uout, int dir, const StepScalars& sc_host,
                            const StepScalars* sc_dev, DevScratch* scr, int check_state, StepScalars* sc_next,
                            double tmax, cudaStream_t stream) {
  if (P.riemann_solver == 1) {
    if (dir == 0)
      return Sweep<double, 0, 32, 8, 128, FACE_HLLC>::launch(P, Uin, Uout, sc_host, sc_dev, scr, check_state, sc_next,
                                                             tmax, stream);
    return Sweep<double, 1, 16, 32, 256, FACE_HLLC>::launch(P, Uin, Uout, sc_host, sc_dev, scr, check_state, sc_next,
                                                            tmax, stream);
  }
  if (dir == 0)
    return Sweep<double, 0, 32, 8, 128, FACE_PLAIN>::launch(P, Uin, Uout, sc_host, sc_dev, scr, check_state, sc_next,
                                                            tmax, stream);
  return Sweep<double, 1, 16, 32, 256, FACE_PLAIN>::launch(P, Uin, Uout, sc_host, sc_dev, scr, check_state, sc_next,
                                                           tmax, stream);
}

}  // namespace hydro
