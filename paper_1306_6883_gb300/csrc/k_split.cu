// FP32 sweeps of the dimensionally split variant and the precision dispatch.
#include "sweep_kernels.cuh"

namespace hydro {

cudaError_t split_sweep(int precision, const KParams& P, const void* Uin, void* Uout, int dir,
                        const StepScalars& sc_host, const StepScalars* sc_dev, DevScratch* scr, int check_state,
                        StepScalars* sc_next, double tmax, cudaStream_t stream) {
  if (P.reconstruction == 1) return split_sweep_ppm(precision, P, Uin, Uout, dir, sc_host, sc_dev, scr, check_state,
                                                    sc_next, tmax, stream);
  if (precision == 0)
    return split_sweep_f64(P, (const double*)Uin, (double*)Uout, dir, sc_host, sc_dev, scr, check_state, sc_next, tmax, stream);
  const float* in = (const float*)Uin;
  float* out = (float*)Uout;
  // x sweeps: rows of 64 cells, 16 rows per CTA; y sweeps: 32 columns of 32 cells (consecutive columns are
  // consecutive addresses); both 61-64 KB of shared memory, 3 CTAs per SM
  if (P.riemann_solver == 1) {
    if (dir == 0)
      return Sweep<float, 0, 64, 16, SWEEP_F32_NT, FACE_HLLC>::launch(P, in, out, sc_host, sc_dev, scr, check_state, sc_next,
                                                             tmax, stream);
    return Sweep<float, 1, 32, 32, SWEEP_F32_NT, FACE_HLLC>::launch(P, in, out, sc_host, sc_dev, scr, check_state, sc_next,
                                                           tmax, stream);
  }
  if (dir == 0)
    return Sweep<float, 0, 64, 16, SWEEP_F32_NT, FACE_PLAIN>::launch(P, in, out, sc_host, sc_dev, scr, check_state, sc_next,
                                                            tmax, stream);
  return Sweep<float, 1, 32, 32, SWEEP_F32_NT, FACE_PLAIN>::launch(P, in, out, sc_host, sc_dev, scr, check_state, sc_next,
                                                          tmax, stream);
}

}  // namespace hydro
