// FP64 instantiations of the batched dt and step kernels.  Compiled with -fmad=false, like k_ctu_f64.cu, so
// a member's FP64 step rounds exactly like the same problem run alone.
#include "batch_kernels.cuh"

namespace hydro {

cudaError_t batch_dt_f64(const BatchMember* mem, const int4* tab, int nblocks, int parity, int advance,
                         cudaStream_t stream) {
  batch_dt_kernel<double><<<nblocks, 256, 0, stream>>>(mem, tab, parity, advance);
  return cudaGetLastError();
}

cudaError_t batch_step_f64(const BatchMember* mem, const int4* tiles, int ntiles, unsigned int* queue, int parity,
                           DevScratch* agg, cudaStream_t stream, int* grid_out, int advance) {
  return BatchStep<double, 16, 16, 256>::launch(mem, tiles, ntiles, queue, parity, agg, stream, grid_out, nullptr,
                                                advance);
}

cudaError_t batch_prepare_f64() { return BatchStep<double, 16, 16, 256>::prepare(); }

}  // namespace hydro
