// Batched kernels: the FP32 instantiations and the precision dispatch (FP64 in k_batch_f64.cu).
#include "batch_kernels.cuh"

namespace hydro {

// ---------------------------------------------------------------------------------------------------
// launchers

cudaError_t batch_dt(int precision, const BatchMember* mem, const int4* tab, int nblocks, int parity, int advance,
                     cudaStream_t stream) {
  if (nblocks <= 0) return cudaSuccess;
  if (precision == 0) return batch_dt_f64(mem, tab, nblocks, parity, advance, stream);
  batch_dt_kernel<float><<<nblocks, 256, 0, stream>>>(mem, tab, parity, advance);
  return cudaGetLastError();
}

// Tile shapes the autotuner chooses from (index = shape id).
const TileShape kTileShapes[] = {
    {32, 16, 384}, {16, 16, 256}, {32, 8, 256}, {32, 16, 256},
};
const int kNumTileShapes = sizeof(kTileShapes) / sizeof(kTileShapes[0]);

cudaError_t batch_step(int precision, int shape, const BatchMember* mem, const int4* tiles, int ntiles,
                       unsigned int* queue, int parity, DevScratch* agg, cudaStream_t stream, int* grid_out,
                       const CUtensorMap* tmaps, int advance, const MlpBlob* mlp) {
  if (precision == 0)  // the FP64 path keeps one shape (its cost is the FP64 pipe, not the tile)
    return mlp ? cudaErrorInvalidValue : batch_step_f64(mem, tiles, ntiles, queue, parity, agg, stream, grid_out, advance);
  if (mlp) {
    switch (shape) {
      case 0: return BatchStep<float, 32, 16, 384, FACE_LEARNED>::launch(mem, tiles, ntiles, queue, parity, agg,
                                                                         stream, grid_out, tmaps, advance, mlp);
      case 1: return BatchStep<float, 16, 16, 256, FACE_LEARNED>::launch(mem, tiles, ntiles, queue, parity, agg,
                                                                         stream, grid_out, tmaps, advance, mlp);
      case 2: return BatchStep<float, 32, 8, 256, FACE_LEARNED>::launch(mem, tiles, ntiles, queue, parity, agg,
                                                                        stream, grid_out, tmaps, advance, mlp);
      case 3: return BatchStep<float, 32, 16, 256, FACE_LEARNED>::launch(mem, tiles, ntiles, queue, parity, agg,
                                                                         stream, grid_out, tmaps, advance, mlp);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (shape) {
    case 0: return BatchStep<float, 32, 16, 384>::launch(mem, tiles, ntiles, queue, parity, agg, stream, grid_out,
                                                              tmaps, advance);
    case 1: return BatchStep<float, 16, 16, 256>::launch(mem, tiles, ntiles, queue, parity, agg, stream, grid_out,
                                                              tmaps, advance);
    case 2: return BatchStep<float, 32, 8, 256>::launch(mem, tiles, ntiles, queue, parity, agg, stream, grid_out,
                                                              tmaps, advance);
    case 3: return BatchStep<float, 32, 16, 256>::launch(mem, tiles, ntiles, queue, parity, agg, stream, grid_out,
                                                              tmaps, advance);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_prepare(int precision) {
  if (precision == 0) return batch_prepare_f64();
  cudaError_t e = BatchStep<float, 32, 16, 384>::prepare();
  if (e == cudaSuccess) e = BatchStep<float, 16, 16, 256>::prepare();
  if (e == cudaSuccess) e = BatchStep<float, 32, 8, 256>::prepare();
  if (e == cudaSuccess) e = BatchStep<float, 32, 16, 256>::prepare();
  if (e == cudaSuccess) e = BatchStep<float, 32, 16, 384, FACE_LEARNED>::prepare();
  if (e == cudaSuccess) e = BatchStep<float, 16, 16, 256, FACE_LEARNED>::prepare();
  if (e == cudaSuccess) e = BatchStep<float, 32, 8, 256, FACE_LEARNED>::prepare();
  if (e == cudaSuccess) e = BatchStep<float, 32, 16, 256, FACE_LEARNED>::prepare();
  return e;
}

}  // namespace hydro
