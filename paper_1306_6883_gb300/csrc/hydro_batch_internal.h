// Internal interface of the batched (ensemble) kernels (not installed).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "hydro_device.cuh"
#include "mlp.cuh"

namespace hydro {

// One ensemble member as the batched kernels see it (device memory).
struct BatchMember {
  KParams P;
  void* U[2];        // the member's two state buffers; parity p reads U[p] and writes U[1 - p]
  DevScratch* scr;   // the member's own dt, step factors, time and status
  int tma;           // 1: the member's tiles load by TMA from the tensor maps 2*member + parity
};

constexpr int BATCH_DT_CELLS = 2048;  // cells reduced by one block of the batched dt kernel

struct TileShape {
  int tx, ty, threads;
};
extern const TileShape kTileShapes[];
extern const int kNumTileShapes;

// tab[b] = (member, first cell, member's block count, 0); advance = 0 leaves time and step count alone; the
// member's factors are also written to scf[parity] for the fused step
cudaError_t batch_dt(int precision, const BatchMember* mem, const int4* tab, int nblocks, int parity, int advance,
                     cudaStream_t stream);
// tiles[k] = (member, tile x, tile y, the member's tile count) for tile shape `shape` (FP64 always uses
// 16 x 16).  The fused step: reads each member's factors scf[parity] (set by batch_dt or by the previous
// step), and the member's last tile writes scf[1 - parity] and, if advance, adds the step to its time.
// tmaps (FP32, may be NULL): device array of two TMA descriptors per member (one per state buffer) with the
// box of `shape`, used for members whose tma flag is set
// mlp (FP32 only, may be NULL): every member's Riemann iterations start from the learned proposal of
// these weights
cudaError_t batch_step(int precision, int shape, const BatchMember* mem, const int4* tiles, int ntiles,
                       unsigned int* queue, int parity, DevScratch* agg, cudaStream_t stream, int* grid_out,
                       const CUtensorMap* tmaps, int advance, const MlpBlob* mlp = nullptr);
// set the kernel attributes of every shape (call once before any stream capture)
cudaError_t batch_prepare(int precision);

// FP64 forms (k_batch_f64.cu, compiled without multiply-add contraction)
cudaError_t batch_dt_f64(const BatchMember* mem, const int4* tab, int nblocks, int parity, int advance,
                         cudaStream_t stream);
cudaError_t batch_step_f64(const BatchMember* mem, const int4* tiles, int ntiles, unsigned int* queue, int parity,
                           DevScratch* agg, cudaStream_t stream, int* grid_out, int advance);
cudaError_t batch_prepare_f64();

}  // namespace hydro
