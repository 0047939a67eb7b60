// Internal launch interface between the C-ABI layer and the CUDA kernels (not installed).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/hydro.h"
#include "hydro_device.cuh"
#include "mlp.cuh"

namespace hydro {

// precision: 0 = double, 1 = float.  All launches are asynchronous on `stream`.
cudaError_t fill_ghost(int precision, const KParams& P, void* U, cudaStream_t stream);

// CFL reduction.  Writes scr->dt = cfl * min(...), clamped to tmax - scr->t when tmax > 0 and, if
// advance_time, adds it to scr->t and increments scr->nsteps.  Sets status bits for non-finite or
// non-positive cells.  The min accumulator and block counter are reset by the last block.
// sc_out (optional): also receives the step factors.
cudaError_t cfl_dt(int precision, const KParams& P, const void* U, DevScratch* scr, double tmax, int advance_time,
                   StepScalars* sc_out, cudaStream_t stream);

// One fused CTU step (ghost cells from the boundary map, CFL of the new state folded in): reads the step
// factors at sc_cur; the last block adds sc_cur->dt to the time, counts the step and writes the next step's
// factors (dt = cfl * min, clamped to tmax - t when tmax > 0) to sc_next.
// tmap (FP32 only, may be NULL): TMA descriptor of Uin as a 3-D tensor (x over the padded width, y over the
// padded height, the 4 conserved components) with a (TX+8) x (TY+8) x 4 box; tiles whose box is valid are
// then loaded by one bulk tensor copy.
// band (optional): tile rows [band.x, band.x + band.y) only (band.y <= 0: the whole step); bands of one
// step may run concurrently, the last tile of all of them finishes the step.  fused_tile_rows: the step's
// number of tile rows for the precision.  mlp (FP32 piecewise-linear two-shock steps only, may be NULL):
// start the Riemann iterations from the learned proposal of these weights (FACE_LEARNED).
cudaError_t ctu_step_fused(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars* sc_cur,
                           StepScalars* sc_next, DevScratch* scr, double tmax, const CUtensorMap* tmap,
                           cudaStream_t stream, int2 band = make_int2(0, 0), const MlpBlob* mlp = nullptr);
int fused_tile_rows(int precision, const KParams& P);
int fused_tile_height(int precision);

// Conserved totals into scr->totals (deterministic two-level reduction; partials has room for
// totals_max_blocks() * 4 doubles).
int totals_max_blocks();
cudaError_t conserved_totals(int precision, const KParams& P, const void* U, double* partials, DevScratch* scr,
                             cudaStream_t stream);

// One fused CTU step Uin -> Uout with the time-step factors from sc_dev if not NULL, else sc_host.
// mode: FACE_PLAIN, FACE_HARVEST or FACE_LEARNED (the last two FP32 only; hook carries their buffers).
cudaError_t ctu_step(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars& sc_host,
                     const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream, int mode = 0,
                     const FaceHook* hook = nullptr, const CUtensorMap* tmap = nullptr);

// The same two launches with the HLLC solver at every face (k_ctu_hllc.cu, k_ctu_hllc_f64.cu); ctu_step and
// ctu_step_fused dispatch to them when P.riemann_solver == 1.
cudaError_t ctu_step_hllc(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars& sc_host,
                          const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream, const CUtensorMap* tmap);
cudaError_t ctu_step_fused_hllc(int precision, const KParams& P, const void* Uin, void* Uout,
                                const StepScalars* sc_cur, StepScalars* sc_next, DevScratch* scr, double tmax,
                                const CUtensorMap* tmap, cudaStream_t stream, int2 band);
cudaError_t ctu_step_hllc_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars& sc_host,
                              const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream);
cudaError_t ctu_step_fused_hllc_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars* sc_cur,
                                    StepScalars* sc_next, DevScratch* scr, double tmax, cudaStream_t stream,
                                    int2 band);

// The same two launches with piecewise-parabolic reconstruction, with either solver (k_ctu_ppm.cu,
// k_ctu_ppm_f64.cu); ctu_step and ctu_step_fused dispatch to them when P.reconstruction == 1.
cudaError_t ctu_step_ppm(int precision, const KParams& P, const void* Uin, void* Uout, const StepScalars& sc_host,
                         const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream, const CUtensorMap* tmap);
cudaError_t ctu_step_fused_ppm(int precision, const KParams& P, const void* Uin, void* Uout,
                               const StepScalars* sc_cur, StepScalars* sc_next, DevScratch* scr, double tmax,
                               const CUtensorMap* tmap, cudaStream_t stream, int2 band);
cudaError_t ctu_step_ppm_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars& sc_host,
                             const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream);
cudaError_t ctu_step_fused_ppm_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars* sc_cur,
                                   StepScalars* sc_next, DevScratch* scr, double tmax, cudaStream_t stream,
                                   int2 band);

// Tile box of the FP32 single-problem step kernels (the TMA box is (F32_TILE_X + 8) x (F32_TILE_Y + 8) x 4).
int f32_tile_x();
int f32_tile_y();

// FP64 forms of the two step launches (k_ctu_f64.cu, compiled without multiply-add contraction).
cudaError_t ctu_step_fused_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars* sc_cur,
                               StepScalars* sc_next, DevScratch* scr, double tmax, cudaStream_t stream,
                               int2 band = make_int2(0, 0));
cudaError_t ctu_step_f64(const KParams& P, const double* Uin, double* Uout, const StepScalars& sc_host,
                         const StepScalars* sc_dev, DevScratch* scr, cudaStream_t stream);

// One sweep of the dimensionally split variant (sweep_kernels.cuh) along dir (0: x, 1: y) of the state Uin
// into Uout (interior cells only; halo cells outside the domain are read through the boundary map, so Uin
// needs no ghost fill), with sigma = dt/dx or dt/dy from sc_dev if not NULL, else sc_host.  check_state:
// flag non-finite / non-positive cells of the result in the status word.  sc_next != NULL: the second sweep
// of a fused step -- also reduce the CFL dt of the result; the last block advances the device time by this
// step's dt and writes the next step's factors to sc_next (dt clamped to reach tmax when tmax > 0).
cudaError_t split_sweep(int precision, const KParams& P, const void* Uin, void* Uout, int dir,
                        const StepScalars& sc_host, const StepScalars* sc_dev, DevScratch* scr, int check_state,
                        StepScalars* sc_next, double tmax, cudaStream_t stream);
cudaError_t split_sweep_f64(const KParams& P, const double* Uin, double* Uout, int dir, const StepScalars& sc_host,
                            const StepScalars* sc_dev, DevScratch* scr, int check_state, StepScalars* sc_next,
                            double tmax, cudaStream_t stream);
// The same sweeps with piecewise-parabolic reconstruction (k_split_ppm.cu, k_split_ppm_f64.cu); split_sweep
// dispatches to them when P.reconstruction == 1.
cudaError_t split_sweep_ppm(int precision, const KParams& P, const void* Uin, void* Uout, int dir,
                            const StepScalars& sc_host, const StepScalars* sc_dev, DevScratch* scr, int check_state,
                            StepScalars* sc_next, double tmax, cudaStream_t stream);
cudaError_t split_sweep_ppm_f64(const KParams& P, const double* Uin, double* Uout, int dir,
                                const StepScalars& sc_host, const StepScalars* sc_dev, DevScratch* scr,
                                int check_state, StepScalars* sc_next, double tmax, cudaStream_t stream);

// Host copy of the device hash32 (mlp.cuh), for per-step sampling seeds.
inline unsigned int host_hash32(unsigned int x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Kernel parameters of one problem from the public parameters (validated by the caller).
void fill_kparams(const hydro_params* p, KParams* k);

// Copy `rows` dense host rows of row_bytes each (host_dev: device-side address of pinned, mapped host memory)
// into the device array dst with a row pitch of dst_pitch_bytes.
cudaError_t upload_rows(const void* host_dev, void* dst, size_t row_bytes, size_t dst_pitch_bytes, int rows,
                        cudaStream_t stream);

// TMA descriptor of one FP32 state buffer with the (tile_x + 8) x (tile_y + 8) x 4 box of a tile (host);
// 0 when the precision, alignment or driver does not allow one.
int make_state_tensor_map(CUtensorMap* map, const KParams& k, int precision, void* base, int tile_x, int tile_y);

// Scratch initialisation (min accumulator = +inf, counters 0).
cudaError_t init_scratch(DevScratch* scr, cudaStream_t stream);

}  // namespace hydro
