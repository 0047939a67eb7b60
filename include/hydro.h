/*
 * hydro.h -- C ABI of the GB300 (sm_103a) library for the unsplit piecewise-linear Godunov / CTU step
 * of a gamma-law gas in 2-D (paper §3.2 "Compressible hydrodynamics", Eqs. 8-13, built on the CTU
 * construction of §3.1, Eqs. 3-6).
 *
 * The calls follow the paper's single driver loop (§2): fill boundary conditions, get the time step,
 * evolve one step, t += dt.  All compute runs in the library's CUDA kernels on the caller's stream.
 *
 * Conventions shared by every call
 *  - Plain C types only.  "Device pointer" means memory from cudaMalloc (or any allocator handing out
 *    device memory, e.g. PyTorch) on the device that is current when hydro_init is called.
 *  - Every call returns a hydro_status and never aborts or throws.  On failure the context keeps a
 *    message retrievable with hydro_last_error().
 *  - Invalid parameters are rejected with HYDRO_EINVAL before anything is allocated or launched.
 *  - Calls on one context are not thread safe; different contexts are independent.
 *
 * State layout (device): structure of arrays U[k][j][i] with k in {rho, rho u, rho v, rho E},
 * j in [0, ny + 2 ng) the row (y), i in [0, nx + 2 ng) the column (x).  Element (k, j, i) lives at
 * offset (k * (ny + 2 ng) + j) * pitch + i, with pitch = hydro_state_pitch(params) elements (the row
 * length rounded up so every row starts on a 128-byte boundary).  Interior cells are
 * i in [ng, ng + nx), j in [ng, ng + ny); the ng >= 4 cells around them are ghost cells.  Element type
 * is double for HYDRO_FP64 and float for HYDRO_FP32.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HYDRO_OK = 0,
  HYDRO_EINVAL = 1,      /* bad argument or parameter */
  HYDRO_ENOMEM = 2,      /* device or host allocation failed */
  HYDRO_ECUDA = 3,       /* a CUDA runtime call failed (message in hydro_last_error) */
  HYDRO_ENONFINITE = 4,  /* a NaN or Inf was found in the state */
  HYDRO_ENEGATIVE = 5,   /* density or pressure <= 0 was found in the state */
  HYDRO_ENONCONV = 6,    /* at least one Riemann solve hit riemann_maxiter without converging */
  HYDRO_ETIMEOUT = 7,    /* a bounded device-side wait ran out */
  HYDRO_ERANGE = 8       /* a size is beyond a fixed maximum of the call (see the call) */
} hydro_status;

/* Boundary conditions (paper §2 ghost cells; §3.2 Rayleigh-Taylor problem for the hydrostatic wall).
 * OUTFLOW: zero gradient.  PERIODIC: wrap (both sides of an axis).  REFLECT: mirror image of the interior
 * with the normal momentum negated.  HYDROSTATIC (y sides only): density and momenta copied from the row
 * next to the wall, pressure integrated with dp/dy = rho g from that row's cell, energy rebuilt from it.
 * The fused step (hydro_step_fused, hydro_advance) and the split sweeps read every kind of side through
 * the same map instead of a ghost fill. */
typedef enum {
  HYDRO_BC_OUTFLOW = 0,
  HYDRO_BC_PERIODIC = 1,
  HYDRO_BC_REFLECT = 2,
  HYDRO_BC_HYDROSTATIC = 3
} hydro_bc;

/* Riemann solvers (paper §3.2).  TWO_SHOCK: Newton iteration of the two-shock approximation (the default).
 * HLLC: Toro's three-wave HLLC flux, outer wave speeds min(u_L - c_L, u_R - c_R), max(u_L + c_L, u_R + c_R);
 * no iterations (the iteration counters then stay 0). */
typedef enum { HYDRO_RIEMANN_TWO_SHOCK = 0, HYDRO_RIEMANN_HLLC = 1 } hydro_riemann;

/* Reconstruction of the interface states (paper §3.2).  PLM: limited linear profiles (the paper's method).
 * PPM: Colella & Woodward's parabolic profiles (MC-limited interface values, monotonicity constraints,
 * flattening toward the cell average) traced along the characteristics, the fastest wave's average as the
 * reference state. */
typedef enum { HYDRO_RECON_PLM = 0, HYDRO_RECON_PPM = 1 } hydro_recon;

typedef enum {
  HYDRO_FP64 = 0, /* state and arithmetic in double */
  HYDRO_FP32 = 1  /* state and stencil arithmetic in float; the pressure of a cell whose kinetic energy
                     is within 0.1% of its total energy (recover_ke_frac) is recomputed in double; dt and
                     conserved totals are reduced in double */
} hydro_precision;

/* Parameters of one problem (the paper's RuntimeParameters for the compressible solver, §2). */
typedef struct {
  int nx, ny;                       /* interior cells, >= 1 */
  int ng;                           /* ghost cells per side, must be >= 4 (stencil reach of the step) */
  double xmin, xmax, ymin, ymax;    /* domain; dx = (xmax - xmin)/nx, dy = (ymax - ymin)/ny */
  double gamma;                     /* gamma-law EOS p = rho e (gamma - 1) (Eq. 12), > 1 */
  double cfl;                       /* CFL number C of Eq. 6, > 0 */
  int bc_xlo, bc_xhi, bc_ylo, bc_yhi; /* hydro_bc; periodic sides must be paired and have n >= ng */
  int limiter;                      /* 0 piecewise constant, 1 MC, 2 fourth-order MC (default) */
  int use_flattening;               /* shock flattening, 0/1 (default 1) */
  double cvisc;                     /* artificial-viscosity coefficient (default 0.1), >= 0 */
  int riemann_maxiter;              /* Newton iteration cap of the two-shock solver (default 32) */
  double riemann_tol;               /* relative |dp|/p stopping tolerance (default 1e-14 FP64, 1e-6 FP32) */
  double small_dens, small_pres;    /* floors on working copies only, never on the stored state */
  int precision;                    /* hydro_precision */
  int use_learned_guess;            /* 1: start each Riemann iteration from a learned proposal (FP32 only;
                                       see hydro_set_riemann_model), default 0 */
  double grav;                      /* constant gravitational acceleration along y (paper §3.2 Euler
                                       equations' rho g and rho U.g sources), default 0 */
  int split;                        /* 0: unsplit CTU step (default).  1: dimensionally split step (paper
                                       §3.1: a one-dimensional sweep along x and one along y, each acting on
                                       the state the other left; the context's k-th step, counted from
                                       hydro_init, sweeps x first when k is even; gravity's sources are
                                       added by the y sweep).  Needs use_learned_guess = 0; single problems
                                       only (not hydro_batch_*). */
  int riemann_solver;               /* hydro_riemann: the two-shock iteration (default) or HLLC (§3.2 names
                                       both; HLLC needs use_learned_guess = 0, no harvest, and is for single
                                       problems only, not hydro_batch_*) */
  int reconstruction;               /* hydro_recon: piecewise linear (default; `limiter` applies) or
                                       piecewise parabolic (the PPM upgrade §3.2 points to; `limiter` is
                                       unused; same restrictions as HLLC) */
  double recover_ke_frac;           /* FP32 only (EOS of Eqs. 11-12): where the kinetic energy of a cell or
                                       face state exceeds this fraction of its total energy, the pressure
                                       (gamma - 1)(E - rho |u|^2 / 2) is recomputed in double from the float
                                       conserved values, so the cancellation of E - rho |u|^2 / 2 is not left
                                       to float arithmetic.  Default 0.999; 0 recomputes every one; a value
                                       above 1 never does.  Must be finite and >= 0.  FP64 ignores it. */
} hydro_params;

typedef struct hydro_ctx hydro_ctx;

/* Fill *p with the defaults above for an nx x ny grid on [0,1]^2, outflow on all sides, FP64.
 * Returns HYDRO_EINVAL if p is NULL. */
hydro_status hydro_default_params(hydro_params* p, int nx, int ny, int precision);

/* sizeof(hydro_params) as compiled into the library, for bindings that mirror the struct. */
size_t hydro_params_size(void);

/* Row pitch (elements) and total byte size of one state array for these parameters; 0 if invalid. */
size_t hydro_state_pitch(const hydro_params* p);
size_t hydro_state_bytes(const hydro_params* p);

/* Paper §2 Simulation.initialize(): validate parameters and create a context.
 *   d_state, d_state_alt: two caller-owned device buffers of hydro_state_bytes(p) bytes each, in the
 *     layout above.  The library borrows them (they must outlive the context): a step reads the current
 *     one and writes the other, then they swap roles.  d_state holds the initial state.
 *   cuda_stream: a cudaStream_t (NULL = legacy default stream) on which every kernel is launched.
 * The context allocates its own small device scratch (reduction partials, status word, time).
 * Errors: HYDRO_EINVAL (bad params or NULL/unaligned pointers: both buffers must be 256-byte aligned),
 * HYDRO_ENOMEM, HYDRO_ECUDA. */
hydro_status hydro_init(const hydro_params* p, void* d_state, void* d_state_alt, void* cuda_stream, hydro_ctx** out);

/* Release the context's own resources (not the borrowed state buffers).  NULL is a no-op. */
void hydro_destroy(hydro_ctx* ctx);

/* Device pointer of the buffer that currently holds the state (d_state or d_state_alt). */
void* hydro_state(const hydro_ctx* ctx);

/* Fill the ghost cells of the current state (paper §2, CellCenterData2d ghost filling; Fig. 1):
 * outflow copies the nearest interior cell (zero gradient), periodic wraps, reflect mirrors with the
 * normal momentum negated, hydrostatic integrates the pressure (see hydro_bc); a ghost cell (i, j) takes
 * its value from interior cell (map_x(i), map_y(j)), which also defines the corners.  Async. */
hydro_status hydro_fill_ghost(hydro_ctx* ctx);

/* CFL time step (Eq. 6 with signal speeds |u| + c and |v| + c):
 * *dt_out = cfl * min over interior cells of min(dx/(|u|+c), dy/(|v|+c)), c = sqrt(gamma p / rho).
 * Synchronises the stream.  Also checks the state: returns HYDRO_ENONFINITE / HYDRO_ENEGATIVE (and
 * leaves *dt_out unchanged) if any interior cell is non-finite or has rho <= 0 or p <= 0. */
hydro_status hydro_cfl_dt(hydro_ctx* ctx, double* dt_out);

/* One unsplit CTU step of length dt > 0 on the (ghost-filled) current state (paper §3.2 algorithm,
 * update Eq. 5): slopes + flattening, characteristic tracing (Eq. 13), Riemann solves on the traced
 * states, transverse flux-difference correction, final Riemann solves + artificial viscosity,
 * conservative update, with the Riemann solver and reconstruction the parameters select.  Writes the other buffer and swaps.  Asynchronous: problems found on the device
 * (non-finite or non-positive results, unconverged Riemann solves) are recorded in the context's status
 * word and reported by hydro_sync_status().  With split = 1 the step is the dimensionally split one (§3.1):
 * a one-dimensional sweep into the other buffer and the other sweep back into the current buffer (two
 * launches; cells outside the domain are read through the boundary map). */
hydro_status hydro_step(hydro_ctx* ctx, double dt);

/* CFL time step kept on the device: reduce the dt of hydro_cfl_dt into the context's device memory,
 * clamp it so the simulated time does not pass tmax (tmax <= 0: no clamp), and advance the device-side
 * time and step counter by it.  Asynchronous (no host synchronisation); the state checks of
 * hydro_cfl_dt are recorded in the status word instead of returned. */
hydro_status hydro_cfl_dt_async(hydro_ctx* ctx, double tmax);

/* hydro_step with the time step produced by the last hydro_cfl_dt_async on this context (read on the
 * device).  Asynchronous. */
hydro_status hydro_step_device_dt(hydro_ctx* ctx);

/* The driver loop of §2 kept on the device: for each of nsteps steps, fill ghosts, reduce the CFL dt
 * into device memory, clamp it so the simulated time does not pass tmax (tmax <= 0: no clamp), and step
 * with it.  No host synchronisation; time and step count stay on the device (hydro_get_time). */
hydro_status hydro_advance(hydro_ctx* ctx, int nsteps, double tmax);
/* Same results as nsteps x {hydro_fill_ghost, hydro_cfl_dt_async(tmax), hydro_step_device_dt}, run as
 * nsteps x hydro_step_fused(tmax); the ghost cells of the final state are not filled. */

/* One step of the driver loop as a single kernel launch: the step kernel reads ghost cells through the
 * boundary conditions' map of the interior (the values hydro_fill_ghost would write, for every kind of
 * side, so no fill pass), and reduces the CFL time step of the state it writes (so no dt pass); its last
 * block advances the device time by this step's dt and keeps the next step's dt (clamped to reach tmax
 * when tmax > 0).  The
 * first call after any other state change (hydro_step, hydro_step_device_dt, hydro_upload) computes this
 * step's dt with one extra reduction.  With split = 1: the two sweeps of hydro_step, the second one
 * reducing the next dt.  FP32 contexts with a learned model or a harvest run the separate passes instead.
 * Asynchronous. */
hydro_status hydro_step_fused(hydro_ctx* ctx, double tmax);

/* One step with host-resident state: host_in (pinned, layout of hydro_upload) is uploaded, stepped as
 * hydro_step_fused(tmax) does, and the new state written to host_out (layout of hydro_download; must not
 * be host_in).  The rows go up into an unpitched device copy of the state, one chunk per band of tile
 * rows; the fused step runs as one launch per band (five bands) on the context's own streams, and each
 * band's rows are copied back while later bands compute.  The whole pipeline is captured once as a CUDA
 * graph for each pair of host buffers (and tmax) and replayed.  Returns when host_out holds the new state; the
 * context's current buffer holds it too.  The interior of host_out and of the current state equals what
 * hydro_upload, hydro_step_fused and hydro_download give; ghost cells are not filled (host_out's read as
 * 0 or as the values an earlier step left there).  Contexts with a learned model, a harvest or split = 1
 * run those three calls in turn.  The first call allocates two device copies of the state (unpitched,
 * 4 (nx + 2 ng)(ny + 2 ng) elements each), which the context keeps until hydro_destroy.
 * Errors: HYDRO_EINVAL (NULL pointers, host_in == host_out), HYDRO_ECUDA. */
hydro_status hydro_step_host(hydro_ctx* ctx, const void* host_in, void* host_out, double tmax);

/* hydro_step_host for a run kept in host memory, step after step: when host_in is the host_out of the
 * previous hydro_step_host / hydro_step_host_chained call on this context, unchanged since, with the same
 * tmax and no other call that steps or replaces the state in between, this step's CFL time step is the
 * one the previous step reduced from the state it wrote (as hydro_step_fused keeps it), so no reduction
 * waits for the whole upload: each band of tile rows starts as soon as its rows and their 4-row halo
 * have arrived (eight bands), and the upload overlaps the step.  Otherwise the same as hydro_step_host.  The caller
 * must not modify host_out between the calls (the library checks the pointer, not the contents).  Same
 * results as hydro_step_host. */
hydro_status hydro_step_host_chained(hydro_ctx* ctx, const void* host_in, void* host_out, double tmax);

/* Simulated time and number of steps of the device-side loop (hydro_cfl_dt_async, hydro_step_fused,
 * hydro_advance, hydro_step_host; hydro_step with a host dt does not count).  Synchronises. */
hydro_status hydro_get_time(hydro_ctx* ctx, double* t, long long* nsteps);

/* Conserved totals out[k] = sum over interior cells of U_k dx dy, accumulated in double in a fixed
 * order (deterministic).  Synchronises. */
hydro_status hydro_conserved_totals(hydro_ctx* ctx, double out[4]);

/* Conserved totals for callers that cannot allocate device memory (no counterpart in the paper; it is
 * a runtime convenience).  Such callers are code running while another allocator owns the device memory
 * (a framework's caching allocator or a fixed pool, where a stray cudaMalloc would fragment or overrun
 * the budget) and diagnostics taken after an out-of-memory error, when cudaMalloc itself fails.
 *   p:        parameters of the state (validated as in hydro_init).
 *   d_state:  device pointer to one state in the layout above, ghost cells need not be filled.
 *   cuda_stream: the stream to run on (NULL = legacy default stream).
 *   out:      host array receiving sum over interior cells of U_k dx dy, k = 0..3, accumulated in double.
 * Needs no context and calls no cudaMalloc, cudaFree or other allocating routine.  Its reduction scratch
 * is one file-scope device array of (4 HYDRO_NOALLOC_MAX_ROWS + 8) doubles (512 KB), which every GPU
 * that loads the library holds until the process exits.  The first call on a device looks up that
 * array's device address (with that device current) and caches it for the rest of the process, so make
 * the first call on each device before any stream capture; a cudaDeviceReset of the device invalidates the
 * cached address, and calls after one are not supported.  Every call shares the one array: calls whose
 * kernels overlap on the GPU (two streams, two threads) race and return wrong totals; serialise them.
 * The call synchronises the stream and copies the totals into `out` before it returns.
 * Errors: HYDRO_EINVAL (bad params or NULL pointers), HYDRO_ERANGE (ny > HYDRO_NOALLOC_MAX_ROWS),
 * HYDRO_ECUDA. */
#define HYDRO_NOALLOC_MAX_ROWS 16384
hydro_status hydro_conserved_totals_noalloc(const hydro_params* p, const void* d_state, void* cuda_stream,
                                            double out[4]);

/* Read and clear the device status word: HYDRO_OK, or the first of HYDRO_ENONFINITE, HYDRO_ENEGATIVE,
 * HYDRO_ENONCONV, HYDRO_ETIMEOUT (a tile's TMA copy did not land within the bounded wait) recorded since
 * the last call.  After HYDRO_ETIMEOUT the state the steps wrote is not to be trusted: discard it and
 * upload a known state again (hydro_last_error says whether a copy was still outstanding when its tile
 * gave up, in which case later tiles on the same SM may have been overwritten as well).  Synchronises.  If stats is not NULL it receives
 * {riemann solves, riemann iterations, unconverged solves} accumulated since hydro_init. */
hydro_status hydro_sync_status(hydro_ctx* ctx, unsigned long long stats[3]);

/* Copy a host array into / out of the current state.  host has the dense layout
 * [4][ny + 2 ng][nx + 2 ng] (no pitch) of the context's element type.  Pinned host memory makes the
 * copies asynchronous; the call returns after enqueueing (upload) or after the copy (download).  An upload
 * from pinned memory the device can address is done by a copy kernel reading the host memory directly
 * (faster than the copy engine for this pitched copy on a Grace system); the host buffer must then stay
 * unchanged until the stream has passed the upload. */
hydro_status hydro_upload(hydro_ctx* ctx, const void* host);
hydro_status hydro_download(hydro_ctx* ctx, void* host);

/* ---- Learned starting pressure for the two-shock iteration -----------------------------------------
 * Not in the paper, which starts the iteration of §3.2 from the acoustic (linearised) estimate.  A small
 * network (6 -> 64 -> 64 -> 1, ReLU) proposes ln(p_star / p_ref) from the face's left/right (rho, u_n, p) in
 * reference units (rho_ref = sqrt(rho_L rho_R), p_ref = sqrt(p_L p_R), c_ref = sqrt(p_ref/rho_ref),
 * velocities relative to their mean); the Newton iteration then runs from that proposal to the same
 * tolerance, so the answer is still decided by the method.  Training data are faces sampled from CTU
 * steps (hydro_set_harvest).  FP32 contexts only.  Inference runs on the tensor cores (BF16 weights and
 * activations, FP32 accumulation), 32 faces per warp; a warp evaluates the network only when one of its
 * faces has |ln(p_L/p_R)|/2 > gate_dp or |u_L - u_R|/c_ref > gate_du, otherwise its faces start from the
 * acoustic estimate. */
typedef struct hydro_mlp hydro_mlp;

/* Create a network with He-normal weights drawn from `seed` (counter-based generator on the device).
 * Parameter vector (4673 floats): W1[64][6], b1[64], W2[64][64], b2[64], W3[64], b3. */
hydro_status hydro_mlp_create(unsigned long long seed, void* cuda_stream, hydro_mlp** out);
void hydro_mlp_destroy(hydro_mlp* m);
hydro_status hydro_mlp_set_weights(hydro_mlp* m, const float* host_theta);
hydro_status hydro_mlp_get_weights(hydro_mlp* m, float* host_theta);
/* Gate of the fused inference (defaults 0.35 and 1.0). */
hydro_status hydro_mlp_set_gate(hydro_mlp* m, double gate_dp, double gate_du);
/* Gradient (host array of 4673 floats) and loss of the mean squared error of ln(p_star / p_ref) over n
 * samples.  d_samples: device array [n][8] = (rho_L, u_L, p_L, rho_R, u_R, p_R, p*, iterations). */
hydro_status hydro_mlp_gradient(hydro_mlp* m, const float* d_samples, long long n, float* host_grad, double* loss);
/* `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on minibatches of `batch` samples
 * (a multiple of 64) drawn from d_samples with a counter-based generator seeded by `seed`; *last_loss
 * receives the last minibatch's loss.  Synchronises. */
hydro_status hydro_mlp_train(hydro_mlp* m, const float* d_samples, long long n, int steps, int batch, double lr,
                             unsigned long long seed, double* last_loss);
/* Network outputs y = ln(p_star / p_ref) of n samples into the device array d_out, with the FP32 master weights
 * (use_tensor_cores = 0) or the BF16 tensor-core inference path (1). */
hydro_status hydro_mlp_predict(hydro_mlp* m, const float* d_samples, long long n, int use_tensor_cores, float* d_out);
/* Diagnostic: mean FP32 two-shock iterations per sample (tolerance tol, cap maxiter, EOS gamma) of n
 * device samples when started from the acoustic estimate (learned = 0) or from the network (learned = 1,
 * tensor-core inference, no gate); *nonconv receives the unconverged count.  Synchronises. */
hydro_status hydro_mlp_iterations(hydro_mlp* m, const float* d_samples, long long n, int learned, double gamma,
                                  double tol, int maxiter, double* mean_iters, long long* nonconv);
/* Device address of the packed inference weights (for the CTU kernels). */
const void* hydro_mlp_device_blob(const hydro_mlp* m);
const char* hydro_mlp_last_error(const hydro_mlp* m);

/* Use network m as the starting pressure of every Riemann solve of ctx's steps (the context must have been
 * created with use_learned_guess = 1; m = NULL clears it).  m must outlive its use. */
hydro_status hydro_set_riemann_model(hydro_ctx* ctx, const hydro_mlp* m);

/* Record Riemann problems during steps: each face solve is kept with probability `rate` (hash of the face
 * and the step), writing 8 floats (rho_L, u_L, p_L, rho_R, u_R, p_R, p*, iterations) at slot
 * atomicAdd(d_count, 1) of the device buffer d_buf while the slot is < capacity.  d_count is a caller-owned
 * device counter (zero it before use).  d_buf = NULL stops recording.  FP32 contexts only. */
hydro_status hydro_set_harvest(hydro_ctx* ctx, void* d_buf, unsigned long long capacity, double rate,
                               unsigned long long* d_count);

/* Also record every face past the learned proposal's gate (|ln(p_L/p_R)|/2 >= gate_dp or
 * |u_L - u_R| / c_ref >= gate_du, see hydro_mlp_set_gate), whatever its hash, so that the rare faces the
 * network is used on are not thinned out with the rest.  gate_dp <= 0 and gate_du <= 0 switch it off
 * (the default).  Returns HYDRO_EINVAL for a half-set gate (one of them <= 0) or values beyond
 * gate_dp = 40, gate_du = 1e9.  No paper counterpart (training-data selection). */
hydro_status hydro_set_harvest_gate(hydro_ctx* ctx, double gate_dp, double gate_du);

/* ---- Ensembles of independent problems (uneven grids, own time steps) ----------------------------
 * Not in the paper, which runs one problem at a time; this batches many independent copies of the §2
 * driver loop.  Each member has its own parameters (all members share one precision) and two caller-owned
 * state buffers, as for hydro_init.  A run of n steps = the CFL dt of every member (its own), then n fused
 * CTU steps of every member with its own dt: each step runs as one persistent kernel per tile shape whose
 * CTAs take tiles of any member from a work queue, read ghost cells through the member's boundary map, and
 * reduce the member's next dt (the member's last tile hands it on).  Ghost cells of the states are not
 * filled. */
typedef struct hydro_batch hydro_batch;

/* Create an ensemble of n members.  params, d_states, d_states_alt: arrays of n entries.  Members take the
 * unsplit piecewise-linear step with the two-shock solver; all share one precision and one use_learned_guess
 * (1: FP32 members whose iterations start from the network set by hydro_batch_set_riemann_model).
 * Errors: HYDRO_EINVAL (bad member, mixed precisions or use_learned_guess, split = 1, the HLLC solver or PPM),
 * HYDRO_ENOMEM, HYDRO_ECUDA. */
hydro_status hydro_batch_create(int n, const hydro_params* params, void* const* d_states, void* const* d_states_alt,
                                void* cuda_stream, hydro_batch** out);
void hydro_batch_destroy(hydro_batch* b);

/* Start every member's Riemann iterations from the learned proposal of network m (see hydro_set_riemann_model;
 * the members must have been created with use_learned_guess = 1; m = NULL clears it, and such an ensemble
 * then refuses to run).  One copy of the weights serves all members; warps read it from global memory only
 * where their gate opens.  m must outlive its use.  Captured graphs are dropped when m changes. */
hydro_status hydro_batch_set_riemann_model(hydro_batch* b, const hydro_mlp* m);

/* Tile-shape autotuner: for every size class time `reps` launches of each candidate tile shape on the
 * current states (without advancing them) and keep the fastest.  chosen_shapes (optional) receives one
 * shape id per class.  Synchronises.  Cached graphs are dropped. */
hydro_status hydro_batch_autotune(hydro_batch* b, int reps, int* chosen_shapes);

/* Size classes (largest first) and the tile shape each uses. */
int hydro_batch_num_classes(const hydro_batch* b);
hydro_status hydro_batch_class_info(const hydro_batch* b, int k, int* nx, int* ny, int* members, int* tile_x,
                                    int* tile_y, int* threads);

/* Advance every member by nsteps steps, each with its own CFL dt.  use_graph != 0: the nsteps steps are
 * captured once into a CUDA graph (cached per nsteps and buffer parity) and launched as one graph;
 * use_graph = 0 launches the kernels directly.  Asynchronous. */
hydro_status hydro_batch_run(hydro_batch* b, int nsteps, int use_graph);

/* Device pointer of the buffer holding member i's current state. */
void* hydro_batch_state(const hydro_batch* b, int member);

/* Member time and step count (synchronises). */
hydro_status hydro_batch_get_time(hydro_batch* b, int member, double* t, long long* nsteps);

/* Read and clear the status words of the ensemble (first of HYDRO_ENONFINITE, HYDRO_ENEGATIVE,
 * HYDRO_ENONCONV); stats receives {riemann solves, iterations, unconverged} of the step kernels. */
hydro_status hydro_batch_sync_status(hydro_batch* b, unsigned long long stats[3]);

/* Conserved totals of member i (as hydro_conserved_totals; synchronises). */
hydro_status hydro_batch_conserved_totals(hydro_batch* b, int member, double out[4]);

const char* hydro_batch_last_error(const hydro_batch* b);

/* Message of the last failure on this context ("" if none).  Valid until the next call. */
const char* hydro_last_error(const hydro_ctx* ctx);

/* Library build string (compute capability and options), never NULL. */
const char* hydro_build_info(void);

/* 1 if the context's step kernels load tiles by TMA bulk tensor copies (FP32 contexts with ng a multiple of
 * 4 on a driver that provides the tensor-map encoder; tiles whose halo leaves the interior, or the padded
 * array for the unfused step, are still loaded cell by cell), 0 otherwise or if ctx is NULL.  No paper
 * counterpart: how the data reaches shared memory does not change what a step computes. */
int hydro_tma_enabled(const hydro_ctx* ctx);

/* Failure-path test of the bounded device-side wait (no paper counterpart).  drop = 1: the step kernels
 * issue no TMA tile copy, so each such tile's mbarrier waits for bytes that never arrive; the wait gives up
 * after `polls` polls (1000 if 0), the tile is left unwritten and the status word records a timeout
 * (HYDRO_ETIMEOUT from hydro_sync_status).  Nothing is in flight when a tile gives up, and the context
 * stays usable.  drop = 0 restores normal operation.  Returns HYDRO_EINVAL for other values of drop. */
hydro_status hydro_test_drop_tile_copies(hydro_ctx* ctx, int drop, unsigned int polls);

#ifdef __cplusplus
}
#endif
#endif
