// C-ABI layer (include/hydro.h): parameter validation, context, scratch, and kernel launches on the
// caller's stream.  The calls follow the single driver loop of the paper (§2): fill boundary conditions,
// get the time step, evolve one step.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "../../include/hydro.h"
#include "hydro_kernels.h"

using hydro::DevScratch;
using hydro::KParams;

struct hydro_ctx {
  hydro_params p;
  KParams kp;
  void* state[2];
  int cur;
  cudaStream_t stream;
  int device;
  DevScratch* scr;  // device
  double* partials; // device, totals per-block partials
  DevScratch* host_scr;  // pinned host mirror for reads
  // optional face-solve variants (FP32 contexts)
  hydro::FaceHook hook;  // harvest buffer and counter, network weights
  int harvest;           // 1: sample Riemann inputs and star pressures during steps
  const hydro_mlp* mlp;  // learned starting pressure, used when p.use_learned_guess == 1
  unsigned int step_calls;
  // fused steps: the factors of the next step are in scr->scf[fused_parity] when fused_valid
  int fused_parity;
  int fused_valid;
  // FP32: TMA descriptors of the two state buffers (tile loads by bulk tensor copy) when tma_ok
  CUtensorMap tmap[2];
  int tma_ok;
  unsigned long long split_steps;  // split variant: steps taken (x sweep first on even counts)
  // host steps (created on first use): streams for the bands of the fused step, for the copies up and
  // for the copies back, and their events; two unpitched copies of the state (input and output of the
  // banded step).  Without row padding a band's rows in the four planes are four contiguous blocks, which
  // one 2-D copy (a row per plane) moves at the link's rate; the copy engine moves the padded layout's
  // 4 KB rows at under half of it.
  static constexpr int HOST_BANDS = 8;
  int host_pipe;
  cudaStream_t band_stream[HOST_BANDS];
  cudaStream_t d2h_stream, h2d_stream;
  cudaEvent_t ev_ready, ev_start, ev_done, ev_band[HOST_BANDS], ev_up[HOST_BANDS];
  void* stage[2];
  CUtensorMap stage_map;  // of stage[0], when stage_tma
  int stage_tma;
  // host steps replay as CUDA graphs: the pipeline of one host step (copies up, bands, copies back, the
  // copy into the context's buffer) is captured once for each set of values it bakes in and then runs as
  // one launch instead of ~40 API calls (KH 64^2 FP32, chained: 46 us per step against 53 us; at 1024^2
  // the link bounds the step either way); a few graphs are kept, replaced in turn
  static constexpr int HOST_GRAPHS = 4;
  struct HostGraph {
    const void* in;
    void* out;
    int cur, parity, chained;
    double tmax;
    cudaGraphExec_t exec;
    int used;  // slot holds this key; exec == nullptr: its capture failed (the step then runs uncaptured)
  } hgraph[HOST_GRAPHS];
  int hgraph_next;
  // chained host steps: the buffer the last host step wrote, and the step count and tmax it left behind
  const void* chain_out;
  unsigned int chain_step;
  double chain_tmax;
  char err[512];
};

// The driver's tensor-map encoder, looked up once through the runtime (no link against the driver library).
typedef CUresult (*encode_tiled_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static encode_tiled_fn tensor_map_encoder() {
  static const encode_tiled_fn fn = [] {  // looked up once (thread-safe static initialisation)
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (encode_tiled_fn)f;
    return (encode_tiled_fn) nullptr;
  }();
  return fn;
}

namespace hydro {

// Describe one FP32 state buffer as a 3-D tensor (x over the padded width, y over the padded height, the 4
// conserved components) with a (tile_x + 8) x (tile_y + 8) x 4 box.  TMA wants 16-byte aligned bases and
// strides (buffers are 256-byte aligned and rows padded to 128 bytes) and 16-byte aligned x coordinates:
// tile boxes start at x = ng - 4 + k * tile_x, so ng - 4 and tile_x must be multiples of 4.  Returns 0
// (tiles then load cell by cell) when a condition or the encoder is missing.
int make_state_tensor_map(CUtensorMap* map, const KParams& k, int precision, void* base, int tile_x, int tile_y) {
  if (precision != HYDRO_FP32 || (k.ng - 4) % 4 != 0 || tile_x % 4 != 0) return 0;
  encode_tiled_fn enc = tensor_map_encoder();
  if (!enc) return 0;
  const cuuint64_t row = (cuuint64_t)k.pitch * sizeof(float);
  const cuuint64_t dims[3] = {(cuuint64_t)k.NX, (cuuint64_t)k.NY, 4};
  const cuuint64_t strides[2] = {row, row * (cuuint64_t)k.NY};
  const cuuint32_t box[3] = {(cuuint32_t)tile_x + 8, (cuuint32_t)tile_y + 8, 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (row % 16 != 0 || (uintptr_t)base % 16 != 0 || box[0] > 256 || box[1] > 256) return 0;
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace hydro

// Tensor maps of the context's two buffers for the single-problem FP32 tile.
static int make_tensor_maps(hydro_ctx* c) {
  for (int b = 0; b < 2; ++b)
    if (!hydro::make_state_tensor_map(&c->tmap[b], c->kp, c->p.precision, c->state[b], hydro::f32_tile_x(),
                                      hydro::f32_tile_y()))
      return 0;
  return 1;
}

static size_t elem_size(int precision) { return precision == HYDRO_FP32 ? sizeof(float) : sizeof(double); }

static int params_valid(const hydro_params* p, char* why, size_t n) {
#define BAD(msg)                       \
  do {                                 \
    if (why) snprintf(why, n, "%s", msg); \
    return 0;                          \
  } while (0)
  if (!p) BAD("params is NULL");
  if (p->nx < 1 || p->ny < 1) BAD("nx and ny must be >= 1");
  if (p->ng < 4) BAD("ng must be >= 4 (stencil reach of the CTU step)");
  if ((long long)(p->nx + 2 * p->ng) * (p->ny + 2 * p->ng) > (1ll << 31)) BAD("grid too large (padded cells > 2^31)");
  if (!(p->xmax > p->xmin) || !(p->ymax > p->ymin)) BAD("empty domain");
  if (!(p->gamma > 1.0)) BAD("gamma must be > 1");
  if (!(p->cfl > 0.0)) BAD("cfl must be > 0");
  const int bcs[4] = {p->bc_xlo, p->bc_xhi, p->bc_ylo, p->bc_yhi};
  for (int k = 0; k < 4; ++k)
    if (bcs[k] < HYDRO_BC_OUTFLOW || bcs[k] > HYDRO_BC_HYDROSTATIC) BAD("unknown boundary condition");
  if (p->bc_xlo == HYDRO_BC_HYDROSTATIC || p->bc_xhi == HYDRO_BC_HYDROSTATIC)
    BAD("hydrostatic boundaries are for the y sides (gravity acts along y)");
  // a mirrored ghost cell's source must be an interior cell
  if ((p->bc_xlo == HYDRO_BC_REFLECT || p->bc_xhi == HYDRO_BC_REFLECT) && p->nx < p->ng)
    BAD("reflecting x walls need nx >= ng");
  if ((p->bc_ylo == HYDRO_BC_REFLECT || p->bc_yhi == HYDRO_BC_REFLECT) && p->ny < p->ng)
    BAD("reflecting y walls need ny >= ng");
  if (!(p->grav > -1e30 && p->grav < 1e30)) BAD("grav must be finite");
  if ((p->bc_xlo == HYDRO_BC_PERIODIC) != (p->bc_xhi == HYDRO_BC_PERIODIC) ||
      (p->bc_ylo == HYDRO_BC_PERIODIC) != (p->bc_yhi == HYDRO_BC_PERIODIC))
    BAD("periodic boundaries must be paired");
  if (p->bc_xlo == HYDRO_BC_PERIODIC && p->nx < p->ng) BAD("periodic x needs nx >= ng");
  if (p->bc_ylo == HYDRO_BC_PERIODIC && p->ny < p->ng) BAD("periodic y needs ny >= ng");
  if (p->limiter < 0 || p->limiter > 2) BAD("limiter must be 0, 1 or 2");
  if (p->use_flattening != 0 && p->use_flattening != 1) BAD("use_flattening must be 0 or 1");
  if (!(p->cvisc >= 0.0)) BAD("cvisc must be >= 0");
  if (p->riemann_maxiter < 1 || p->riemann_maxiter > 1000) BAD("riemann_maxiter must be in [1, 1000]");
  if (!(p->riemann_tol > 0.0)) BAD("riemann_tol must be > 0");
  if (!(p->small_dens > 0.0) || !(p->small_pres > 0.0)) BAD("small_dens and small_pres must be > 0");
  if (p->precision != HYDRO_FP64 && p->precision != HYDRO_FP32) BAD("precision must be HYDRO_FP64 or HYDRO_FP32");
  if (p->precision == HYDRO_FP32 && (p->small_pres < 1e-30 || p->small_dens < 1e-30))
    BAD("FP32 floors must be normal float numbers (>= 1e-30)");
  if (p->use_learned_guess != 0 && p->use_learned_guess != 1) BAD("use_learned_guess must be 0 or 1");
  if (p->use_learned_guess == 1 && p->precision != HYDRO_FP32) BAD("the learned proposal is an FP32 path");
  if (p->split != 0 && p->split != 1) BAD("split must be 0 or 1");
  if (p->split == 1 && p->use_learned_guess != 0) BAD("the split variant has no learned proposal");
  if (p->riemann_solver != HYDRO_RIEMANN_TWO_SHOCK && p->riemann_solver != HYDRO_RIEMANN_HLLC)
    BAD("riemann_solver must be HYDRO_RIEMANN_TWO_SHOCK or HYDRO_RIEMANN_HLLC");
  if (p->riemann_solver == HYDRO_RIEMANN_HLLC && p->use_learned_guess != 0)
    BAD("the learned proposal starts the two-shock iteration; HLLC has none");
  if (p->reconstruction != HYDRO_RECON_PLM && p->reconstruction != HYDRO_RECON_PPM)
    BAD("reconstruction must be HYDRO_RECON_PLM or HYDRO_RECON_PPM");
  if (p->reconstruction == HYDRO_RECON_PPM && p->use_learned_guess != 0)
    BAD("the learned proposal runs with the piecewise-linear step only");
  if (!(p->recover_ke_frac >= 0.0 && p->recover_ke_frac < 1e30)) BAD("recover_ke_frac must be finite and >= 0");
  return 1;
#undef BAD
}

static void set_err(hydro_ctx* c, const char* fmt, ...) {
  if (!c) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof c->err, fmt, ap);
  va_end(ap);
}

static hydro_status cuda_fail(hydro_ctx* c, cudaError_t e, const char* where) {
  set_err(c, "%s: %s", where, cudaGetErrorString(e));
  return HYDRO_ECUDA;
}

namespace hydro {

// Kernel parameters of one problem (shared by single-problem contexts and ensembles).
void fill_kparams(const hydro_params* p, KParams* kp) {
  KParams& k = *kp;
  memset(&k, 0, sizeof k);
  k.nx = p->nx;
  k.ny = p->ny;
  k.ng = p->ng;
  k.pitch = (int)hydro_state_pitch(p);
  k.NX = p->nx + 2 * p->ng;
  k.NY = p->ny + 2 * p->ng;
  k.bc[0] = p->bc_xlo;
  k.bc[1] = p->bc_xhi;
  k.bc[2] = p->bc_ylo;
  k.bc[3] = p->bc_yhi;
  k.dx = (p->xmax - p->xmin) / p->nx;
  k.dy = (p->ymax - p->ymin) / p->ny;
  k.gamma = p->gamma;
  k.gm1 = p->gamma - 1.0;
  k.g1 = (p->gamma + 1.0) / (2.0 * p->gamma);
  k.cfl = p->cfl;
  k.limiter = p->limiter;
  k.use_flattening = p->use_flattening;
  k.cvisc = p->cvisc;
  k.riemann_maxiter = p->riemann_maxiter;
  k.riemann_tol = p->riemann_tol;
  k.small_dens = p->small_dens;
  k.small_pres = p->small_pres;
  k.grav = p->grav;
  k.grav_f = (float)p->grav;
  k.use_grav = p->grav != 0.0;
  k.riemann_solver = p->riemann_solver;
  k.reconstruction = p->reconstruction;
  k.bc_general = p->bc_xlo >= HYDRO_BC_REFLECT || p->bc_xhi >= HYDRO_BC_REFLECT || p->bc_ylo >= HYDRO_BC_REFLECT ||
                 p->bc_yhi >= HYDRO_BC_REFLECT;
  k.gamma_f = (float)k.gamma;
  k.gm1_f = (float)k.gm1;
  k.igm1_f = (float)(1.0 / k.gm1);
  k.idx_f = (float)(1.0 / k.dx);
  k.idy_f = (float)(1.0 / k.dy);
  k.g1_f = (float)k.g1;
  k.small_dens_f = (float)k.small_dens;
  k.small_pres_f = (float)k.small_pres;
  k.tol_f = (float)k.riemann_tol;
  k.cvisc_f = (float)k.cvisc;
  k.dx_f = (float)k.dx;
  k.dy_f = (float)k.dy;
  k.rec_f = (float)p->recover_ke_frac;
}

}  // namespace hydro

extern "C" {

hydro_status hydro_default_params(hydro_params* p, int nx, int ny, int precision) {
  if (!p) return HYDRO_EINVAL;
  memset(p, 0, sizeof *p);
  p->nx = nx;
  p->ny = ny;
  p->ng = 4;
  p->xmin = 0.0;
  p->xmax = 1.0;
  p->ymin = 0.0;
  p->ymax = 1.0;
  p->gamma = 1.4;
  p->cfl = 0.8;
  p->bc_xlo = p->bc_xhi = p->bc_ylo = p->bc_yhi = HYDRO_BC_OUTFLOW;
  p->limiter = 2;
  p->use_flattening = 1;
  p->cvisc = 0.1;
  p->riemann_maxiter = precision == HYDRO_FP32 ? 16 : 32;
  p->riemann_tol = precision == HYDRO_FP32 ? 1e-6 : 1e-14;
  p->small_dens = 1e-10;
  p->small_pres = 1e-20;
  p->precision = precision;
  p->use_learned_guess = 0;
  p->grav = 0.0;
  p->split = 0;
  p->riemann_solver = HYDRO_RIEMANN_TWO_SHOCK;
  p->reconstruction = HYDRO_RECON_PLM;
  p->recover_ke_frac = 0.999;
  return HYDRO_OK;
}

size_t hydro_params_size(void) { return sizeof(hydro_params); }

size_t hydro_state_pitch(const hydro_params* p) {
  if (!params_valid(p, nullptr, 0)) return 0;
  const size_t row = (size_t)p->nx + 2 * (size_t)p->ng;
  const size_t per = 128 / elem_size(p->precision);  // elements per 128 bytes
  return (row + per - 1) / per * per;
}

size_t hydro_state_bytes(const hydro_params* p) {
  const size_t pitch = hydro_state_pitch(p);
  if (!pitch) return 0;
  return 4 * pitch * ((size_t)p->ny + 2 * (size_t)p->ng) * elem_size(p->precision);
}

hydro_status hydro_init(const hydro_params* p, void* d_state, void* d_state_alt, void* cuda_stream, hydro_ctx** out) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  char why[256];
  if (!params_valid(p, why, sizeof why)) return HYDRO_EINVAL;
  if (!d_state || !d_state_alt || d_state == d_state_alt) return HYDRO_EINVAL;
  if (((uintptr_t)d_state & 255) || ((uintptr_t)d_state_alt & 255)) return HYDRO_EINVAL;
  hydro_ctx* c = new (std::nothrow) hydro_ctx();
  if (!c) return HYDRO_ENOMEM;
  c->p = *p;
  c->state[0] = d_state;
  c->state[1] = d_state_alt;
  c->cur = 0;
  c->stream = (cudaStream_t)cuda_stream;
  c->err[0] = 0;
  hydro::fill_kparams(p, &c->kp);
  c->tma_ok = make_tensor_maps(c);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return HYDRO_ECUDA;
  }
  e = cudaMalloc((void**)&c->scr, sizeof(DevScratch));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->partials, sizeof(double) * 4 * hydro::totals_max_blocks());
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->host_scr, sizeof(DevScratch));
  if (e == cudaSuccess) e = hydro::init_scratch(c->scr, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    hydro_destroy(c);
    return e == cudaErrorMemoryAllocation ? HYDRO_ENOMEM : HYDRO_ECUDA;
  }
  *out = c;
  return HYDRO_OK;
}

void hydro_destroy(hydro_ctx* c) {
  if (!c) return;
  if (c->host_pipe) {
    for (int b = 0; b < hydro_ctx::HOST_BANDS; ++b) {
      cudaStreamDestroy(c->band_stream[b]);
      cudaEventDestroy(c->ev_band[b]);
      cudaEventDestroy(c->ev_up[b]);
    }
    for (int k = 0; k < hydro_ctx::HOST_GRAPHS; ++k)
      if (c->hgraph[k].exec) cudaGraphExecDestroy(c->hgraph[k].exec);
    cudaStreamDestroy(c->d2h_stream);
    cudaStreamDestroy(c->h2d_stream);
    cudaEventDestroy(c->ev_ready);
    cudaEventDestroy(c->ev_start);
    cudaEventDestroy(c->ev_done);
    cudaFree(c->stage[0]);
    cudaFree(c->stage[1]);
  }
  if (c->scr) cudaFree(c->scr);
  if (c->partials) cudaFree(c->partials);
  if (c->host_scr) cudaFreeHost(c->host_scr);
  delete c;
}

void* hydro_state(const hydro_ctx* c) { return c ? c->state[c->cur] : nullptr; }

hydro_status hydro_fill_ghost(hydro_ctx* c) {
  if (!c) return HYDRO_EINVAL;
  cudaError_t e = hydro::fill_ghost(c->p.precision, c->kp, c->state[c->cur], c->stream);
  return e == cudaSuccess ? HYDRO_OK : cuda_fail(c, e, "fill_ghost");
}

static hydro_status read_scratch(hydro_ctx* c) {
  cudaError_t e = cudaMemcpyAsync(c->host_scr, c->scr, sizeof(DevScratch), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? HYDRO_OK : cuda_fail(c, e, "read scratch");
}

static hydro_status status_from_flags(unsigned int f) {
  if (f & hydro::STATUS_NONFINITE) return HYDRO_ENONFINITE;
  if (f & hydro::STATUS_NEGATIVE) return HYDRO_ENEGATIVE;
  if (f & hydro::STATUS_NONCONV) return HYDRO_ENONCONV;
  if (f & hydro::STATUS_TIMEOUT) return HYDRO_ETIMEOUT;
  return HYDRO_OK;
}

hydro_status hydro_cfl_dt(hydro_ctx* c, double* dt_out) {
  if (!c || !dt_out) return HYDRO_EINVAL;
  cudaError_t e = hydro::cfl_dt(c->p.precision, c->kp, c->state[c->cur], c->scr, 0.0, 0, nullptr, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cfl_dt");
  hydro_status s = read_scratch(c);
  if (s != HYDRO_OK) return s;
  const unsigned int f = c->host_scr->status & (hydro::STATUS_NONFINITE | hydro::STATUS_NEGATIVE);
  if (f) {
    set_err(c, "cfl_dt: the state holds %s cells", (f & hydro::STATUS_NONFINITE) ? "non-finite" : "non-positive");
    return status_from_flags(f);
  }
  *dt_out = c->host_scr->dt;
  return HYDRO_OK;
}

// one CTU step on the context's stream with the face-solve variant its settings select
static cudaError_t launch_step(hydro_ctx* c, const hydro::StepScalars& sc_host, const hydro::StepScalars* sc_dev) {
  int mode = hydro::FACE_PLAIN;
  if (c->p.use_learned_guess == 1) {
    mode = hydro::FACE_LEARNED;
    c->hook.mlp = (const hydro::MlpBlob*)hydro_mlp_device_blob(c->mlp);
  } else if (c->harvest) {
    mode = hydro::FACE_HARVEST;
    c->hook.hseed = hydro::host_hash32(c->step_calls * 0x9E3779B1u + 0x6A09E667u);
  }
  ++c->step_calls;
  return hydro::ctu_step(c->p.precision, c->kp, c->state[c->cur], c->state[1 - c->cur], sc_host, sc_dev, c->scr,
                         c->stream, mode, &c->hook, c->tma_ok ? &c->tmap[c->cur] : nullptr);
}

// one dimensionally split step (paper §3.1) on the current state: sweep along the first direction into the
// other buffer, then along the second direction back into the current buffer (which then holds the new
// state).  The sweeps read cells outside the domain through the boundary map, so no ghost fill is needed.
// sc_next != NULL: the second sweep also reduces the next step's dt (the fused step).
static cudaError_t launch_split_step(hydro_ctx* c, const hydro::StepScalars& sc_host, const hydro::StepScalars* sc_dev,
                                     hydro::StepScalars* sc_next = nullptr, double tmax = 0.0) {
  const int first = (int)(c->split_steps & 1ull);
  const int prec = c->p.precision;
  void* a = c->state[c->cur];
  void* b = c->state[1 - c->cur];
  cudaError_t e = hydro::split_sweep(prec, c->kp, a, b, first, sc_host, sc_dev, c->scr, 0, nullptr, 0.0, c->stream);
  if (e == cudaSuccess)
    e = hydro::split_sweep(prec, c->kp, b, a, 1 - first, sc_host, sc_dev, c->scr, 1, sc_next, tmax, c->stream);
  if (e == cudaSuccess) ++c->split_steps;
  return e;
}

static void drop_host_graphs(hydro_ctx* c);

static hydro_status check_model(hydro_ctx* c) {
  if (c->p.use_learned_guess == 1 && !c->mlp) {
    set_err(c, "use_learned_guess = 1 needs a model (hydro_set_riemann_model)");
    return HYDRO_EINVAL;
  }
  return HYDRO_OK;
}

// The network the fused step starts its Riemann iterations from (NULL: the acoustic start).
static const hydro::MlpBlob* ctx_model(const hydro_ctx* c) {
  return c->p.use_learned_guess == 1 && c->mlp ? (const hydro::MlpBlob*)hydro_mlp_device_blob(c->mlp) : nullptr;
}

hydro_status hydro_step(hydro_ctx* c, double dt) {
  if (!c || !(dt > 0.0) || !(dt < 1e300)) return HYDRO_EINVAL;
  if (check_model(c) != HYDRO_OK) return HYDRO_EINVAL;
  const hydro::StepScalars sc = hydro::make_step_scalars(dt, c->kp.dx, c->kp.dy, c->kp.grav);
  c->fused_valid = 0;
  if (c->p.split) {
    cudaError_t e = launch_split_step(c, sc, nullptr);
    return e == cudaSuccess ? HYDRO_OK : cuda_fail(c, e, "split_step");
  }
  cudaError_t e = launch_step(c, sc, nullptr);
  if (e != cudaSuccess) return cuda_fail(c, e, "ctu_step");
  c->cur = 1 - c->cur;
  return HYDRO_OK;
}

hydro_status hydro_step_fused(hydro_ctx* c, double tmax) {
  if (!c) return HYDRO_EINVAL;
  if (c->p.split) {
    // two sweeps, the second folding in the next step's dt; the new state is in the current buffer
    cudaError_t e = cudaSuccess;
    if (!c->fused_valid)
      e = hydro::cfl_dt(c->p.precision, c->kp, c->state[c->cur], c->scr, tmax, 0, &c->scr->scf[c->fused_parity],
                        c->stream);
    if (e == cudaSuccess)
      e = launch_split_step(c, hydro::StepScalars{}, &c->scr->scf[c->fused_parity],
                            &c->scr->scf[1 - c->fused_parity], tmax);
    if (e != cudaSuccess) return cuda_fail(c, e, "split_step_fused");
    ++c->step_calls;
    c->fused_parity = 1 - c->fused_parity;
    c->fused_valid = 1;
    return HYDRO_OK;
  }
  if (check_model(c) != HYDRO_OK) return HYDRO_EINVAL;
  if (c->harvest) {  // the harvest's face variant uses the separate passes
    cudaError_t e = hydro::fill_ghost(c->p.precision, c->kp, c->state[c->cur], c->stream);
    if (e == cudaSuccess) e = hydro::cfl_dt(c->p.precision, c->kp, c->state[c->cur], c->scr, tmax, 1, nullptr, c->stream);
    c->fused_valid = 0;
    if (e == cudaSuccess) e = launch_step(c, hydro::StepScalars{}, &c->scr->sc);
    if (e != cudaSuccess) return cuda_fail(c, e, "advance");
    c->cur = 1 - c->cur;
    return HYDRO_OK;
  }
  cudaError_t e = cudaSuccess;
  if (!c->fused_valid)  // factors of this step from the current state, time unchanged
    e = hydro::cfl_dt(c->p.precision, c->kp, c->state[c->cur], c->scr, tmax, 0, &c->scr->scf[c->fused_parity],
                      c->stream);
  if (e == cudaSuccess)
    e = hydro::ctu_step_fused(c->p.precision, c->kp, c->state[c->cur], c->state[1 - c->cur],
                              &c->scr->scf[c->fused_parity], &c->scr->scf[1 - c->fused_parity], c->scr, tmax,
                              c->tma_ok ? &c->tmap[c->cur] : nullptr, c->stream, make_int2(0, 0), ctx_model(c));
  if (e != cudaSuccess) return cuda_fail(c, e, "step_fused");
  ++c->step_calls;
  c->cur = 1 - c->cur;
  c->fused_parity = 1 - c->fused_parity;
  c->fused_valid = 1;
  return HYDRO_OK;
}

hydro_status hydro_set_harvest(hydro_ctx* c, void* d_buf, unsigned long long capacity, double rate,
                               unsigned long long* d_count) {
  if (!c) return HYDRO_EINVAL;
  if (!d_buf) {
    c->harvest = 0;
    return HYDRO_OK;
  }
  if (c->p.precision != HYDRO_FP32 || c->p.split || c->p.riemann_solver != HYDRO_RIEMANN_TWO_SHOCK ||
      c->p.reconstruction != HYDRO_RECON_PLM || !d_count || capacity == 0 || !(rate > 0.0) || !(rate <= 1.0))
    return HYDRO_EINVAL;
  c->hook.hbuf = (float*)d_buf;
  c->hook.hcount = d_count;
  c->hook.hcap = capacity;
  c->hook.hthresh = rate >= 1.0 ? 0xFFFFFFFFu : (unsigned int)(rate * 4294967296.0);
  c->harvest = 1;
  return HYDRO_OK;
}

hydro_status hydro_set_harvest_gate(hydro_ctx* c, double gate_dp, double gate_du) {
  if (!c) return HYDRO_EINVAL;
  if (gate_dp <= 0.0 && gate_du <= 0.0) {
    c->hook.hgate_ratio = 0.f;
    c->hook.hgate_u4 = 0.f;
    return HYDRO_OK;
  }
  if (!(gate_dp > 0.0) || !(gate_du > 0.0) || gate_dp > 40.0 || gate_du > 1e9) return HYDRO_EINVAL;
  c->hook.hgate_ratio = (float)exp(2.0 * gate_dp);
  c->hook.hgate_u4 = (float)(gate_du * gate_du * gate_du * gate_du);
  return HYDRO_OK;
}

hydro_status hydro_set_riemann_model(hydro_ctx* c, const hydro_mlp* m) {
  if (!c) return HYDRO_EINVAL;
  if (m && c->p.precision != HYDRO_FP32) return HYDRO_EINVAL;
  if (m != c->mlp) drop_host_graphs(c);  // captured host steps hold the old weights' address
  c->mlp = m;
  return HYDRO_OK;
}

hydro_status hydro_cfl_dt_async(hydro_ctx* c, double tmax) {
  if (!c) return HYDRO_EINVAL;
  cudaError_t e = hydro::cfl_dt(c->p.precision, c->kp, c->state[c->cur], c->scr, tmax, 1, nullptr, c->stream);
  return e == cudaSuccess ? HYDRO_OK : cuda_fail(c, e, "cfl_dt_async");
}

hydro_status hydro_step_device_dt(hydro_ctx* c) {
  if (!c) return HYDRO_EINVAL;
  if (check_model(c) != HYDRO_OK) return HYDRO_EINVAL;
  c->fused_valid = 0;
  if (c->p.split) {
    cudaError_t e = launch_split_step(c, hydro::StepScalars{}, &c->scr->sc);
    return e == cudaSuccess ? HYDRO_OK : cuda_fail(c, e, "step_device_dt");
  }
  cudaError_t e = launch_step(c, hydro::StepScalars{}, &c->scr->sc);
  if (e != cudaSuccess) return cuda_fail(c, e, "step_device_dt");
  c->cur = 1 - c->cur;
  return HYDRO_OK;
}

hydro_status hydro_advance(hydro_ctx* c, int nsteps, double tmax) {
  if (!c || nsteps < 0) return HYDRO_EINVAL;
  c->fused_valid = 0;  // tmax may differ from the previous call's
  for (int n = 0; n < nsteps; ++n) {
    hydro_status s = hydro_step_fused(c, tmax);
    if (s != HYDRO_OK) return s;
  }
  return HYDRO_OK;
}

hydro_status hydro_get_time(hydro_ctx* c, double* t, long long* nsteps) {
  if (!c) return HYDRO_EINVAL;
  hydro_status s = read_scratch(c);
  if (s != HYDRO_OK) return s;
  if (t) *t = c->host_scr->t;
  if (nsteps) *nsteps = c->host_scr->nsteps;
  return HYDRO_OK;
}

hydro_status hydro_conserved_totals(hydro_ctx* c, double out[4]) {
  if (!c || !out) return HYDRO_EINVAL;
  cudaError_t e = hydro::conserved_totals(c->p.precision, c->kp, c->state[c->cur], c->partials, c->scr, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "conserved_totals");
  hydro_status s = read_scratch(c);
  if (s != HYDRO_OK) return s;
  for (int k = 0; k < 4; ++k) out[k] = c->host_scr->totals[k];
  return HYDRO_OK;
}

hydro_status hydro_sync_status(hydro_ctx* c, unsigned long long stats[3]) {
  if (!c) return HYDRO_EINVAL;
  hydro_status s = read_scratch(c);
  if (s != HYDRO_OK) return s;
  const unsigned int f = c->host_scr->status;
  if (stats)
    for (int k = 0; k < 3; ++k) stats[k] = c->host_scr->stats[k];
  if (f) {
    cudaError_t e = cudaMemsetAsync(&c->scr->status, 0, sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "clear status");
    if (f & hydro::STATUS_TIMEOUT_INFLIGHT)
      set_err(c, "device status flags 0x%x: a tile copy had not landed after two bounded waits; discard the "
                 "state and upload it again", f);
    else if (f & hydro::STATUS_TIMEOUT)
      set_err(c, "device status flags 0x%x: a tile copy timed out; discard the state and upload it again", f);
    else
      set_err(c, "device status flags 0x%x", f);
  }
  return status_from_flags(f);
}

hydro_status hydro_upload(hydro_ctx* c, const void* host) {
  if (!c || !host) return HYDRO_EINVAL;
  const size_t es = elem_size(c->p.precision);
  const size_t w = (size_t)c->kp.NX * es, pitchb = (size_t)c->kp.pitch * es;
  // pinned host memory the device can address is read by a copy kernel (about twice the copy engine's
  // rate for this pitched copy on a Grace system); other host memory goes through the copy engine
  cudaPointerAttributes at;
  cudaError_t e;
  if (cudaPointerGetAttributes(&at, host) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer)
    e = hydro::upload_rows(at.devicePointer, c->state[c->cur], w, pitchb, 4 * c->kp.NY, c->stream);
  else
    e = cudaMemcpy2DAsync(c->state[c->cur], pitchb, host, w, w, (size_t)4 * c->kp.NY, cudaMemcpyHostToDevice,
                          c->stream);
  cudaGetLastError();  // a failed attribute query of unregistered memory leaves no sticky error
  c->fused_valid = 0;
  return e == cudaSuccess ? HYDRO_OK : cuda_fail(c, e, "upload");
}

hydro_status hydro_download(hydro_ctx* c, void* host) {
  if (!c || !host) return HYDRO_EINVAL;
  const size_t es = elem_size(c->p.precision);
  const size_t w = (size_t)c->kp.NX * es, pitchb = (size_t)c->kp.pitch * es;
  cudaError_t e = cudaMemcpy2DAsync(host, w, c->state[c->cur], pitchb, w, (size_t)4 * c->kp.NY,
                                    cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? HYDRO_OK : cuda_fail(c, e, "download");
}

// The staging copies have no row padding.
static hydro::KParams stage_kparams(const hydro_ctx* c) {
  hydro::KParams ks = c->kp;
  ks.pitch = ks.NX;
  return ks;
}

// Band b's stream gets a higher priority than band b + 1's, so that the block scheduler finishes the bands
// in order and the first rows can go back to the host while the later ones compute.
static cudaError_t make_host_pipe(hydro_ctx* c) {
  if (c->host_pipe) return cudaSuccess;
  constexpr int NB = hydro_ctx::HOST_BANDS;
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  // streams: the bands (priorities from `greatest`, numerically lowest, down to `least`), the copies back
  // (least), the copies up (greatest); events: ready, start, done, one per band, one per band's rows up
  cudaStream_t streams[NB + 2] = {};
  cudaEvent_t events[2 * NB + 3] = {};
  void* stage[2] = {};
  for (int b = 0; b < NB + 2 && e == cudaSuccess; ++b) {
    const int prio = b == NB + 1 ? greatest : b == NB ? least : (greatest + b < least ? greatest + b : least);
    e = cudaStreamCreateWithPriority(&streams[b], cudaStreamNonBlocking, prio);
  }
  for (int k = 0; k < 2 * NB + 3 && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&events[k], cudaEventDisableTiming);
  const size_t bytes = 4 * (size_t)c->kp.NX * (size_t)c->kp.NY * elem_size(c->p.precision);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaMalloc(&stage[k], bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(stage[k], 0, bytes, c->stream);  // ghost cells read as 0
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {  // release whatever was created
    for (int b = 0; b < NB + 2; ++b)
      if (streams[b]) cudaStreamDestroy(streams[b]);
    for (int k = 0; k < 2 * NB + 3; ++k)
      if (events[k]) cudaEventDestroy(events[k]);
    for (int k = 0; k < 2; ++k)
      if (stage[k]) cudaFree(stage[k]);
    return e;
  }
  for (int b = 0; b < NB; ++b) {
    c->band_stream[b] = streams[b];
    c->ev_band[b] = events[3 + b];
    c->ev_up[b] = events[3 + NB + b];
  }
  c->ev_done = events[2];
  c->d2h_stream = streams[NB];
  c->h2d_stream = streams[NB + 1];
  c->ev_ready = events[0];
  c->ev_start = events[1];
  c->stage[0] = stage[0];
  c->stage[1] = stage[1];
  c->stage_tma = c->tma_ok && hydro::make_state_tensor_map(&c->stage_map, stage_kparams(c), c->p.precision, stage[0],
                                                           hydro::f32_tile_x(), hydro::f32_tile_y());
  c->host_pipe = 1;
  return cudaSuccess;
}

// Enqueue one host step through the staging copies, all of it forked from and joined back into the upload
// stream (so that it can be captured as one graph from there).  The input's rows go up in one chunk per
// band of tile rows, each chunk one 2-D copy of the band's rows (and their 4-row halo) in the four planes;
// the bands of the fused step run on their streams, and each band's rows go back as soon as it has
// finished; the new state is then copied into the context's other buffer.  When `chained`, this step's
// factors are those the previous host step reduced from the state it wrote, which is host_in, so band b
// starts as soon as its rows have arrived; otherwise the CFL step of the uploaded state is reduced first
// and every band waits for it.
static cudaError_t enqueue_host_step(hydro_ctx* c, const void* host_in, void* host_out, double tmax, int chained) {
  constexpr int NB = hydro_ctx::HOST_BANDS;
  const int prec = c->p.precision;
  const hydro::KParams ks = stage_kparams(c);
  const size_t es = elem_size(prec), w = (size_t)ks.NX * es, plane = w * (size_t)ks.NY;
  const size_t pitchb = (size_t)c->kp.pitch * es;
  const unsigned char* hin = (const unsigned char*)host_in;
  unsigned char* hout = (unsigned char*)host_out;
  unsigned char* s_in = (unsigned char*)c->stage[0];
  unsigned char* s_out = (unsigned char*)c->stage[1];
  hydro::StepScalars* sc_cur = &c->scr->scf[c->fused_parity];
  hydro::StepScalars* sc_next = &c->scr->scf[1 - c->fused_parity];
  cudaStream_t up = c->h2d_stream;
  // bands of tile rows, in sixteenths: 1/8, 1/8, 1/4, 1/4, 1/4 when every band waits for the dt (small
  // first bands start the copies back early); when chained, eight bands of 1/16, 1/8, 1/8, 3/16, 3/16, 1/8,
  // 1/8, 1/16 (a small first band starts the copies back early, a small last one ends the step early after
  // the whole upload; KH 1024^2 FP32: 181 us per step, 186 us with 1/8, 1/4, 1/4, 1/4, 1/8, 185-200 us with
  // five other splits); grids of fewer than 16 tile rows split evenly into at most five bands
  static const int sixteenths_dt[6] = {0, 2, 4, 8, 12, 16};
  static const int sixteenths_chain[NB + 1] = {0, 1, 3, 5, 8, 11, 13, 15, 16};
  const int ty = hydro::fused_tile_rows(prec, c->kp);
  const int tile_h = hydro::fused_tile_height(prec);  // cells per tile row
  const int nb = ty < 16 ? (ty < 5 ? ty : 5) : chained ? NB : 5;
  const int* sixteenths = chained ? sixteenths_chain : sixteenths_dt;
  int yb[NB + 1];
  for (int b = 0; b <= nb; ++b) yb[b] = ty >= 16 ? ty * sixteenths[b] / 16 : b * ty / nb;
  auto rows_up = [&](int r0, int r1) -> cudaError_t {  // padded rows [r0, r1) of the four planes
    return r1 > r0 ? cudaMemcpy2DAsync(s_in + (size_t)r0 * w, plane, hin + (size_t)r0 * w, plane,
                                       (size_t)(r1 - r0) * w, 4, cudaMemcpyHostToDevice, up)
                   : cudaSuccess;
  };
  // the first chunk also carries the rows the first band reads as periodic images of the top edge
  // (interior rows ny - 4 .. ny - 1 and the ghost rows above them); band b needs padded rows up to
  // ng + (its last tile row's end) + 4
  cudaError_t e = cudaSuccess;
  int top = ks.NY - ks.ng - 4;
  int done = 0;  // padded rows [0, done) and [top, NY) are on their way up
  for (int b = 0; b < nb && e == cudaSuccess; ++b) {
    int hi = b == nb - 1 ? ks.NY : ks.ng + yb[b + 1] * tile_h + 4;
    if (hi > ks.NY) hi = ks.NY;
    if (b == 0) {
      if (top <= hi) top = ks.NY;  // the first chunk reaches the top already
      e = rows_up(top, ks.NY);
    }
    if (hi > top) hi = top;
    if (e == cudaSuccess && hi > done) {
      e = rows_up(done, hi);
      done = hi;
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_up[b], up);
  }
  if (!chained) {  // this step's factors from the uploaded state, time unchanged
    if (e == cudaSuccess) e = hydro::cfl_dt(prec, ks, s_in, c->scr, tmax, 0, sc_cur, up);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_ready, up);
  }
  for (int b = 0; b < nb && e == cudaSuccess; ++b) {
    cudaStream_t bs = c->band_stream[b];
    e = cudaStreamWaitEvent(bs, chained ? c->ev_up[b] : c->ev_ready, 0);
    if (e == cudaSuccess)
      e = hydro::ctu_step_fused(prec, ks, s_in, s_out, sc_cur, sc_next, c->scr, tmax,
                                c->stage_tma ? &c->stage_map : nullptr, bs, make_int2(yb[b], yb[b + 1] - yb[b]),
                                ctx_model(c));
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_band[b], bs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->d2h_stream, c->ev_band[b], 0);
    // the band's padded rows in the four planes (the first and last bands also carry the ghost rows below
    // and above)
    const int r0 = b == 0 ? 0 : ks.ng + yb[b] * tile_h;
    const int r1 = b == nb - 1 ? ks.NY : ks.ng + yb[b + 1] * tile_h;
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(hout + (size_t)r0 * w, plane, s_out + (size_t)r0 * w, plane, (size_t)(r1 - r0) * w, 4,
                            cudaMemcpyDeviceToHost, c->d2h_stream);
  }
  // after every band, the new state into the context's other buffer by the row-copy kernel (here from
  // device memory; the copy engine takes several times longer over the padded layout's short rows); the
  // copies back join last
  for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(up, c->ev_band[b], 0);
  if (e == cudaSuccess) e = hydro::upload_rows(s_out, c->state[1 - c->cur], w, pitchb, 4 * ks.NY, up);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_done, c->d2h_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(up, c->ev_done, 0);
  return e;
}

static void drop_host_graphs(hydro_ctx* c) {
  for (int k = 0; k < hydro_ctx::HOST_GRAPHS; ++k)
    if (c->hgraph[k].used) {
      if (c->hgraph[k].exec) cudaGraphExecDestroy(c->hgraph[k].exec);
      c->hgraph[k] = hydro_ctx::HostGraph{};
    }
}

// The graph of this host step: found among the kept ones, else captured from the upload stream and
// instantiated.  nullptr when capture or instantiation fails (pageable host memory, for one, cannot be
// captured; the step then runs uncaptured, and the failure is kept so that the next call does not retry).
static cudaGraphExec_t host_step_graph(hydro_ctx* c, const void* host_in, void* host_out, double tmax, int chained) {
  for (int k = 0; k < hydro_ctx::HOST_GRAPHS; ++k) {
    const hydro_ctx::HostGraph& g = c->hgraph[k];
    if (g.used && g.in == host_in && g.out == host_out && g.cur == c->cur && g.parity == c->fused_parity &&
        g.chained == chained && g.tmax == tmax)
      return g.exec;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(c->h2d_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const cudaError_t e = enqueue_host_step(c, host_in, host_out, tmax, chained);
  const cudaError_t ec = cudaStreamEndCapture(c->h2d_stream, &graph);
  if (e == cudaSuccess && ec == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
    exec = nullptr;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();  // a failed capture leaves no sticky error; the step then runs uncaptured
  hydro_ctx::HostGraph& slot = c->hgraph[c->hgraph_next];
  c->hgraph_next = (c->hgraph_next + 1) % hydro_ctx::HOST_GRAPHS;
  if (slot.exec) cudaGraphExecDestroy(slot.exec);
  slot = hydro_ctx::HostGraph{host_in, host_out, c->cur, c->fused_parity, chained, tmax, exec, 1};
  return exec;
}

// One host step: the graph of its pipeline launched on the context's stream (so it follows the work
// enqueued there before), or the same work enqueued directly, then a wait for the new state in host_out.
static hydro_status step_host(hydro_ctx* c, const void* host_in, void* host_out, double tmax, int chained) {
  cudaError_t e = make_host_pipe(c);
  if (e != cudaSuccess) return cuda_fail(c, e, "step_host streams");
  c->chain_out = nullptr;
  cudaGraphExec_t exec = host_step_graph(c, host_in, host_out, tmax, chained);
  if (exec) {
    e = cudaGraphLaunch(exec, c->stream);
  } else {
    e = cudaEventRecord(c->ev_start, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->h2d_stream, c->ev_start, 0);
    if (e == cudaSuccess) e = enqueue_host_step(c, host_in, host_out, tmax, chained);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_start, c->h2d_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_start, 0);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "step_host");
  ++c->step_calls;
  c->cur = 1 - c->cur;
  c->fused_parity = 1 - c->fused_parity;
  c->fused_valid = 1;
  c->chain_out = host_out;
  c->chain_step = c->step_calls;
  c->chain_tmax = tmax;
  return HYDRO_OK;
}

static hydro_status host_step_entry(hydro_ctx* c, const void* host_in, void* host_out, double tmax, int chain) {
  if (!c || !host_in || !host_out || host_in == host_out) return HYDRO_EINVAL;
  if (check_model(c) != HYDRO_OK) return HYDRO_EINVAL;
  if (c->harvest || c->p.split) {  // no banded fused launch for these
    c->chain_out = nullptr;
    hydro_status st = hydro_upload(c, host_in);
    if (st == HYDRO_OK) st = hydro_step_fused(c, tmax);
    return st == HYDRO_OK ? hydro_download(c, host_out) : st;
  }
  // a chain holds while host_in is the buffer the last host step wrote and nothing has stepped or replaced
  // the state since (each of those clears fused_valid or counts a step)
  const int chained = chain && c->fused_valid && c->chain_out == host_in && c->chain_step == c->step_calls &&
                      c->chain_tmax == tmax;
  return step_host(c, host_in, host_out, tmax, chained);
}

hydro_status hydro_step_host(hydro_ctx* c, const void* host_in, void* host_out, double tmax) {
  return host_step_entry(c, host_in, host_out, tmax, 0);
}

hydro_status hydro_step_host_chained(hydro_ctx* c, const void* host_in, void* host_out, double tmax) {
  return host_step_entry(c, host_in, host_out, tmax, 1);
}

const char* hydro_last_error(const hydro_ctx* c) { return c ? c->err : "no context"; }

const char* hydro_build_info(void) {
  return "hydro sm_103a; kernels: fill_ghost, cfl_dt, ctu_step and ctu_step_fused (fp64 16x16/256 exact rounding, "
         "fp32 32x16/384 with TMA tile loads), batch fill/dt/step, totals, mlp";
}

int hydro_tma_enabled(const hydro_ctx* c) { return c ? c->tma_ok : 0; }

hydro_status hydro_test_drop_tile_copies(hydro_ctx* c, int drop, unsigned int polls) {
  if (!c || (drop != 0 && drop != 1)) return HYDRO_EINVAL;
  c->kp.tma_test_drop = drop;
  c->kp.tma_polls = drop ? (polls ? polls : 1000u) : 0u;
  drop_host_graphs(c);  // they hold the old parameters
  c->fused_valid = 0;
  return HYDRO_OK;
}

}  // extern "C"
