// C-ABI layer of ensembles (include/hydro.h, hydro_batch_*): members with their own grids and time steps
// advanced together.  A run of n steps is one CFL dt pass over every member and then, per step, one
// persistent fused CTU kernel over the tiles of every size class that uses the same tile shape (one launch
// when all classes share it, so small classes do not each end in a partial wave); the step reads ghost cells
// through each member's boundary map and reduces each member's next dt.  hydro_batch_run captures such a
// run into one CUDA graph, launched once.  hydro_batch_autotune
// times the tile shapes of each size class and keeps the fastest.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "../../include/hydro.h"
#include "hydro_batch_internal.h"
#include "hydro_kernels.h"

using hydro::BatchMember;
using hydro::DevScratch;

namespace {

struct SizeClass {
  int nx, ny;
  std::vector<int> members;  // member indices, in input order
  int shape = 0;             // tile shape id (autotuned)
  int4* d_tiles = nullptr;   // (member, bx, by, 0) for the current shape
  int ntiles = 0;
  unsigned int* d_queue = nullptr;
};

// Size classes that share a tile shape, stepped by one persistent launch: their tiles in class order
// (largest classes first) behind one work queue.
struct ShapeGroup {
  int shape = 0;
  int4* d_tiles = nullptr;
  int ntiles = 0;
  unsigned int* d_queue = nullptr;
};

}  // namespace

struct hydro_batch {
  int n = 0;
  int precision = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;  // private stream used only for graph capture
  std::vector<hydro_params> params;
  std::vector<BatchMember> hmem;  // host copy of the member table
  BatchMember* d_mem = nullptr;
  DevScratch* d_scr = nullptr;    // n member scratch blocks
  DevScratch* d_agg = nullptr;    // aggregate counters of the step kernels
  DevScratch* h_scr = nullptr;    // pinned host mirror of one scratch block
  double* d_partials = nullptr;   // totals partials
  int4* d_dt = nullptr;
  int ndt = 0;
  std::vector<SizeClass> classes;
  std::vector<ShapeGroup> groups;
  CUtensorMap* d_tmaps = nullptr; // FP32: two TMA descriptors per member (its buffers, its class's tile box)
  int parity = 0;                 // members' current state is U[parity]
  int learned = 0;                // the members were created with use_learned_guess = 1
  const hydro_mlp* mlp = nullptr; // their network (hydro_batch_set_riemann_model)
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (nsteps, parity) -> executable graph
  char err[512] = {0};
};

static hydro_status fail(hydro_batch* b, cudaError_t e, const char* where) {
  if (b) snprintf(b->err, sizeof b->err, "%s: %s", where, cudaGetErrorString(e));
  return HYDRO_ECUDA;
}

// tiles (member, tile x, tile y, 0) of a class for a tile shape, appended to `tiles`
static void class_tiles(const hydro_batch* b, const SizeClass& c, int shape, std::vector<int4>& tiles) {
  const hydro::TileShape ts = hydro::kTileShapes[shape];
  const int tx = b->precision == HYDRO_FP64 ? 16 : ts.tx, ty = b->precision == HYDRO_FP64 ? 16 : ts.ty;
  for (int m : c.members) {
    const int nbx = (c.nx + tx - 1) / tx, nby = (c.ny + ty - 1) / ty;
    for (int by = 0; by < nby; ++by)
      for (int bx = 0; bx < nbx; ++bx) tiles.push_back(make_int4(m, bx, by, nbx * nby));
  }
}

static void free_groups(hydro_batch* b) {
  for (auto& g : b->groups) {
    if (g.d_tiles) cudaFree(g.d_tiles);
    if (g.d_queue) cudaFree(g.d_queue);
  }
  b->groups.clear();
}

// one group per distinct tile shape of the classes, in the order the shapes first appear
static cudaError_t rebuild_groups(hydro_batch* b) {
  free_groups(b);
  cudaError_t e = cudaSuccess;
  std::vector<int> shapes;
  for (const auto& c : b->classes)
    if (std::find(shapes.begin(), shapes.end(), c.shape) == shapes.end()) shapes.push_back(c.shape);
  for (int sh : shapes) {
    std::vector<int4> tiles;
    for (const auto& c : b->classes)
      if (c.shape == sh) class_tiles(b, c, sh, tiles);
    ShapeGroup g;
    g.shape = sh;
    g.ntiles = (int)tiles.size();
    e = cudaMalloc((void**)&g.d_tiles, sizeof(int4) * std::max<size_t>(tiles.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&g.d_queue, sizeof(unsigned int));
    b->groups.push_back(g);  // owned by the batch from here on, freed with it
    if (e == cudaSuccess)
      e = cudaMemcpy(b->groups.back().d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
  }
  return e;
}

static cudaError_t build_tiles(hydro_batch* b, SizeClass& c, int shape) {
  const hydro::TileShape ts = hydro::kTileShapes[shape];
  const int tx = b->precision == HYDRO_FP64 ? 16 : ts.tx, ty = b->precision == HYDRO_FP64 ? 16 : ts.ty;
  std::vector<int4> tiles;
  class_tiles(b, c, shape, tiles);
  if (c.d_tiles) cudaFree(c.d_tiles);
  c.d_tiles = nullptr;
  cudaError_t e = cudaMalloc((void**)&c.d_tiles, sizeof(int4) * std::max<size_t>(tiles.size(), 1));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(c.d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice);
  c.ntiles = (int)tiles.size();
  c.shape = shape;
  // TMA descriptors of the class's members for this tile box (members without them load cell by cell)
  if (e == cudaSuccess && b->d_tmaps) {
    for (int m : c.members) {
      CUtensorMap maps[2];
      BatchMember& bm = b->hmem[m];
      bm.tma = hydro::make_state_tensor_map(&maps[0], bm.P, b->precision, bm.U[0], tx, ty) &&
               hydro::make_state_tensor_map(&maps[1], bm.P, b->precision, bm.U[1], tx, ty);
      if (bm.tma && e == cudaSuccess) e = cudaMemcpy(b->d_tmaps + 2 * m, maps, sizeof maps, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(b->d_mem + m, &bm, sizeof bm, cudaMemcpyHostToDevice);
    }
  }
  return e;
}

static void drop_graphs(hydro_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

// The network the members start their Riemann iterations from (NULL: the acoustic start).
static const hydro::MlpBlob* batch_model(const hydro_batch* b) {
  return b->learned && b->mlp ? (const hydro::MlpBlob*)hydro_mlp_device_blob(b->mlp) : nullptr;
}

// nsteps steps of every member from parity p0 on stream s (used directly and under stream capture): the dt
// of the current states, then the fused steps, each handing its members' next factors to the following one
static cudaError_t enqueue_run(hydro_batch* b, int nsteps, int p0, cudaStream_t s) {
  cudaError_t e = hydro::batch_dt(b->precision, b->d_mem, b->d_dt, b->ndt, p0, 0, s);
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k)
    for (auto& g : b->groups) {
      if (e != cudaSuccess) break;
      e = hydro::batch_step(b->precision, g.shape, b->d_mem, g.d_tiles, g.ntiles, g.d_queue, (p0 + k) & 1, b->d_agg,
                            s, nullptr, b->d_tmaps, 1, batch_model(b));
    }
  return e;
}

extern "C" {

hydro_status hydro_batch_create(int n, const hydro_params* params, void* const* d_states, void* const* d_states_alt,
                                void* cuda_stream, hydro_batch** out) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  if (n < 1 || !params || !d_states || !d_states_alt) return HYDRO_EINVAL;
  const int prec = params[0].precision;
  for (int i = 0; i < n; ++i) {
    if (hydro_state_pitch(&params[i]) == 0 || params[i].precision != prec || params[i].split ||
        params[i].riemann_solver != HYDRO_RIEMANN_TWO_SHOCK || params[i].reconstruction != HYDRO_RECON_PLM ||
        params[i].use_learned_guess != params[0].use_learned_guess)
      return HYDRO_EINVAL;
    if (!d_states[i] || !d_states_alt[i] || ((uintptr_t)d_states[i] & 255) || ((uintptr_t)d_states_alt[i] & 255))
      return HYDRO_EINVAL;
  }
  hydro_batch* b = new (std::nothrow) hydro_batch();
  if (!b) return HYDRO_ENOMEM;
  b->n = n;
  b->precision = prec;
  b->stream = (cudaStream_t)cuda_stream;
  b->params.assign(params, params + n);
  b->learned = params[0].use_learned_guess;
  cudaError_t e = cudaMalloc((void**)&b->d_scr, sizeof(DevScratch) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_agg, sizeof(DevScratch));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_mem, sizeof(BatchMember) * n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_scr, sizeof(DevScratch));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_partials, sizeof(double) * 4 * hydro::totals_max_blocks());
  for (int i = 0; i < n && e == cudaSuccess; ++i) e = hydro::init_scratch(b->d_scr + i, b->stream);
  if (e == cudaSuccess) e = hydro::init_scratch(b->d_agg, b->stream);
  if (e != cudaSuccess) {
    hydro_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? HYDRO_ENOMEM : HYDRO_ECUDA;
  }
  // member table: the same kernel parameters a single-problem context would use
  b->hmem.resize(n);
  std::vector<int4> dtab;
  std::map<std::pair<int, int>, int> class_of;
  for (int i = 0; i < n; ++i) {
    const hydro_params& p = params[i];
    BatchMember& m = b->hmem[i];
    memset(&m, 0, sizeof m);
    hydro::fill_kparams(&p, &m.P);
    m.U[0] = d_states[i];
    m.U[1] = d_states_alt[i];
    m.scr = b->d_scr + i;
    const int cells = p.nx * p.ny;
    const int nb = (cells + hydro::BATCH_DT_CELLS - 1) / hydro::BATCH_DT_CELLS;
    for (int s = 0; s < nb; ++s) dtab.push_back(make_int4(i, s * hydro::BATCH_DT_CELLS, nb, 0));
    auto key = std::make_pair(p.nx, p.ny);
    if (!class_of.count(key)) {
      class_of[key] = (int)b->classes.size();
      SizeClass c;
      c.nx = p.nx;
      c.ny = p.ny;
      b->classes.push_back(c);
    }
    b->classes[class_of[key]].members.push_back(i);
  }
  // largest classes first, so their tiles start early
  std::sort(b->classes.begin(), b->classes.end(),
            [](const SizeClass& a, const SizeClass& c) { return (long long)a.nx * a.ny > (long long)c.nx * c.ny; });
  b->ndt = (int)dtab.size();
  e = cudaMemcpy(b->d_mem, b->hmem.data(), sizeof(BatchMember) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && prec == HYDRO_FP32) e = cudaMalloc((void**)&b->d_tmaps, sizeof(CUtensorMap) * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_dt, sizeof(int4) * std::max(b->ndt, 1));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_dt, dtab.data(), sizeof(int4) * b->ndt, cudaMemcpyHostToDevice);
  for (auto& c : b->classes) {
    if (e != cudaSuccess) break;
    e = cudaMalloc((void**)&c.d_queue, sizeof(unsigned int));
    if (e == cudaSuccess) e = build_tiles(b, c, 0);
  }
  if (e == cudaSuccess) e = rebuild_groups(b);
  if (e == cudaSuccess) e = hydro::batch_prepare(prec);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    hydro_batch_destroy(b);
    return HYDRO_ECUDA;
  }
  *out = b;
  return HYDRO_OK;
}

void hydro_batch_destroy(hydro_batch* b) {
  if (!b) return;
  drop_graphs(b);
  free_groups(b);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  for (auto& c : b->classes) {
    if (c.d_tiles) cudaFree(c.d_tiles);
    if (c.d_queue) cudaFree(c.d_queue);
  }
  if (b->d_mem) cudaFree(b->d_mem);
  if (b->d_scr) cudaFree(b->d_scr);
  if (b->d_agg) cudaFree(b->d_agg);
  if (b->h_scr) cudaFreeHost(b->h_scr);
  if (b->d_partials) cudaFree(b->d_partials);
  if (b->d_dt) cudaFree(b->d_dt);
  if (b->d_tmaps) cudaFree(b->d_tmaps);
  delete b;
}

hydro_status hydro_batch_set_riemann_model(hydro_batch* b, const hydro_mlp* m) {
  if (!b) return HYDRO_EINVAL;
  if (m && !b->learned) {
    snprintf(b->err, sizeof b->err, "the members were created with use_learned_guess = 0");
    return HYDRO_EINVAL;
  }
  if (m != b->mlp) drop_graphs(b);  // captured runs hold the old weights' address
  b->mlp = m;
  return HYDRO_OK;
}

static hydro_status check_batch_model(hydro_batch* b) {
  if (b->learned && !b->mlp) {
    snprintf(b->err, sizeof b->err, "use_learned_guess = 1 needs a model (hydro_batch_set_riemann_model)");
    return HYDRO_EINVAL;
  }
  return HYDRO_OK;
}

hydro_status hydro_batch_autotune(hydro_batch* b, int reps, int* chosen_shapes) {
  if (!b || reps < 1) return HYDRO_EINVAL;
  if (check_batch_model(b) != HYDRO_OK) return HYDRO_EINVAL;
  // valid step factors for the current state, without advancing time
  cudaError_t e = hydro::batch_dt(b->precision, b->d_mem, b->d_dt, b->ndt, b->parity, 0, b->stream);
  if (e != cudaSuccess) return fail(b, e, "autotune set-up");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int nshape = b->precision == HYDRO_FP64 ? 1 : hydro::kNumTileShapes;
  int ci = 0;
  for (auto& c : b->classes) {
    float best = 1e30f;
    int best_shape = 0;
    for (int sh = 0; sh < nshape && e == cudaSuccess; ++sh) {
      e = build_tiles(b, c, sh);
      // one untimed launch, then reps timed launches (they write the next buffer only)
      for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        if (r == 1) cudaEventRecord(e0, b->stream);
        e = hydro::batch_step(b->precision, sh, b->d_mem, c.d_tiles, c.ntiles, c.d_queue, b->parity, b->d_agg,
                              b->stream, nullptr, b->d_tmaps, 0, batch_model(b));
      }
      cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_shape = sh;
      }
    }
    if (e == cudaSuccess) e = build_tiles(b, c, best_shape);
    if (chosen_shapes) chosen_shapes[ci] = best_shape;
    ++ci;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = rebuild_groups(b);
  // the trial launches counted solves; clear the aggregate counters
  if (e == cudaSuccess) e = hydro::init_scratch(b->d_agg, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  return e == cudaSuccess ? HYDRO_OK : fail(b, e, "autotune");
}

int hydro_batch_num_classes(const hydro_batch* b) { return b ? (int)b->classes.size() : 0; }

hydro_status hydro_batch_class_info(const hydro_batch* b, int k, int* nx, int* ny, int* members, int* tile_x,
                                    int* tile_y, int* threads) {
  if (!b || k < 0 || k >= (int)b->classes.size()) return HYDRO_EINVAL;
  const SizeClass& c = b->classes[k];
  const hydro::TileShape ts = b->precision == HYDRO_FP64 ? hydro::TileShape{16, 16, 256} : hydro::kTileShapes[c.shape];
  if (nx) *nx = c.nx;
  if (ny) *ny = c.ny;
  if (members) *members = (int)c.members.size();
  if (tile_x) *tile_x = ts.tx;
  if (tile_y) *tile_y = ts.ty;
  if (threads) *threads = ts.threads;
  return HYDRO_OK;
}

hydro_status hydro_batch_run(hydro_batch* b, int nsteps, int use_graph) {
  if (!b || nsteps < 0) return HYDRO_EINVAL;
  if (check_batch_model(b) != HYDRO_OK) return HYDRO_EINVAL;
  if (nsteps == 0) return HYDRO_OK;
  cudaError_t e = cudaSuccess;
  if (!use_graph) {
    e = enqueue_run(b, nsteps, b->parity, b->stream);
  } else {
    auto key = std::make_pair(nsteps, b->parity);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
      // capture on a private stream (the caller's may be the legacy default stream, which cannot be
      // captured); capturing executes nothing, and the graph is then launched on the caller's stream
      if (!b->capture_stream) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return fail(b, e, "capture stream");
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) e = enqueue_run(b, nsteps, b->parity, b->capture_stream);
      cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &g);
      if (e == cudaSuccess) e = e2;
      cudaGraphExec_t ge = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(b, e, "graph capture");
      it = b->graphs.emplace(key, ge).first;
    }
    e = cudaGraphLaunch(it->second, b->stream);
  }
  if (e != cudaSuccess) return fail(b, e, "batch run");
  b->parity = (b->parity + nsteps) & 1;
  return HYDRO_OK;
}

void* hydro_batch_state(const hydro_batch* b, int member) {
  if (!b || member < 0 || member >= b->n) return nullptr;
  return b->hmem[member].U[b->parity];
}

static hydro_status read_member(hydro_batch* b, const DevScratch* src) {
  cudaError_t e = cudaMemcpyAsync(b->h_scr, src, sizeof(DevScratch), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? HYDRO_OK : fail(b, e, "read scratch");
}

hydro_status hydro_batch_get_time(hydro_batch* b, int member, double* t, long long* nsteps) {
  if (!b || member < 0 || member >= b->n) return HYDRO_EINVAL;
  hydro_status s = read_member(b, b->d_scr + member);
  if (s != HYDRO_OK) return s;
  if (t) *t = b->h_scr->t;
  if (nsteps) *nsteps = b->h_scr->nsteps;
  return HYDRO_OK;
}

hydro_status hydro_batch_sync_status(hydro_batch* b, unsigned long long stats[3]) {
  if (!b) return HYDRO_EINVAL;
  hydro_status s = read_member(b, b->d_agg);
  if (s != HYDRO_OK) return s;
  unsigned int f = b->h_scr->status;
  if (stats)
    for (int k = 0; k < 3; ++k) stats[k] = b->h_scr->stats[k];
  for (int i = 0; i < b->n; ++i) {
    s = read_member(b, b->d_scr + i);
    if (s != HYDRO_OK) return s;
    f |= b->h_scr->status;
  }
  if (f) {
    cudaError_t e = cudaMemsetAsync(&b->d_agg->status, 0, sizeof(unsigned int), b->stream);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i)
      e = cudaMemsetAsync(&b->d_scr[i].status, 0, sizeof(unsigned int), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(b, e, "clear status");
    snprintf(b->err, sizeof b->err, "device status flags 0x%x", f);
  }
  if (f & hydro::STATUS_NONFINITE) return HYDRO_ENONFINITE;
  if (f & hydro::STATUS_NEGATIVE) return HYDRO_ENEGATIVE;
  if (f & hydro::STATUS_NONCONV) return HYDRO_ENONCONV;
  return HYDRO_OK;
}

hydro_status hydro_batch_conserved_totals(hydro_batch* b, int member, double out[4]) {
  if (!b || !out || member < 0 || member >= b->n) return HYDRO_EINVAL;
  const BatchMember& m = b->hmem[member];
  cudaError_t e = hydro::conserved_totals(b->precision, m.P, m.U[b->parity], b->d_partials, m.scr, b->stream);
  if (e != cudaSuccess) return fail(b, e, "batch totals");
  hydro_status s = read_member(b, m.scr);
  if (s != HYDRO_OK) return s;
  for (int k = 0; k < 4; ++k) out[k] = b->h_scr->totals[k];
  return HYDRO_OK;
}

const char* hydro_batch_last_error(const hydro_batch* b) { return b ? b->err : "no batch"; }

}  // extern "C"
