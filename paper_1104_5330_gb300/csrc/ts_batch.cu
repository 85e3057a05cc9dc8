// Batched steps of many independent problems, and the tile-shape autotuner.
//
// A batch holds one grid per problem (uneven sizes, any number of groups).
// Each pass of a stage is ONE persistent launch over the tiles of every
// problem: CTAs (as many as fit on the GPU) take tile numbers from an atomic
// work queue, find the owning problem by binary search over the per-problem
// tile offsets, and run the run-time-size form of the single-problem tile
// functions, so a batched step performs the operations of stepping each
// problem on its own (results agree to rounding). One step (a counter reset and 12 or 13 persistent launches) is
// captured once into a CUDA graph and replayed for every step.
//
// The autotuner times the candidate tile shapes of the three forward passes of
// a grid with CUDA events and keeps the fastest; results are cached per
// (precision, N_r, N_theta, N_phi, N_Theta, N_Phi) in memory and, when the
// environment variable TS_AUTOTUNE_CACHE names a file, on disk.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "ts_launch.cuh"

namespace ts {

template <typename T, typename C>
struct BatchItem {
  Problem p;                // sizes, coefficient fields, inflow data, tile shapes (resolved)
  Tables<C> t;
  const double* Dr64;
  T *F, *U, *K, *Acc;
  double dt;
  int split, tau;
  long long off[4];         // first queue tile of this problem: angular, plane, radial, collision
};

template <typename T, typename C, int PASS>
__global__ void __launch_bounds__(kThreads)
k_batch_pass(const BatchItem<T, C>* __restrict__ items, int nitems, long long total,
             unsigned long long* counter, int stage, int rmode) {
  __shared__ long long s_tile;
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long tile = (long long)atomicAdd(counter, 1ull);
      int lo = 0;
      if (tile < total) {
        int hi = nitems - 1;  // largest item with off <= tile (items have nonzero tiles there)
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (items[mid].off[PASS] <= tile) lo = mid;
          else hi = mid - 1;
        }
      }
      s_tile = tile;
      s_item = lo;
    }
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= total) return;
    const BatchItem<T, C>& it = items[s_item];
    const long long lt = tile - it.off[PASS];
    const T* in = stage == 0 ? it.F : it.U;
    if (PASS == 0)
      angular_tile_any<T, C>(it.p, it.t, in, it.K, (C)-1, !it.split, it.p.tp.nb, lt);
    else if (PASS == 1)
      plane_tile_any<T, C>(it.p, it.t, in, it.K, (C)-1, it.p.tp.c, lt);
    else if (PASS == 2)
      radial_tile_any<T, C>(it.p, it.t, it.Dr64, in, it.K, (C)-1, it.tau, rmode, it.F,
                        it.Acc, it.U, nullptr, (C)it.dt, it.p.tp.W, lt);
    else
      implicit_collision_tile<T, C>(it.p, it.t, it.F, it.dt, kThreads / 32, lt);
    __syncthreads();  // s_tile and the shared tiles are reused by the next iteration
  }
}

// ------------------------------------------------------------ tile shapes
inline long long tiles_angular(const Dims& d, int nb) { return (d.nblk + nb - 1) / nb; }
inline long long tiles_plane(const Dims& d, int c) {
  return (long long)d.G * d.Nr * d.NT * (d.NP / 2 / c);
}
inline long long tiles_radial(const Dims& d, int W) {
  const int S = d.NT * d.NP;
  return (long long)d.G * d.Nt * d.Np * ((S + W - 1) / W);
}
inline long long tiles_collision(const Dims& d) { return (d.nblk + kThreads / 32 - 1) / (kThreads / 32); }

// Resolve 0 (heuristic) entries of the forward tile shapes.
template <typename T, typename C>
TileParams resolve(const Dims& d, TileParams tp) {
  if (tp.nb <= 0) tp.nb = angular_nb<T, C>(d, 1, tp.rb & 1);
  if (tp.c <= 0) tp.c = plane_c<T, C>(d, 1, tp.rb & 2);
  if (tp.W <= 0) tp.W = radial_W<T, C>(d, 2, tp.rb & 4);
  return tp;
}

// ------------------------------------------------------------- autotuner
std::mutex g_tune_mu;
std::map<std::string, TileParams> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_key(const ts_grid* g) {
  std::ostringstream k;
  k << (g->es == 8 ? "f64" : "f32") << ":" << g->d.Nr << "x" << g->d.Nt << "x" << g->d.Np << "x"
    << g->d.NT << "x" << g->d.NP << ":rb" << g->tp.rb << ":r64" << (g->desc.precision == TS_FP32_R64);
  return k.str();
}

void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("TS_AUTOTUNE_CACHE");
  if (!path) return;
  std::ifstream f(path);
  std::string key;
  TileParams tp;
  while (f >> key >> tp.nb >> tp.c >> tp.W) g_tune_cache[key] = tp;
}

void tune_store_locked(const std::string& key, const TileParams& tp) {
  g_tune_cache[key] = tp;
  const char* path = std::getenv("TS_AUTOTUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << tp.nb << " " << tp.c << " " << tp.W << "\n";
}

template <typename T, typename C>
cudaError_t tune_grid(ts_grid* g, const Tables<C>& t, cudaStream_t st, TileParams* out) {
  Problem p = problem_of(g);
  const Dims& d = p.d;
  T* U = static_cast<T*>(g->U);
  T* K = static_cast<T*>(g->K);
  cudaError_t e = cudaMemsetAsync(U, 0, (size_t)d.total * sizeof(T), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(K, 0, (size_t)d.total * sizeof(T), st);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto timeit = [&](int pass, const TileParams& tp, float* ms) -> cudaError_t {
    p.tp = tp;
    cudaError_t r = cudaSuccess;
    for (int rep = 0; rep < 4 && r == cudaSuccess; ++rep) {
      if (rep == 1) r = cudaEventRecord(a, st);
      if (r != cudaSuccess) break;
      if (pass == 0) r = Launch<T, C>::angular(p, t, U, K, (C)-1, true, st);
      else if (pass == 1) r = Launch<T, C>::plane(p, t, U, K, (C)-1, st);
      else r = Launch<T, C>::radial(p, t, g->t64.Dr, U, K, (C)-1, false, RAD_RHS, nullptr,
                                    nullptr, nullptr, K, 0.0, st);
    }
    if (r == cudaSuccess) r = cudaEventRecord(b, st);
    if (r == cudaSuccess) r = cudaEventSynchronize(b);
    if (r == cudaSuccess) r = cudaEventElapsedTime(ms, a, b);
    return r;
  };
  TileParams base{};
  base.rb = g->tp.rb;
  TileParams best = resolve<T, C>(d, base);
  const bool rbA = best.rb & 1, rbP = best.rb & 2, rbR = best.rb & 4;
  float tbest;
  // angular: nb
  if (e == cudaSuccess) e = timeit(0, best, &tbest);
  for (int nb = 1; nb <= 64 && e == cudaSuccess; nb *= 2) {
    const size_t sm = rbA ? smem_angular_pp<C>(d, nb) : smem_angular<C>(d, nb, false);
    if (nb * d.NT * d.NP > 16384 || sm > kSmemMax || nb == best.nb) continue;
    TileParams c = best;
    c.nb = nb;
    float ms;
    e = timeit(0, c, &ms);
    if (e == cudaSuccess && ms < tbest) { tbest = ms; best.nb = nb; }
  }
  // plane: c (divisors of NP/2; multiples of 4 for the register-blocked form)
  if (e == cudaSuccess) e = timeit(1, best, &tbest);
  for (int c = 1; c <= d.NP / 2 && e == cudaSuccess; ++c) {
    const size_t sm = rbP ? smem_plane_pp<C>(d, c) : smem_plane<C>(d, c, false);
    if ((d.NP / 2) % c || (rbP && c % 4) || sm > kSmemMax || c == best.c) continue;
    TileParams cand = best;
    cand.c = c;
    float ms;
    e = timeit(1, cand, &ms);
    if (e == cudaSuccess && ms < tbest) { tbest = ms; best.c = c; }
  }
  // radial: W
  if (e == cudaSuccess) e = timeit(2, best, &tbest);
  for (int W = 16; W <= 512 && e == cudaSuccess; W *= 2) {
    const size_t sm = smem_radial<C>(d, W, rbR);
    if (W > d.NT * d.NP || sm > kSmemMax || W == best.W) continue;
    TileParams cand = best;
    cand.W = W;
    float ms;
    e = timeit(2, cand, &ms);
    if (e == cudaSuccess && ms < tbest) { tbest = ms; best.W = W; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *out = best;
  return e;
}

// --------------------------------------------------------------- batches
template <typename T, typename C>
cudaError_t set_batch_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = allow_smem(k_batch_pass<T, C, 0>);
  if (e == cudaSuccess) e = allow_smem(k_batch_pass<T, C, 1>);
  if (e == cudaSuccess) e = allow_smem(k_batch_pass<T, C, 2>);
  if (e == cudaSuccess) e = allow_smem(k_batch_pass<T, C, 3>);
  done = e == cudaSuccess;
  return e;
}

}  // namespace ts

// Problems with at least this many points fill the GPU on their own: the batch
// steps them with their grid's single-problem passes (the compiled line-length
// forms where the sizes have them), recorded into the batch's graph; the
// smaller ones share the persistent work-queue launches.
constexpr long long kBatchOwnPassesPoints = 1LL << 22;

struct ts_batch {
  int n = 0;
  size_t es = 8;
  std::vector<ts_grid*> grids;
  std::vector<int> queued;   // problems stepped by the work-queue launches (the rest: own passes)
  std::vector<char> own;     // own[q]: problem q is stepped by its grid's passes
  void* items_dev = nullptr;
  void* items_host = nullptr;  // pinned staging copy of the item table
  size_t items_bytes = 0;
  unsigned long long* counters = nullptr;  // 13 queue counters per step
  long long total[4] = {0, 0, 0, 0};
  size_t smem[4] = {0, 0, 0, 0};
  int ctas[4] = {0, 0, 0, 0};
  bool any_split = false;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t exec = nullptr;
  // TS_AB2 batches: every problem takes one stage derivative per step; the first
  // step after a restart is forward Euler (its own graph, exec_start), and the
  // batch's history is valid once a step has run on the current fields
  bool ab2 = false, hist = false;
  cudaGraphExec_t exec_start = nullptr;
  std::vector<void*> lastF;
  std::vector<double> lastdt;
  std::vector<unsigned> lastgen;   // per-problem ts_grid::gen at the last upload
};

namespace {

using ts::BatchItem;

template <typename T, typename C>
const ts::Tables<C>& tables_of(const ts_grid* g);
template <>
const ts::Tables<double>& tables_of<double, double>(const ts_grid* g) { return g->t64; }
template <>
const ts::Tables<float>& tables_of<float, float>(const ts_grid* g) { return g->t32; }

template <typename T, typename C>
void fill_items(ts_batch* b, void* const* F, const double* dt) {
  BatchItem<T, C>* it = static_cast<BatchItem<T, C>*>(b->items_host);
  long long off[4] = {0, 0, 0, 0};
  for (size_t k = 0; k < b->queued.size(); ++k) {
    const int q = b->queued[k];
    ts_grid* g = b->grids[q];
    BatchItem<T, C>& x = it[k];
    x.p = ts::problem_of(g);
    x.p.tp = ts::resolve<T, C>(g->d, g->tp);
    x.t = tables_of<T, C>(g);
    x.Dr64 = g->t64.Dr;
    x.F = static_cast<T*>(F[q]);
    x.U = static_cast<T*>(g->U);
    x.K = static_cast<T*>(g->K);
    x.Acc = static_cast<T*>(g->Acc);
    x.dt = dt[q];
    x.split = g->desc.scheme == TS_RK4_SPLIT_IMPLICIT;
    x.tau = g->desc.bc == TS_BC_TAU_INFLOW;
    const long long nt[4] = {ts::tiles_angular(g->d, x.p.tp.nb), ts::tiles_plane(g->d, x.p.tp.c),
                             ts::tiles_radial(g->d, x.p.tp.W),
                             x.split ? ts::tiles_collision(g->d) : 0};
    for (int a = 0; a < 4; ++a) {
      x.off[a] = off[a];
      off[a] += nt[a];
    }
  }
  for (int a = 0; a < 4; ++a) b->total[a] = off[a];
}

template <typename T, typename C>
cudaError_t layout_batch(ts_batch* b) {
  cudaError_t ea = ts::set_batch_attrs<T, C>();
  if (ea != cudaSuccess) return ea;
  size_t sm[3] = {0, 0, 0};
  for (int q : b->queued) {
    ts_grid* g = b->grids[q];
    const ts::TileParams tp = ts::resolve<T, C>(g->d, g->tp);
    sm[0] = std::max(sm[0], ts::smem_angular<C>(g->d, tp.nb, tp.rb & 1));
    sm[1] = std::max(sm[1], ts::smem_plane<C>(g->d, tp.c, tp.rb & 2));
    sm[2] = std::max(sm[2], ts::smem_radial<C>(g->d, tp.W, tp.rb & 4));
    if (g->desc.scheme == TS_RK4_SPLIT_IMPLICIT) b->any_split = true;
  }
  b->smem[0] = sm[0];
  b->smem[1] = sm[1];
  b->smem[2] = sm[2];
  b->smem[3] = 0;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const void* kers[4] = {(const void*)ts::k_batch_pass<T, C, 0>, (const void*)ts::k_batch_pass<T, C, 1>,
                         (const void*)ts::k_batch_pass<T, C, 2>, (const void*)ts::k_batch_pass<T, C, 3>};
  for (int a = 0; a < 4 && e == cudaSuccess; ++a) {
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kers[a], ts::kThreads, b->smem[a]);
    b->ctas[a] = std::max(1, occ) * nsm;
  }
  return e;
}

// One step of every problem. RK4 batches: four stages; TS_AB2 batches: one
// stage derivative, forward Euler when `first` (the step after a restart).
template <typename T, typename C>
cudaError_t enqueue_step(ts_batch* b, cudaStream_t st, bool first) {
  const BatchItem<T, C>* items = static_cast<const BatchItem<T, C>*>(b->items_dev);
  const int ni = (int)b->queued.size();
  const int nstage = b->ab2 ? 1 : 4;
  cudaError_t e = cudaSuccess;
  if (ni > 0) {
    e = cudaMemsetAsync(b->counters, 0, 13 * sizeof(unsigned long long), st);
    for (int s = 0; s < nstage && e == cudaSuccess; ++s) {
      const int rm = b->ab2 ? (first ? ts::RAD_AB2_START : ts::RAD_AB2) : ts::RAD_STAGE0 + s;
      ts::k_batch_pass<T, C, 0><<<b->ctas[0], ts::kThreads, b->smem[0], st>>>(items, ni, b->total[0], b->counters + 3 * s + 0, s, rm);
      ts::k_batch_pass<T, C, 1><<<b->ctas[1], ts::kThreads, b->smem[1], st>>>(items, ni, b->total[1], b->counters + 3 * s + 1, s, rm);
      ts::k_batch_pass<T, C, 2><<<b->ctas[2], ts::kThreads, b->smem[2], st>>>(items, ni, b->total[2], b->counters + 3 * s + 2, s, rm);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess && b->any_split) {
      ts::k_batch_pass<T, C, 3><<<b->ctas[3], ts::kThreads, 0, st>>>(items, ni, b->total[3], b->counters + 12, 0, 0);
      e = cudaGetLastError();
    }
  }
  // the large problems: one step of each by its grid's own passes
  for (int q = 0; q < b->n && e == cudaSuccess; ++q) {
    if (!b->own[q]) continue;
    e = b->ab2 ? ts::step_grid_ab2(b->grids[q], b->lastF[q], b->lastdt[q], first, st)
               : ts::step_grid(b->grids[q], b->lastF[q], b->lastdt[q], 1, st);
  }
  return e;
}

// Record one step into a graph (the batch's stream is idle).
template <typename T, typename C>
cudaError_t record_step(ts_batch* b, bool first, cudaGraphExec_t* exec) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = enqueue_step<T, C>(b, b->st, first);
    e = cudaStreamEndCapture(b->st, &graph);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return e;
}

template <typename T, typename C>
ts_status batch_step(ts_batch* b, void* const* F, const double* dt, int nsteps, cudaStream_t user) {
  bool changed = b->lastF.empty();
  for (int q = 0; q < b->n && !changed; ++q)
    changed = b->lastF[q] != F[q] || b->lastdt[q] != dt[q] || b->lastgen[q] != b->grids[q]->gen;
  cudaError_t e = cudaSuccess;
  if (changed) {
    e = cudaStreamSynchronize(b->st);  // the staging copy may still be read by an earlier upload
    if (e != cudaSuccess) return ts::cuda_status(e, "ts_batch_step");
    fill_items<T, C>(b, F, dt);
    b->lastF.assign(F, F + b->n);
    b->lastdt.assign(dt, dt + b->n);
    b->lastgen.resize(b->n);
    for (int q = 0; q < b->n; ++q) b->lastgen[q] = b->grids[q]->gen;
    // the large problems' launches carry their fields and steps in their
    // arguments: record the graphs again
    if (b->exec && b->queued.size() < (size_t)b->n) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (b->exec_start && b->queued.size() < (size_t)b->n) {
      cudaGraphExecDestroy(b->exec_start);
      b->exec_start = nullptr;
    }
    b->hist = false;   // new fields, steps or coefficients: AB2 restarts
  }
  // a grid stepped or restarted on its own since the last batch step keeps the
  // batch's history only if its Acc still holds the history of this field
  if (b->ab2)
    for (int q = 0; q < b->n; ++q)
      if (!b->grids[q]->hist || b->grids[q]->hist_F != F[q]) b->hist = false;
  e = cudaEventRecord(b->ev_in, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->ev_in, 0);
  if (e == cudaSuccess && changed)
    e = cudaMemcpyAsync(b->items_dev, b->items_host, b->items_bytes, cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess && !b->exec) e = record_step<T, C>(b, false, &b->exec);
  if (e == cudaSuccess && b->ab2 && !b->exec_start)
    e = record_step<T, C>(b, true, &b->exec_start);
  for (int n = 0; n < nsteps && e == cudaSuccess; ++n) {
    const bool start = b->ab2 && !b->hist;
    e = cudaGraphLaunch(start ? b->exec_start : b->exec, b->st);
    if (e == cudaSuccess && b->ab2) b->hist = true;
  }
  if (e != cudaSuccess) b->hist = false;
  // the grids' own AB2 state: their Acc holds K_{n-1} of these fields
  if (e == cudaSuccess && b->ab2)
    for (int q = 0; q < b->n; ++q) ts::set_ab2_history(b->grids[q], F[q]);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, b->ev_out, 0);
  return e == cudaSuccess ? TS_OK : ts::cuda_status(e, "ts_batch_step");
}

}  // namespace

extern "C" {

ts_status ts_autotune(ts_grid* g, void* stream) {
  if (!g) return ts::fail_status(TS_ERR_ARG, "grid is NULL");
  const std::string key = ts::tune_key(g);
  {
    std::lock_guard<std::mutex> lock(ts::g_tune_mu);
    ts::tune_load_locked();
    auto it = ts::g_tune_cache.find(key);
    if (it != ts::g_tune_cache.end()) {
      g->tp.nb = it->second.nb;
      g->tp.c = it->second.c;
      g->tp.W = it->second.W;
      return TS_OK;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ts::TileParams tp;
  cudaError_t e = g->es == 8 ? ts::tune_grid<double, double>(g, g->t64, st, &tp)
                             : ts::tune_grid<float, float>(g, g->t32, st, &tp);
  if (e != cudaSuccess) return ts::cuda_status(e, "ts_autotune");
  g->tp.nb = tp.nb;
  g->tp.c = tp.c;
  g->tp.W = tp.W;
  std::lock_guard<std::mutex> lock(ts::g_tune_mu);
  ts::tune_store_locked(key, tp);
  return TS_OK;
}

ts_status ts_tile_shape(const ts_grid* g, int* nb, int* c, int* W) {
  if (!g) return ts::fail_status(TS_ERR_ARG, "grid is NULL");
  ts::TileParams tp = g->es == 8 ? ts::resolve<double, double>(g->d, g->tp)
                                 : ts::resolve<float, float>(g->d, g->tp);
  if (nb) *nb = tp.nb;
  if (c) *c = tp.c;
  if (W) *W = tp.W;
  return TS_OK;
}

ts_status ts_batch_destroy(ts_batch* b) {
  if (!b) return TS_OK;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->exec_start) cudaGraphExecDestroy(b->exec_start);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->st) cudaStreamDestroy(b->st);
  if (b->items_dev) cudaFree(b->items_dev);
  if (b->items_host) cudaFreeHost(b->items_host);
  if (b->counters) cudaFree(b->counters);
  for (ts_grid* g : b->grids) ts_destroy_grid(g);
  delete b;
  return TS_OK;
}

ts_status ts_batch_create(const ts_grid_desc* descs, int n, int autotune, ts_batch** out) {
  if (!out) return ts::fail_status(TS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!descs || n < 1) return ts::fail_status(TS_ERR_ARG, "need descs and n >= 1");
  for (int q = 1; q < n; ++q)
    if (descs[q].precision != descs[0].precision)
      return ts::fail_status(TS_ERR_UNSUPPORTED, "all problems of a batch share one precision");
  for (int q = 0; q < n; ++q)
    if (descs[q].radial != TS_RADIAL_CHEBYSHEV || descs[q].form != TS_FORM_ADVECTIVE)
      return ts::fail_status(TS_ERR_UNSUPPORTED,
                             "batches run the advective form on the Chebyshev radial grid");
  for (int q = 0; q < n; ++q)
    if ((descs[q].scheme == TS_AB2) != (descs[0].scheme == TS_AB2))
      return ts::fail_status(TS_ERR_UNSUPPORTED,
                             "a batch runs TS_AB2 on all its problems or on none");
  ts_batch* b = new ts_batch();
  b->n = n;
  for (int q = 0; q < n; ++q) {
    ts_grid* g = nullptr;
    ts_status s = ts_create_grid(&descs[q], &g);
    if (s != TS_OK) {
      ts_batch_destroy(b);
      return s;
    }
    b->grids.push_back(g);
    if (autotune) {
      s = ts_autotune(g, nullptr);
      if (s != TS_OK) {
        ts_batch_destroy(b);
        return s;
      }
    }
  }
  b->es = b->grids[0]->es;
  b->ab2 = descs[0].scheme == TS_AB2;
  b->own.assign(n, 0);
  for (int q = 0; q < n; ++q) {
    if ((long long)b->grids[q]->d.total >= kBatchOwnPassesPoints) b->own[q] = 1;
    else b->queued.push_back(q);
  }
  b->items_bytes = (size_t)n * (b->es == 8 ? sizeof(BatchItem<double, double>) : sizeof(BatchItem<float, float>));
  cudaError_t e = cudaMalloc(&b->items_dev, b->items_bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&b->items_host, b->items_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->counters, 16 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = b->es == 8 ? layout_batch<double, double>(b) : layout_batch<float, float>(b);
  if (e != cudaSuccess) {
    ts_batch_destroy(b);
    cudaGetLastError();
    return ts::cuda_status(e, "ts_batch_create");
  }
  *out = b;
  return TS_OK;
}

ts_status ts_batch_grid(ts_batch* b, int problem, ts_grid** grid) {
  if (!b || !grid || problem < 0 || problem >= b->n)
    return ts::fail_status(TS_ERR_ARG, "bad batch, problem index or output pointer");
  *grid = b->grids[problem];
  return TS_OK;
}

ts_status ts_batch_step(ts_batch* b, void* const* F, const double* dt, int nsteps, void* stream) {
  if (!b || !F || !dt || nsteps < 0) return ts::fail_status(TS_ERR_ARG, "bad batch step arguments");
  for (int q = 0; q < b->n; ++q) {
    if (!F[q]) return ts::fail_status(TS_ERR_ARG, "a field pointer is NULL");
    if (!ts::aligned16(F[q])) return ts::fail_status(TS_ERR_ARG, "a field pointer is not 16-byte aligned");
    if (!std::isfinite(dt[q])) return ts::fail_status(TS_ERR_ARG, "dt must be finite");
    if (!b->grids[q]->coeffs) return ts::fail_status(TS_ERR_STATE, "ts_set_coeffs missing for a problem");
  }
  if (nsteps == 0) return TS_OK;
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  return b->es == 8 ? batch_step<double, double>(b, F, dt, nsteps, user)
                    : batch_step<float, float>(b, F, dt, nsteps, user);
}

}  // extern "C"
