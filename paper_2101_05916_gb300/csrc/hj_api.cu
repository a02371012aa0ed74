// hj_api.cu -- C ABI of the HJ safe-set library: grid lifecycle, problem set-up,
// the single-grid solve driver, prolongation, value I/O and queries.
//
// Solve driver (Eq. 2 iterated "until convergence", Sec. II-A):
//   init kernel (W = l, or min(prior, l))
//   -> alpha max-reduction, read back once; dt = cfl / sum a_i / h_i
//   -> repeat check windows of ceil(check_dt / dt) TVD-RK3 steps.  Each step
//      is three stage launches.  The last stage of a window also folds
//      max |W - W_window_start| into a device scalar.  That scalar is the
//      only value read back per window.
// A window is captured once as a CUDA graph and replayed, so the launch cost
// of the many small kernels of a 2-D grid is paid once per graph.
#include <algorithm>
#include <cstdint>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "hj_grid.h"

namespace hja {

static std::mutex g_alloc_mu;
static Allocator g_alloc;

Allocator current_allocator() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_alloc;
}

cudaError_t dev_malloc(const Allocator& a, void** p, size_t bytes) {
  *p = nullptr;
  if (!a.alloc) return cudaMalloc(p, bytes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  *p = a.alloc(bytes, dev, a.user);
  if (!*p) return cudaErrorMemoryAllocation;
  // fields are 256-byte aligned plus guard floats, and tiles load 16 bytes
  if (reinterpret_cast<uintptr_t>(*p) & 255u) {
    a.free(*p, dev, a.user);
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaSuccess;
}

void dev_free(const Allocator& a, void* p) {
  if (!p) return;
  if (!a.free) {
    cudaFree(p);
    return;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  a.free(p, dev, a.user);
}

static thread_local char t_err[1024] = "";

hj_status fail(hj_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err, sizeof(t_err), fmt, ap);
  va_end(ap);
  return s;
}

hjd::DevGrid devgrid(const hj_grid g) {
  hjd::DevGrid d;
  std::memset(&d, 0, sizeof(d));
  d.ndim = g->ndim;
  long long s = 1;
  for (int i = g->ndim - 1; i >= 0; --i) {
    d.n[i] = g->n[i];
    d.stride[i] = (int)s;
    s *= g->n[i];
  }
  d.npts = (int)g->npts;
  d.plane = g->ndim == 4 ? (int)(g->npts / g->n[0]) : (int)g->npts;
  d.nrows = (int)(g->npts / g->n[g->ndim - 1]);
  d.tile_rows = g->tile_rows;
  // multiply-shift reciprocals of the three fastest axis lengths (see fast_div)
  for (int k = 0; k < 3; ++k) {
    int ax = g->ndim - 1 - k;
    hjd::div_consts(ax >= 0 ? (unsigned)g->n[ax] : 2u, d.div_m[k], d.div_s[k]);
  }
  for (int i = 0; i < g->ndim; ++i) {
    d.lo[i] = (float)g->lo[i];
    d.h[i] = (float)g->h[i];
    d.lo_d[i] = g->lo[i];
    d.h_d[i] = g->h[i];
    d.ih_d[i] = 1.0 / g->h[i];
    d.ih2_d[i] = 0.5 / g->h[i];
    d.ih[i] = (float)(1.0 / g->h[i]);
    // WENO epsilon floor: 1e-18 in divided differences, on undivided ones
    // times h^2, times the 3/4 scale of the smoothness indicators
    d.wfloor[i] = (float)(0.75 * 1e-18 * g->h[i] * g->h[i]);
    d.hih[i] = (float)(0.5 / g->h[i]);
    d.haih[i] = (float)(0.5 * (double)g->alpha[i] / g->h[i]);
  }
  d.model = g->model;
  for (int i = 0; i < 8; ++i) d.prm[i] = (float)g->params[i];
  for (int i = 0; i < HJ_MAX_DIM; ++i) {
    d.dlo[i] = (float)g->d_lo[i];
    d.dhi[i] = (float)g->d_hi[i];
  }
  d.con_kind = g->con_kind;
  d.con_mask = 0;
  for (int i = 0; i < g->ndim; ++i) {
    d.ca[i] = (float)g->ca[i];
    d.cb[i] = (float)g->cb[i];
    if (g->con_kind == hjd::C_BOX && !(std::isinf(g->ca[i]) && std::isinf(g->cb[i])))
      d.con_mask |= 1u << i;
  }
  for (int i = 0; i < HJ_MAX_DIM; ++i) d.alpha[i] = g->alpha[i];
  d.tab = g->tab;
  if (g->con_kind == hjd::C_FIELD) d.lfield = g->lfield;
  if (g->dfield_nd > 0) {
    d.dflo = g->dfield;
    d.dfhi = g->dfield + (size_t)g->dfield_nd * (size_t)g->npts;
  }
  return d;
}

static int required_nd(const hj_grid g) { return g->model == HJ_DRIFT ? g->ndim : 1; }

hj_status validate_ready(hj_grid g, int scheme) {
  if (g->model < 0) return fail(HJ_ERR_STATE, "dynamics not set");
  if (g->con_kind < 0) return fail(HJ_ERR_STATE, "constraint not set");
  if (g->nd != required_nd(g))
    return fail(HJ_ERR_STATE, "disturbance bound not set (model needs %d intervals, have %d)",
                required_nd(g), g->nd);
  if (!hjk::stage_supported(g->model, g->ndim, scheme))
    return fail(HJ_ERR_ARG, "scheme %d not available for model %d in %d-D", scheme, g->model,
                g->ndim);
  return HJ_OK;
}

hj_status ensure_alpha(hj_grid g) {
  if (g->alpha_valid) return HJ_OK;
  HJ_CU(cudaMemsetAsync(g->dscal, 0, 4 * sizeof(unsigned), g->stream));
  hjd::DevGrid d = devgrid(g);
  HJ_CU(hjk::launch_alpha(d, g->dscal, g->stream));
  HJ_CU(cudaMemcpyAsync(g->hscal, g->dscal, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost,
                        g->stream));
  HJ_CU(cudaStreamSynchronize(g->stream));
  for (int i = 0; i < g->ndim; ++i) {
    unsigned b = g->hscal[i];
    float f;
    std::memcpy(&f, &b, 4);
    g->alpha[i] = f;
  }
  g->alpha_valid = true;
  return HJ_OK;
}

double cfl_dt(const hj_grid g, double cfl) {
  double s = 0.0;
  for (int i = 0; i < g->ndim; ++i) s += (double)g->alpha[i] / g->h[i];
  return s > 0.0 ? cfl / s : 0.0;
}

static void drop_graph(hj_grid g) {
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  g->gexec = nullptr;
  g->g_per = 0;
}

static void invalidate(hj_grid g) {
  g->alpha_valid = false;
  drop_graph(g);
}

// k TVD-RK3 steps; the last one folds the window residual when check_last.
static cudaError_t enqueue_steps(hj_grid g, const hjd::DevGrid& d, int scheme, int clamp,
                                 float band, int margin, float dt, long long k, bool check_last,
                                 cudaStream_t s, bool allow_jit = true) {
  hjd::StageArgs a1{g->W, g->W, g->A, nullptr, nullptr, dt, 0, clamp, band, margin};
  hjd::StageArgs a2{g->A, g->W, g->B, nullptr, nullptr, dt, 0, clamp, band, margin};
  hjd::StageArgs a3{g->B, g->W, g->W, g->snap, g->dscal + 4, dt, 0, clamp, band, margin};
  const int t = g->threads;
  for (long long i = 0; i < k; ++i) {
    cudaError_t e;
    if ((e = hjk::launch_stage(d, scheme, 1, a1, s, t, allow_jit)) != cudaSuccess) return e;
    if ((e = hjk::launch_stage(d, scheme, 2, a2, s, t, allow_jit)) != cudaSuccess) return e;
    a3.check = (check_last && i == k - 1) ? 1 : 0;
    if ((e = hjk::launch_stage(d, scheme, 3, a3, s, t, allow_jit)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One check window: reset the residual, k steps, copy the residual to pinned host memory.
static cudaError_t enqueue_window(hj_grid g, const hjd::DevGrid& d, int scheme, int clamp,
                                  float band, int margin, float dt, long long k, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(g->dscal + 4, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if ((e = enqueue_steps(g, d, scheme, clamp, band, margin, dt, k, true, s)) != cudaSuccess)
    return e;
  return cudaMemcpyAsync(g->hscal + 4, g->dscal + 4, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
}

static hj_status run_window(hj_grid g, const hjd::DevGrid& d, int scheme, int clamp, float band,
                            int margin, float dt, long long k, bool use_graph) {
  if (use_graph && k <= 4096) {
    // shape-specialised kernels load outside the capture; a graph captured
    // before they were ready is rebuilt once they are
    bool jit = hjk::jit_prepare(d, scheme, g->threads);
    if (!(g->gexec && g->g_per == k && g->g_dt == dt && g->g_scheme == scheme &&
          g->g_clamp == clamp && g->g_band == band && g->g_margin == margin &&
          g->g_threads == g->threads && g->g_tile_rows == g->tile_rows && g->g_jit == jit)) {
      drop_graph(g);
      g->g_jit = jit;
      cudaGraph_t graph = nullptr;
      HJ_CU(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
      unsigned long long before = hjk::g_launches.load();
      cudaError_t e = enqueue_window(g, d, scheme, clamp, band, margin, dt, k, g->cap_stream);
      cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &graph);
      // launches recorded during capture run later, on replay
      hjk::g_launches.store(before);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(HJ_ERR_CUDA, "graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      cudaError_t e3 = cudaGraphInstantiate(&g->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e3 != cudaSuccess) {
        g->gexec = nullptr;
        return fail(HJ_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e3));
      }
      g->g_per = k;
      g->g_dt = dt;
      g->g_scheme = scheme;
      g->g_clamp = clamp;
      g->g_band = band;
      g->g_margin = margin;
      g->g_threads = g->threads;
      g->g_tile_rows = g->tile_rows;
    }
    HJ_CU(cudaGraphLaunch(g->gexec, g->stream));
    hjk::g_launches.fetch_add(3ull * (unsigned long long)k);
  } else {
    HJ_CU(enqueue_window(g, d, scheme, clamp, band, margin, dt, k, g->stream));
  }
  HJ_CU(cudaStreamSynchronize(g->stream));
  return HJ_OK;
}

// Launch shapes tried by the autotuner: the flat mapping at three block
// sizes, and row tiles of the few line counts that fill their warps best.
// The process-wide choices per (model, ndim, scheme, grid shape).
struct Shape {
  int threads;    // flat mapping: threads per block
  int tile_rows;  // > 0: row tiles of this many lines (threads follow from it)
};
static const int kFlatCandidates[3] = {128, 256, 512};
static std::mutex g_tune_mu;
static std::map<std::string, Shape> g_tuned;

// Row-tile line counts worth timing for lines of n nodes: tiles of 128 to
// 1024 threads, ranked by the fraction of their lanes that hold a node.
static std::vector<int> tile_candidates(const hj_grid g) {
  int n = g->n[g->ndim - 1];
  long long lines = g->npts / n;
  std::vector<std::pair<double, int>> scored;
  for (int r = 1; r * n <= hjk::kTileMaxThreads && r <= lines; ++r) {
    int t = (r * n + 31) / 32 * 32;
    if (t < 128) continue;
    scored.push_back({-(double)(r * n) / t - 1e-6 * r, r});
  }
  std::sort(scored.begin(), scored.end());
  std::vector<int> out;
  for (size_t i = 0; i < scored.size() && out.size() < 3; ++i) out.push_back(scored[i].second);
  return out;
}

static bool tile_fits(const hj_grid g, int rows) {
  hjd::DevGrid d = devgrid(g);
  const void* f[3] = {g->W, g->A, g->B};
  return hjk::tile_ok(d, rows, f, 3);
}

static std::string tune_key(const hj_grid g, int scheme) {
  std::string k = std::to_string(g->model) + "/" + std::to_string(scheme);
  for (int i = 0; i < g->ndim; ++i) k += "/" + std::to_string(g->n[i]);
  return k;
}

// Pick the stage kernels' launch shape for this grid: time a few TVD-RK3
// steps of each candidate (flat blocks of 128/256/512 threads, row tiles of
// the best-filling line counts) on the grid's own current field, keep the
// fastest.  Every candidate computes the same values.  W is saved to the
// snapshot field first and restored afterwards, so the grid's value is
// unchanged.  Choices are cached per grid shape for the process.
hj_status autotune(hj_grid g, int scheme, int clamp) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(tune_key(g, scheme));
    if (it != g_tuned.end()) {
      g->threads = it->second.threads;
      g->tile_rows = tile_fits(g, it->second.tile_rows) ? it->second.tile_rows : 0;
      g->tuned_scheme = scheme;
      drop_graph(g);
      return HJ_OK;
    }
  }
  hj_status st = ensure_alpha(g);
  if (st != HJ_OK) return st;
  double dt = cfl_dt(g, 0.5);
  if (!(dt > 0.0)) dt = 1e-3;
  if (!g->has_value) {
    hjd::DevGrid d0 = devgrid(g);
    HJ_CU(hjk::launch_init(d0, g->W, g->snap, 0, g->stream));
  }
  size_t bytes = (size_t)g->npts * sizeof(float);
  HJ_CU(cudaMemcpyAsync(g->snap, g->W, bytes, cudaMemcpyDeviceToDevice, g->stream));
  long long steps = std::max(2ll, std::min(20ll, 400000000ll / std::max(1ll, g->npts)));
  std::vector<Shape> cands;
  for (int c : kFlatCandidates) cands.push_back({c, 0});
  for (int r : tile_candidates(g))
    if (tile_fits(g, r)) cands.push_back({256, r});
  Shape saved{g->threads, g->tile_rows};
  // grids that run shape-specialised kernels are timed with them: start the
  // compiles of every candidate and wait for them (bounded), else time the
  // precompiled kernels
  bool use_jit = false;
  if (hjk::jit_wanted(devgrid(g))) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      bool all = true;
      for (const Shape& c : cands) {
        g->threads = c.threads;
        g->tile_rows = c.tile_rows;
        all = hjk::jit_prepare(devgrid(g), scheme, c.threads) && all;
      }
      if (all) {
        use_jit = true;
        break;
      }
      if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(120)) break;
      std::this_thread::sleep_for(std::chrono::milliseconds(20));
    }
  }
  cudaEvent_t e0, e1;
  HJ_CU(cudaEventCreate(&e0));
  HJ_CU(cudaEventCreate(&e1));
  Shape best = saved;
  float best_ms = 1e30f;
  for (const Shape& c : cands) {
    g->threads = c.threads;
    g->tile_rows = c.tile_rows;
    hjd::DevGrid d = devgrid(g);
    // one untimed step per candidate, then the timed ones
    cudaError_t e = enqueue_steps(g, d, scheme, clamp, 0.f, 0, (float)dt, 1, false, g->stream,
                                  use_jit);
    if (e == cudaSuccess) e = cudaEventRecord(e0, g->stream);
    if (e == cudaSuccess)
      e = enqueue_steps(g, d, scheme, clamp, 0.f, 0, (float)dt, steps, false, g->stream, use_jit);
    if (e == cudaSuccess) e = cudaEventRecord(e1, g->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      g->threads = saved.threads;
      g->tile_rows = saved.tile_rows;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(HJ_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
    HJ_CU(cudaMemcpyAsync(g->W, g->snap, bytes, cudaMemcpyDeviceToDevice, g->stream));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HJ_CU(cudaStreamSynchronize(g->stream));
  g->threads = best.threads;
  g->tile_rows = best.tile_rows;
  g->tuned_scheme = scheme;
  drop_graph(g);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[tune_key(g, scheme)] = best;
  return HJ_OK;
}

static float bits_to_float(unsigned b) {
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

// Localized stepping (hj_solve_opts.local_tol > 0).  Window by window:
//   - the first window steps every slab;
//   - after each window a mask kernel turns the per-slab changes into the
//     slabs that step (changed by more than local_tol, or close enough to
//     one that did for the change to reach them within the next window:
//     the CFL distance of a window along each slab axis plus local_margin)
//     and the rings on which stages 1 and 2 are recomputed (2 and 1
//     stencil radii further), and a list kernel turns them into the row
//     tiles of each stage;
//   - the next window launches exactly those tiles; stage 3 commits only
//     stepping slabs, the others keep W and their snapshot.
// The stop test is the usual one over the nodes that step.  One read-back
// per window carries the residual and the three list lengths.
hj_status solve_local(hj_grid g, const hj_solve_opts& o, double dt, hj_solve_stats& stats,
                      std::chrono::steady_clock::time_point t0) {
  hjd::DevGrid d = devgrid(g);
  // localized launches of the flat mapping use 256-thread blocks
  const int t = 256;
  hjk::LocalLayout L = hjk::local_layout(d, t);
  if (g->local_slabs != L.nslabs || g->local_tiles != L.ntiles) {
    hja::dev_free(g->alloc, g->slab_resid);
    hja::dev_free(g->alloc, g->slab_masks);
    hja::dev_free(g->alloc, g->tile_lists);
    g->slab_resid = nullptr;
    g->slab_masks = nullptr;
    g->tile_lists = nullptr;
    g->local_slabs = g->local_tiles = 0;
    HJ_CU(hja::dev_malloc(g->alloc, (void**)&g->slab_resid, (size_t)L.nslabs * sizeof(unsigned)));
    HJ_CU(hja::dev_malloc(g->alloc, (void**)&g->slab_masks, 3 * (size_t)L.nslabs));
    HJ_CU(hja::dev_malloc(g->alloc, (void**)&g->tile_lists, 3 * (size_t)L.ntiles * sizeof(int)));
    g->local_slabs = L.nslabs;
    g->local_tiles = L.ntiles;
  }
  if (!g->tile_counts) HJ_CU(hja::dev_malloc(g->alloc, (void**)&g->tile_counts, 4 * sizeof(int)));
  if (!g->tile_counts_h) HJ_CU(cudaMallocHost(&g->tile_counts_h, 4 * sizeof(int)));
  cudaStream_t s = g->stream;
  const float fdt = (float)dt;
  long long per = (long long)std::ceil(o.check_dt / dt - 1e-9);
  if (per < 1) per = 1;
  // how far (in slabs) a change can travel along each slab axis in one
  // window: the CFL speed alpha_a dt / h_a cells per step times the steps,
  // plus the caller's margin
  int kax[2] = {0, 0};
  for (int q = 0; q < 2; ++q) {
    int ax = q;  // slab axes: 0 and 1 of a 4-D grid, 0 of a 2-D or 3-D grid
    int slab_axes = g->ndim == 4 ? 2 : (g->ndim >= 2 ? 1 : 0);
    if (ax >= slab_axes) continue;
    double cells = (double)per * (double)g->alpha[ax] * dt / g->h[ax];
    kax[q] = (int)std::ceil(cells) + 1 + o.local_margin;
  }
  int counts[3] = {L.ntiles, L.ntiles, L.ntiles};
  bool first = true;
  double tiles_run = 0.0, tiles_full = 0.0;
  for (;;) {
    long long todo = per;
    if (o.max_steps > 0 && stats.steps + todo > o.max_steps) todo = o.max_steps - stats.steps;
    HJ_CU(cudaMemsetAsync(g->dscal + 4, 0, sizeof(unsigned), s));
    HJ_CU(cudaMemsetAsync(g->slab_resid, 0, (size_t)L.nslabs * sizeof(unsigned), s));
    hjd::StageArgs a1{g->W, g->W, g->A, nullptr, nullptr, fdt, 0, o.clamp, (float)o.band,
                      o.band_margin};
    hjd::StageArgs a2{g->A, g->W, g->B, nullptr, nullptr, fdt, 0, o.clamp, (float)o.band,
                      o.band_margin};
    hjd::StageArgs a3{g->B, g->W, g->W, g->snap, g->dscal + 4, fdt, 0, o.clamp, (float)o.band,
                      o.band_margin};
    if (!first) {
      a1.tiles = g->tile_lists;
      a2.tiles = g->tile_lists + L.ntiles;
      a3.tiles = g->tile_lists + 2 * L.ntiles;
      a1.ntiles = counts[0];
      a2.ntiles = counts[1];
      a3.ntiles = counts[2];
      a3.live = g->slab_masks;
    }
    a3.slab_resid = g->slab_resid;
    for (long long i = 0; i < todo; ++i) {
      HJ_CU(hjk::launch_stage(d, o.scheme, 1, a1, s, t));
      HJ_CU(hjk::launch_stage(d, o.scheme, 2, a2, s, t));
      a3.check = (i == todo - 1) ? 1 : 0;
      HJ_CU(hjk::launch_stage(d, o.scheme, 3, a3, s, t));
    }
    tiles_run += (double)todo * (counts[0] + counts[1] + counts[2]);
    tiles_full += (double)todo * 3.0 * L.ntiles;
    HJ_CU(hjk::launch_local_lists(d, o.scheme, t, g->slab_resid, (float)o.local_tol, kax[0],
                                  kax[1], g->slab_masks, g->tile_lists, g->tile_counts, s));
    HJ_CU(cudaMemcpyAsync(g->hscal + 4, g->dscal + 4, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HJ_CU(cudaMemcpyAsync(g->tile_counts_h, g->tile_counts, 3 * sizeof(int),
                          cudaMemcpyDeviceToHost, s));
    HJ_CU(cudaStreamSynchronize(s));
    for (int q = 0; q < 3; ++q) counts[q] = g->tile_counts_h[q];
    first = false;
    stats.steps += todo;
    stats.windows += 1;
    stats.stepped = tiles_full > 0.0 ? tiles_run / tiles_full : 1.0;
    float r = bits_to_float(g->hscal[4]);
    stats.residual = r;
    if (!std::isfinite(r)) return fail(HJ_ERR_DIVERGED, "non-finite value after %lld steps", stats.steps);
    if ((double)r < o.tol) {
      stats.converged = 1;
      return HJ_OK;
    }
    if (o.max_steps > 0 && stats.steps >= o.max_steps)
      return fail(HJ_ERR_NOT_CONVERGED, "step cap %lld reached (residual %g)", o.max_steps,
                  (double)r);
    double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (o.max_wall_ms > 0.0 && ms > o.max_wall_ms)
      return fail(HJ_ERR_NOT_CONVERGED, "wall-time cap reached (residual %g)", (double)r);
  }
}

}  // namespace hja

using namespace hja;

extern "C" {

const char* hj_last_error(void) { return t_err; }

hj_status hj_set_allocator(hj_alloc_fn alloc, hj_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(HJ_ERR_ARG, "give both allocator functions or neither");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.free = free_fn;
  g_alloc.user = alloc ? user : nullptr;
  return HJ_OK;
}

unsigned long long hj_kernel_launches(void) { return hjk::g_launches.load(); }

long long hj_grid_points(hj_grid g) { return g ? g->npts : 0; }

void hj_default_opts(hj_solve_opts* o) {
  if (!o) return;
  o->scheme = HJ_WENO5;
  o->cfl = 0.5;
  o->dt = 0.0;
  o->tol = 1e-4;
  o->check_dt = 0.1;
  o->max_steps = 1000000;
  o->fixed_steps = 0;
  o->max_wall_ms = 0.0;
  o->clamp = HJ_CLAMP_VI;
  o->use_graph = 1;
  o->band = 0.0;
  o->autotune = 0;
  o->band_margin = 0;
  o->local_tol = 0.0;
  o->local_margin = 1;
}

void hj_grid_destroy(hj_grid g) {
  if (!g) return;
  {
    DeviceGuard dg(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream);
    drop_graph(g);
    for (int i = 0; i < 4; ++i) hja::dev_free(g->alloc, g->raw[i]);
    hja::dev_free(g->alloc, g->tab);
    hja::dev_free(g->alloc, g->dfield);
    hja::dev_free(g->alloc, g->lfield);
    hja::dev_free(g->alloc, g->dscal);
    hja::dev_free(g->alloc, g->qbuf);
    hja::dev_free(g->alloc, g->fdev);
    hja::dev_free(g->alloc, g->slab_resid);
    hja::dev_free(g->alloc, g->slab_masks);
    hja::dev_free(g->alloc, g->tile_lists);
    hja::dev_free(g->alloc, g->tile_counts);
    if (g->tile_counts_h) cudaFreeHost(g->tile_counts_h);
    if (g->fhost) cudaFreeHost(g->fhost);
    if (g->hscal) cudaFreeHost(g->hscal);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  }
  delete g;
}

hj_status hj_grid_create(hj_grid* out, int ndim, const int* n, const double* lo, const double* hi,
                         void* cuda_stream) {
  if (!out) return fail(HJ_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > HJ_MAX_DIM) return fail(HJ_ERR_ARG, "ndim must be 1..%d", HJ_MAX_DIM);
  if (!n || !lo || !hi) return fail(HJ_ERR_ARG, "n/lo/hi is NULL");
  long long npts = 1;
  for (int i = 0; i < ndim; ++i) {
    if (n[i] < 3) return fail(HJ_ERR_ARG, "axis %d has %d nodes (need >= 3)", i, n[i]);
    if (!(hi[i] > lo[i]) || !std::isfinite(lo[i]) || !std::isfinite(hi[i]))
      return fail(HJ_ERR_ARG, "axis %d: need finite lo < hi", i);
    npts *= n[i];
    if (npts >= (1ll << 31)) return fail(HJ_ERR_ARG, "grid has 2^31 or more nodes");
  }
  int dev = 0;
  int count = 0;
  cudaError_t ce = cudaGetDeviceCount(&count);
  if (ce != cudaSuccess || count == 0)
    return fail(HJ_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(ce));
  HJ_CU(cudaGetDevice(&dev));
  hj_grid g = new (std::nothrow) hj_grid_s();
  if (!g) return fail(HJ_ERR_OOM, "host allocation failed");
  g->device = dev;
  g->alloc = current_allocator();
  g->ndim = ndim;
  g->npts = npts;
  for (int i = 0; i < ndim; ++i) {
    g->n[i] = n[i];
    g->lo[i] = lo[i];
    g->hi[i] = hi[i];
    g->h[i] = (hi[i] - lo[i]) / (double)(n[i] - 1);
  }
  g->stream = (cudaStream_t)cuda_stream;
  // each field: guard floats, the nodes, guard floats
  size_t bytes = ((size_t)npts + 2 * kGuard) * sizeof(float);
  bytes = (bytes + 255) & ~(size_t)255;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
    e = hja::dev_malloc(g->alloc, (void**)&g->raw[i], bytes);
    if (e == cudaSuccess) e = cudaMemset(g->raw[i], 0, bytes);
  }
  if (e == cudaSuccess) {
    g->W = g->raw[0] + kGuard;
    g->A = g->raw[1] + kGuard;
    g->B = g->raw[2] + kGuard;
    g->snap = g->raw[3] + kGuard;
  }
  if (e == cudaSuccess) e = hja::dev_malloc(g->alloc, (void**)&g->dscal, 64 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMallocHost(&g->hscal, 64 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    hj_status st = fail(e == cudaErrorMemoryAllocation ? HJ_ERR_OOM : HJ_ERR_CUDA,
                        "grid allocation (%lld nodes): %s", npts, cudaGetErrorString(e));
    cudaGetLastError();
    hj_grid_destroy(g);
    return st;
  }
  *out = g;
  return HJ_OK;
}

hj_status hj_set_stream(hj_grid g, void* cuda_stream) {
  if (!g) return fail(HJ_ERR_ARG, "grid is NULL");
  if (g->stream) cudaStreamSynchronize(g->stream);
  g->stream = (cudaStream_t)cuda_stream;
  return HJ_OK;
}

hj_status hj_set_dynamics(hj_grid g, int model, const double* params, int nparams) {
  if (!g) return fail(HJ_ERR_ARG, "grid is NULL");
  if (nparams < 0 || (nparams > 0 && !params)) return fail(HJ_ERR_ARG, "bad parameter vector");
  if (nparams > 8) return fail(HJ_ERR_ARG, "at most 8 parameters");
  if (model == HJ_QUAD_Z) {
    if (g->ndim != 2) return fail(HJ_ERR_ARG, "HJ_QUAD_Z needs a 2-D grid");
    if (nparams < 4) return fail(HJ_ERR_ARG, "HJ_QUAD_Z needs {kT, g, u_lo, u_hi}");
    if (!(params[2] <= params[3])) return fail(HJ_ERR_ARG, "u_lo > u_hi");
  } else if (model == HJ_QUAD_X4) {
    if (g->ndim != 4) return fail(HJ_ERR_ARG, "HJ_QUAD_X4 needs a 4-D grid");
    if (nparams < 7) return fail(HJ_ERR_ARG, "HJ_QUAD_X4 needs {g, d1, d0, n0, u_lo, u_hi, axis}");
    if (!(params[4] <= params[5])) return fail(HJ_ERR_ARG, "u_lo > u_hi");
    if (params[6] != 0.0 && params[6] != 1.0) return fail(HJ_ERR_ARG, "axis must be 0 or 1");
    double th_max = std::max(std::fabs(g->lo[2]), std::fabs(g->hi[2]));
    if (th_max >= 1.5) return fail(HJ_ERR_ARG, "theta range must stay inside (-1.5, 1.5) rad");
  } else if (model != HJ_DRIFT) {
    return fail(HJ_ERR_ARG, "unknown model %d", model);
  }
  for (int i = 0; i < 8; ++i) g->params[i] = (i < nparams) ? params[i] : 0.0;
  g->model = model;
  DeviceGuard dg(g->device);
  if (model == HJ_QUAD_X4) {
    // g * tan(th_j) for every th node, in double, rounded once to float
    int m = g->n[2];
    float* host = new float[m];
    for (int j = 0; j < m; ++j) host[j] = (float)(params[0] * std::tan(g->lo[2] + j * g->h[2]));
    hja::dev_free(g->alloc, g->tab);
    g->tab = nullptr;
    cudaError_t e = hja::dev_malloc(g->alloc, (void**)&g->tab, m * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g->tab, host, m * sizeof(float), cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    delete[] host;
    if (e != cudaSuccess) return fail(HJ_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
  }
  invalidate(g);
  return HJ_OK;
}

static void drop_lfield(hj_grid g) {
  if (g->lfield) {
    DeviceGuard dg(g->device);
    hja::dev_free(g->alloc, g->lfield);
    g->lfield = nullptr;
  }
}

hj_status hj_set_constraint(hj_grid g, const double* box_lo, const double* box_hi) {
  if (!g) return fail(HJ_ERR_ARG, "grid is NULL");
  if (!box_lo || !box_hi) return fail(HJ_ERR_ARG, "box is NULL");
  int constrained = 0;
  for (int i = 0; i < g->ndim; ++i) {
    if (std::isnan(box_lo[i]) || std::isnan(box_hi[i]) || !(box_lo[i] <= box_hi[i]))
      return fail(HJ_ERR_ARG, "axis %d: need box_lo <= box_hi", i);
    if (!(std::isinf(box_lo[i]) && std::isinf(box_hi[i]))) constrained++;
  }
  if (!constrained) return fail(HJ_ERR_ARG, "no axis is constrained");
  drop_lfield(g);
  g->con_kind = hjd::C_BOX;
  for (int i = 0; i < g->ndim; ++i) {
    g->ca[i] = box_lo[i];
    g->cb[i] = box_hi[i];
  }
  drop_graph(g);
  return HJ_OK;
}

hj_status hj_set_constraint_ball(hj_grid g, const double* centre, double radius) {
  if (!g) return fail(HJ_ERR_ARG, "grid is NULL");
  if (!centre || !(radius > 0.0) || !std::isfinite(radius))
    return fail(HJ_ERR_ARG, "need a centre and a finite radius > 0");
  for (int i = 0; i < g->ndim; ++i)
    if (!std::isfinite(centre[i])) return fail(HJ_ERR_ARG, "centre must be finite");
  drop_lfield(g);
  g->con_kind = hjd::C_BALL_OUT;
  for (int i = 0; i < g->ndim; ++i) {
    if (!std::isfinite(centre[i])) return fail(HJ_ERR_ARG, "centre must be finite");
    g->ca[i] = centre[i];
    g->cb[i] = 0.0;
  }
  g->cb[0] = radius;
  drop_graph(g);
  return HJ_OK;
}

hj_status hj_set_constraint_field(hj_grid g, const float* l, int on_device) {
  if (!g || !l) return fail(HJ_ERR_ARG, "NULL argument");
  DeviceGuard dg(g->device);
  size_t n = (size_t)g->npts;
  if (!g->lfield) HJ_CU(hja::dev_malloc(g->alloc, (void**)&g->lfield, n * sizeof(float)));
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  HJ_CU(cudaMemcpyAsync(g->lfield, l, n * sizeof(float), k, g->stream));
  HJ_CU(cudaMemsetAsync(g->dscal + 5, 0, sizeof(unsigned), g->stream));
  HJ_CU(hjk::launch_field_check(g->lfield, g->lfield, (long long)n, (int*)(g->dscal + 5),
                                g->stream));
  HJ_CU(cudaMemcpyAsync(g->hscal + 5, g->dscal + 5, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        g->stream));
  HJ_CU(cudaStreamSynchronize(g->stream));
  if (g->hscal[5]) {
    // the rejected values are gone with the buffer; no constraint is in force now
    drop_lfield(g);
    g->con_kind = -1;
    drop_graph(g);
    return fail(HJ_ERR_ARG, "constraint field: every value must be finite");
  }
  g->con_kind = hjd::C_FIELD;
  drop_graph(g);
  return HJ_OK;
}

hj_status hj_set_disturbance_bound(hj_grid g, const double* d_lo, const double* d_hi, int nd) {
  if (!g) return fail(HJ_ERR_ARG, "grid is NULL");
  if (nd < 1 || nd > HJ_MAX_DIM || !d_lo || !d_hi) return fail(HJ_ERR_ARG, "bad disturbance box");
  for (int i = 0; i < nd; ++i)
    if (!std::isfinite(d_lo[i]) || !std::isfinite(d_hi[i]) || d_lo[i] > d_hi[i])
      return fail(HJ_ERR_ARG, "input %d: need finite d_lo <= d_hi", i);
  g->nd = nd;
  for (int i = 0; i < HJ_MAX_DIM; ++i) {
    g->d_lo[i] = i < nd ? d_lo[i] : 0.0;
    g->d_hi[i] = i < nd ? d_hi[i] : 0.0;
  }
  g->dfield_nd = 0;  // a uniform box replaces any field
  invalidate(g);
  return HJ_OK;
}

hj_status hj_set_disturbance_field(hj_grid g, const float* d_lo, const float* d_hi, int nd,
                                   int on_device) {
  if (!g || !d_lo || !d_hi) return fail(HJ_ERR_ARG, "NULL argument");
  if (nd < 1 || nd > HJ_MAX_DIM) return fail(HJ_ERR_ARG, "bad number of disturbance inputs");
  DeviceGuard dg(g->device);
  size_t n = (size_t)nd * (size_t)g->npts;
  if (!g->dfield || g->dfield_nd != nd) {
    hja::dev_free(g->alloc, g->dfield);
    g->dfield = nullptr;
    g->dfield_nd = 0;
    HJ_CU(hja::dev_malloc(g->alloc, (void**)&g->dfield, 2 * n * sizeof(float)));
  }
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  HJ_CU(cudaMemcpyAsync(g->dfield, d_lo, n * sizeof(float), k, g->stream));
  HJ_CU(cudaMemcpyAsync(g->dfield + n, d_hi, n * sizeof(float), k, g->stream));
  HJ_CU(cudaMemsetAsync(g->dscal + 5, 0, sizeof(unsigned), g->stream));
  HJ_CU(hjk::launch_field_check(g->dfield, g->dfield + n, (long long)n, (int*)(g->dscal + 5),
                                g->stream));
  HJ_CU(cudaMemcpyAsync(g->hscal + 5, g->dscal + 5, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        g->stream));
  HJ_CU(cudaStreamSynchronize(g->stream));
  if (g->hscal[5]) {
    // the rejected values are gone with the buffer; no bound is in force now
    hja::dev_free(g->alloc, g->dfield);
    g->dfield = nullptr;
    g->dfield_nd = 0;
    g->nd = 0;
    invalidate(g);
    return fail(HJ_ERR_ARG, "disturbance field: need finite d_lo <= d_hi at every node");
  }
  g->dfield_nd = nd;
  g->nd = nd;
  for (int i = 0; i < HJ_MAX_DIM; ++i) g->d_lo[i] = g->d_hi[i] = 0.0;
  invalidate(g);
  return HJ_OK;
}

void hj_set_jit(int enable) { hjk::jit_enable(enable); }

long long hj_jit_kernels(void) { return hjk::jit_compiled(); }

long long hj_jit_pending(void) { return hjk::jit_pending(); }

hj_status hj_autotune(hj_grid g, int scheme, int* threads_out) {
  if (!g) return fail(HJ_ERR_ARG, "grid is NULL");
  hj_status st = validate_ready(g, scheme);
  if (st != HJ_OK) return st;
  DeviceGuard dg(g->device);
  if ((st = autotune(g, scheme, HJ_CLAMP_VI)) != HJ_OK) return st;
  if (threads_out) *threads_out = g->threads;
  return HJ_OK;
}

hj_status hj_set_launch_shape(hj_grid g, int threads, int tile_rows) {
  if (!g) return fail(HJ_ERR_ARG, "grid is NULL");
  if (threads != 128 && threads != 256 && threads != 512)
    return fail(HJ_ERR_ARG, "threads must be 128, 256 or 512");
  if (tile_rows < 0) return fail(HJ_ERR_ARG, "tile_rows must be >= 0");
  if (tile_rows > 0 && !tile_fits(g, tile_rows))
    return fail(HJ_ERR_ARG, "row tiles of %d lines of %d nodes do not fit (at most %d nodes and "
                "%lld lines)", tile_rows, g->n[g->ndim - 1], hjk::kTileMaxThreads,
                g->npts / g->n[g->ndim - 1]);
  g->threads = threads;
  g->tile_rows = tile_rows;
  g->tuned_scheme = 0;
  drop_graph(g);
  return HJ_OK;
}

hj_status hj_get_launch_shape(hj_grid g, int* threads, int* tile_rows) {
  if (!g) return fail(HJ_ERR_ARG, "grid is NULL");
  if (threads) *threads = g->threads;
  if (tile_rows) *tile_rows = g->tile_rows;
  return HJ_OK;
}

hj_status hj_alpha(hj_grid g, double* alpha_out) {
  if (!g || !alpha_out) return fail(HJ_ERR_ARG, "NULL argument");
  if (g->model < 0) return fail(HJ_ERR_STATE, "dynamics not set");
  if (g->nd != (g->model == HJ_DRIFT ? g->ndim : 1)) return fail(HJ_ERR_STATE, "bound not set");
  DeviceGuard dg(g->device);
  hj_status st = ensure_alpha(g);
  if (st != HJ_OK) return st;
  for (int i = 0; i < g->ndim; ++i) alpha_out[i] = g->alpha[i];
  return HJ_OK;
}

hj_status hj_solve(hj_grid g, int mode, const hj_solve_opts* o_in, hj_solve_stats* s) {
  auto t0 = std::chrono::steady_clock::now();
  if (!g) return fail(HJ_ERR_ARG, "grid is NULL");
  hj_solve_opts o;
  hj_default_opts(&o);
  if (o_in) o = *o_in;
  if (mode != HJ_COLD && mode != HJ_WARM) return fail(HJ_ERR_ARG, "mode must be HJ_COLD or HJ_WARM");
  if (!(o.cfl > 0.0) || !(o.tol >= 0.0) || !(o.check_dt > 0.0) || o.dt < 0.0 || !(o.band >= 0.0) ||
      o.band_margin < 0 || !(o.local_tol >= 0.0) || o.local_margin < 0 || o.local_margin > 64)
    return fail(HJ_ERR_ARG, "bad solve options");
  if (o.clamp != HJ_CLAMP_VI && o.clamp != HJ_CLAMP_MONOTONE) return fail(HJ_ERR_ARG, "bad clamp");
  hj_status st = validate_ready(g, o.scheme);
  if (st != HJ_OK) return st;
  if (mode == HJ_WARM && !g->has_value)
    return fail(HJ_ERR_STATE, "warm start asked but the grid holds no prior value");
  DeviceGuard dg(g->device);
  hj_solve_stats stats;
  std::memset(&stats, 0, sizeof(stats));
  stats.stepped = 1.0;

  if ((st = ensure_alpha(g)) != HJ_OK) return st;
  if (o.autotune && g->tuned_scheme != o.scheme && (st = autotune(g, o.scheme, o.clamp)) != HJ_OK)
    return st;
  double dt = o.dt > 0.0 ? o.dt : cfl_dt(g, o.cfl);
  stats.dt = dt;
  hjd::DevGrid d = devgrid(g);
  HJ_CU(hjk::launch_init(d, g->W, g->snap, mode == HJ_WARM ? 1 : 0, g->stream));
  g->has_value = true;
  hj_status rc = HJ_OK;
  float fdt = (float)dt;
  if (dt <= 0.0) {
    // nothing moves: the initial value is the fixed point
    HJ_CU(cudaStreamSynchronize(g->stream));
    stats.converged = 1;
  } else if (o.fixed_steps > 0) {
    HJ_CU(enqueue_steps(g, d, o.scheme, o.clamp, (float)o.band, o.band_margin, fdt, o.fixed_steps,
                        false, g->stream));
    HJ_CU(cudaStreamSynchronize(g->stream));
    stats.steps = o.fixed_steps;
  } else if (o.local_tol > 0.0) {
    rc = solve_local(g, o, dt, stats, t0);
    if (rc != HJ_OK && rc != HJ_ERR_NOT_CONVERGED && rc != HJ_ERR_DIVERGED) return rc;
  } else {
    long long per = (long long)std::ceil(o.check_dt / dt - 1e-9);
    if (per < 1) per = 1;
    for (;;) {
      long long todo = per;
      if (o.max_steps > 0 && stats.steps + todo > o.max_steps) todo = o.max_steps - stats.steps;
      st = run_window(g, d, o.scheme, o.clamp, (float)o.band, o.band_margin, fdt, todo,
                      o.use_graph != 0 && todo == per);
      if (st != HJ_OK) return st;
      stats.steps += todo;
      stats.windows += 1;
      float r = bits_to_float(g->hscal[4]);
      stats.residual = r;
      if (!std::isfinite(r)) {
        rc = fail(HJ_ERR_DIVERGED, "non-finite value after %lld steps", stats.steps);
        break;
      }
      if ((double)r < o.tol) {
        stats.converged = 1;
        break;
      }
      if (o.max_steps > 0 && stats.steps >= o.max_steps) {
        rc = fail(HJ_ERR_NOT_CONVERGED, "step cap %lld reached (residual %g)", o.max_steps,
                  (double)r);
        break;
      }
      double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                      .count();
      if (o.max_wall_ms > 0.0 && ms > o.max_wall_ms) {
        rc = fail(HJ_ERR_NOT_CONVERGED, "wall-time cap reached (residual %g)", (double)r);
        break;
      }
    }
  }
  stats.t = dt * (double)stats.steps;
  stats.wall_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (s) *s = stats;
  return rc;
}

// dst.W = min(src.W(x - shift), l_dst); fill: source points outside the
// source box give l_dst instead of an error.
static hj_status migrate(hj_grid src, hj_grid dst, const double* shift, int fill) {
  DeviceGuard dg(dst->device);
  hjk::Shift sh;
  std::memset(&sh, 0, sizeof(sh));
  for (int i = 0; i < dst->ndim; ++i) sh.s[i] = shift ? shift[i] : 0.0;
  sh.fill_outside = fill;
  cudaEvent_t ev;
  HJ_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaEventRecord(ev, src->stream);
  cudaStreamWaitEvent(dst->stream, ev, 0);
  cudaEventDestroy(ev);
  HJ_CU(cudaMemsetAsync(dst->dscal + 5, 0, sizeof(unsigned), dst->stream));
  HJ_CU(hjk::launch_prolong(devgrid(src), src->W, devgrid(dst), dst->W, sh,
                            (int*)(dst->dscal + 5), dst->stream));
  HJ_CU(cudaMemcpyAsync(dst->hscal + 5, dst->dscal + 5, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        dst->stream));
  HJ_CU(cudaStreamSynchronize(dst->stream));
  if (dst->hscal[5]) return fail(HJ_ERR_ARG, "a fine node lies outside the coarse grid");
  dst->has_value = true;
  return HJ_OK;
}

hj_status hj_prolong(hj_grid coarse, hj_grid fine) {
  if (!coarse || !fine) return fail(HJ_ERR_ARG, "grid is NULL");
  if (coarse == fine) return fail(HJ_ERR_ARG, "source and target are the same grid");
  if (coarse->ndim != fine->ndim) return fail(HJ_ERR_ARG, "grids differ in ndim");
  if (coarse->device != fine->device) return fail(HJ_ERR_ARG, "grids on different devices");
  if (!coarse->has_value) return fail(HJ_ERR_STATE, "coarse grid holds no value");
  if (fine->con_kind < 0) return fail(HJ_ERR_STATE, "fine grid has no constraint");
  for (int i = 0; i < fine->ndim; ++i) {
    double tol = 1e-9 * coarse->h[i];
    if (fine->lo[i] < coarse->lo[i] - tol || fine->hi[i] > coarse->hi[i] + tol)
      return fail(HJ_ERR_ARG, "fine box leaves the coarse box on axis %d", i);
  }
  return migrate(coarse, fine, nullptr, 0);
}

hj_status hj_translate(hj_grid src, hj_grid dst, const double* shift) {
  if (!src || !dst || !shift) return fail(HJ_ERR_ARG, "NULL argument");
  if (src == dst) return fail(HJ_ERR_ARG, "source and target are the same grid");
  if (src->ndim != dst->ndim) return fail(HJ_ERR_ARG, "grids differ in ndim");
  if (src->device != dst->device) return fail(HJ_ERR_ARG, "grids on different devices");
  if (!src->has_value) return fail(HJ_ERR_STATE, "source grid holds no value");
  if (dst->con_kind < 0) return fail(HJ_ERR_STATE, "target grid has no constraint");
  if (src->model != dst->model || src->model < 0)
    return fail(HJ_ERR_ARG, "source and target have different dynamics");
  for (int i = 0; i < 8; ++i)
    if (src->params[i] != dst->params[i])
      return fail(HJ_ERR_ARG, "source and target have different model parameters");
  if (src->dfield_nd > 0 || dst->dfield_nd > 0)
    return fail(HJ_ERR_STATE, "a state-dependent disturbance bound is not translation invariant");
  for (int i = 0; i < dst->ndim; ++i) {
    if (!std::isfinite(shift[i])) return fail(HJ_ERR_ARG, "shift must be finite");
    // f depends on every axis but the position (axis 0) for the quadcopter
    // blocks, on none for the drift
    bool invariant = dst->model == HJ_DRIFT || i == 0;
    if (shift[i] != 0.0 && !invariant)
      return fail(HJ_ERR_ARG, "the dynamics are not invariant along axis %d", i);
  }
  return migrate(src, dst, shift, 1);
}

hj_status hj_set_value(hj_grid g, const float* src, int on_device) {
  if (!g || !src) return fail(HJ_ERR_ARG, "NULL argument");
  DeviceGuard dg(g->device);
  HJ_CU(cudaMemcpyAsync(g->W, src, (size_t)g->npts * sizeof(float),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream));
  HJ_CU(cudaStreamSynchronize(g->stream));
  g->has_value = true;
  return HJ_OK;
}

hj_status hj_get_value(hj_grid g, float* dst, int on_device) {
  if (!g || !dst) return fail(HJ_ERR_ARG, "NULL argument");
  if (!g->has_value) return fail(HJ_ERR_STATE, "grid holds no value yet");
  DeviceGuard dg(g->device);
  HJ_CU(cudaMemcpyAsync(dst, g->W, (size_t)g->npts * sizeof(float),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
  HJ_CU(cudaStreamSynchronize(g->stream));
  return HJ_OK;
}

static hj_status query(hj_grid g, int npts, const double* x, double* out, int grad) {
  if (!g || npts < 0 || (npts > 0 && (!x || !out))) return fail(HJ_ERR_ARG, "bad query arguments");
  if (!g->has_value) return fail(HJ_ERR_STATE, "grid holds no value yet");
  if (npts == 0) return HJ_OK;
  DeviceGuard dg(g->device);
  size_t nin = (size_t)npts * g->ndim;
  size_t nout = grad ? nin : (size_t)npts;
  size_t need = nin + nout;
  if (need > g->qcap) {
    hja::dev_free(g->alloc, g->qbuf);
    g->qbuf = nullptr;
    g->qcap = 0;
    HJ_CU(hja::dev_malloc(g->alloc, (void**)&g->qbuf, need * sizeof(double)));
    g->qcap = need;
  }
  HJ_CU(cudaMemsetAsync(g->dscal + 5, 0, sizeof(unsigned), g->stream));
  HJ_CU(cudaMemcpyAsync(g->qbuf, x, nin * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  HJ_CU(hjk::launch_query(devgrid(g), g->W, npts, g->qbuf, g->qbuf + nin, (int*)(g->dscal + 5),
                          grad, g->stream));
  HJ_CU(cudaMemcpyAsync(out, g->qbuf + nin, nout * sizeof(double), cudaMemcpyDeviceToHost,
                        g->stream));
  HJ_CU(cudaMemcpyAsync(g->hscal + 5, g->dscal + 5, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        g->stream));
  HJ_CU(cudaStreamSynchronize(g->stream));
  if (g->hscal[5]) return fail(HJ_ERR_ARG, "query point outside the grid box");
  return HJ_OK;
}

hj_status hj_query_value(hj_grid g, int npts, const double* x, double* v_out) {
  return query(g, npts, x, v_out, 0);
}

hj_status hj_query_gradient(hj_grid g, int npts, const double* x, double* grad_out) {
  return query(g, npts, x, grad_out, 1);
}

}  // extern "C"
