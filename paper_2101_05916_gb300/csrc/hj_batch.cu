// hj_batch.cu -- decomposed subsystems stepped together (Sec. III-A: the
// x, y and z blocks of the 10-D quadcopter are independent problems, and the
// paper runs them in parallel).
//
// Each TVD-RK3 stage is ONE launch per grid kind (model, ndim, scheme) over
// the blocks of all active grids of that kind.  Within a launch, a block first
// finds its grid (binary search over block offsets), copies that grid's
// descriptor into shared memory, and then runs the same per-node stage code
// as the single-grid kernel.  Each kind is compiled separately, so it keeps
// the register use of the single-grid kernel.  After stage 3, a one-block
// control kernel advances
// every grid's step counter.  It also closes check windows (residual vs.
// tol) and clears the `active` flag of grids that converged, hit their cap or
// went non-finite.  So all stop decisions happen on the device, and a round
// of steps is a fixed launch sequence that is captured once as a CUDA graph
// and replayed.  Blocks of inactive grids return at once; the host compacts
// the launch at the next round boundary.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>

#include "hj_batch.h"
#include "hj_stage.cuh"

namespace hjb {

constexpr int kThreads = hjk::kStageThreads;
// Grids with at least this many nodes launch alone (4096 blocks of 256
// threads: several waves of a GPU with about 150 SMs at 8 resident blocks
// each); smaller grids of one kind are fused.
constexpr int kSoloNodes = 1 << 20;

__host__ __device__ constexpr int kind_code(int model, int ndim, int scheme) {
  return model * 100 + ndim * 10 + scheme;
}

static bool batch_supported(int model, int ndim, int scheme) {
  if (model == hjd::M_QUAD_Z) return ndim == 2;
  if (model == hjd::M_QUAD_X4) return ndim == 4;
  if (model == hjd::M_DRIFT) return (ndim == 1 || ndim == 2) && (scheme == 2 || scheme == 5);
  return false;
}

// One fused launch for up to kPackItems active grids of one kind (model,
// ndim, scheme).  It is compiled for that single variant, so its register use
// matches the single-grid kernel.  The descriptors arrive as a
// __grid_constant__ parameter and are indexed by a block-uniform value, so
// their fields are constant-bank reads, as in the single-grid kernel.
template <int STAGE, int D, int S, int M>
__global__ void __launch_bounds__(kThreads) batch_stage(const __grid_constant__ ItemPack pack,
                                                         Ctl* ctl) {
  int lo = 0, hi = pack.count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pack.block_begin[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const Item& it = pack.items[lo];
  const Ctl& c = ctl[it.slot];
  if (!c.active) return;  // uniform: written only by the control kernel
  int lb = blockIdx.x - pack.block_begin[lo];
  int yb = it.bx >= 2 ? hjd::fast_div(lb, it.bx_m, it.bx_s) : lb;
  int bxi = lb - yb * it.bx;
  bool check = STAGE == 3 && c.check_next != 0;
  unsigned r = hjd::stage_point<D, S, M, STAGE>(it.g, it.a[STAGE - 1], bxi * kThreads + threadIdx.x,
                                                yb, check);
  if (STAGE == 3 && check) hjd::block_max_bits(r, &ctl[it.slot].resid);
}

// One stage launch of one pack; false for a kind without a kernel.
static bool launch_kind(int kind, const ItemPack& pack, int blocks, Ctl* ctl, cudaStream_t s,
                        int stage) {
  using namespace hjd;
  auto go = [&](auto k1, auto k2, auto k3) {
    if (stage == 1) k1<<<blocks, kThreads, 0, s>>>(pack, ctl);
    else if (stage == 2) k2<<<blocks, kThreads, 0, s>>>(pack, ctl);
    else k3<<<blocks, kThreads, 0, s>>>(pack, ctl);
  };
#define HJ_KIND(MODEL, D, S)                                                              \
  case kind_code(MODEL, D, S):                                                            \
    go(batch_stage<1, D, S, MODEL>, batch_stage<2, D, S, MODEL>, batch_stage<3, D, S, MODEL>); \
    return true;
  switch (kind) {
    HJ_KIND(M_QUAD_Z, 2, 1)
    HJ_KIND(M_QUAD_Z, 2, 2)
    HJ_KIND(M_QUAD_Z, 2, 5)
    HJ_KIND(M_QUAD_X4, 4, 1)
    HJ_KIND(M_QUAD_X4, 4, 2)
    HJ_KIND(M_QUAD_X4, 4, 5)
    HJ_KIND(M_DRIFT, 1, 2)
    HJ_KIND(M_DRIFT, 1, 5)
    HJ_KIND(M_DRIFT, 2, 2)
    HJ_KIND(M_DRIFT, 2, 5)
    default: return false;
  }
#undef HJ_KIND
}

__global__ void batch_control(const int* __restrict__ slots, int nitems, Ctl* ctl) {
  for (int k = threadIdx.x; k < nitems; k += blockDim.x) {
    Ctl& c = ctl[slots[k]];
    if (!c.active) continue;
    long long s = ++c.steps;
    c.check_next = ((s + 1) % c.per == 0 || s + 1 >= c.max_steps) ? 1 : 0;
    if (s % c.per == 0 || s >= c.max_steps) {
      float r = __uint_as_float(c.resid);
      c.resid = 0u;
      c.last_resid = r;
      c.windows += 1;
      if (!(r <= FLT_MAX)) {
        c.status = S_NONFINITE;
        c.active = 0;
      } else if ((double)r < c.tol) {
        c.status = S_CONVERGED;
        c.active = 0;
      } else if (s >= c.max_steps) {
        c.status = S_CAP;
        c.active = 0;
      }
    }
  }
}

// ------------------------------------------------------------------ host

Runner::Runner(int device, cudaStream_t stream, int capacity)
    : device_(device), stream_(stream), cap_(capacity), slots_(capacity),
      alloc_(hja::current_allocator()) {}

Runner::~Runner() {
  hja::DeviceGuard dg(device_);
  cudaStreamSynchronize(stream_);
  drop_graphs();
  hja::dev_free(alloc_, dev_ctl_);
  hja::dev_free(alloc_, dev_slots_);
  if (host_ctl_) cudaFreeHost(host_ctl_);
  if (cap_stream_) cudaStreamDestroy(cap_stream_);
}

hj_status Runner::init() {
  hja::DeviceGuard dg(device_);
  HJ_CU(hja::dev_malloc(alloc_, (void**)&dev_ctl_, sizeof(Ctl) * cap_));
  HJ_CU(cudaMallocHost(&host_ctl_, sizeof(Ctl) * cap_));
  std::memset(host_ctl_, 0, sizeof(Ctl) * cap_);
  HJ_CU(cudaMemsetAsync(dev_ctl_, 0, sizeof(Ctl) * cap_, stream_));
  HJ_CU(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
  return HJ_OK;
}

void Runner::drop_graphs() {
  for (auto& kv : graphs_) cudaGraphExecDestroy(kv.second);
  graphs_.clear();
}

int Runner::active() const {
  int n = 0;
  for (int i = 0; i < cap_; ++i)
    if (slots_[i].used && !slots_[i].done) ++n;
  return n;
}

hj_status Runner::add(hj_grid g, int mode, const hj_solve_opts& o, int* slot_out) {
  if (!g) return hja::fail(HJ_ERR_ARG, "grid is NULL");
  if (g->device != device_) return hja::fail(HJ_ERR_ARG, "batch grids must share one device");
  if (mode != HJ_COLD && mode != HJ_WARM) return hja::fail(HJ_ERR_ARG, "bad mode");
  if (!(o.cfl > 0.0) || !(o.tol >= 0.0) || !(o.check_dt > 0.0) || o.dt < 0.0 || !(o.band >= 0.0) ||
      o.band_margin < 0)
    return hja::fail(HJ_ERR_ARG, "bad solve options");
  hj_status st = hja::validate_ready(g, o.scheme);
  if (st != HJ_OK) return st;
  if (!batch_supported(g->model, g->ndim, o.scheme))
    return hja::fail(HJ_ERR_ARG, "model %d, %d-D, scheme %d has no batched kernel", g->model,
                     g->ndim, o.scheme);
  if (mode == HJ_WARM && !g->has_value) return hja::fail(HJ_ERR_STATE, "warm start without prior");
  for (int i = 0; i < cap_; ++i)
    if (slots_[i].used && !slots_[i].done && slots_[i].g == g)
      return hja::fail(HJ_ERR_ARG, "grid already stepping in this batch");
  int k = -1;
  for (int i = 0; i < cap_; ++i)
    if (!slots_[i].used) {
      k = i;
      break;
    }
  if (k < 0) return hja::fail(HJ_ERR_OOM, "batch is full (%d grids)", cap_);
  hja::DeviceGuard dg(device_);
  if ((st = hja::ensure_alpha(g)) != HJ_OK) return st;
  if (o.autotune && g->tuned_scheme != o.scheme && (st = hja::autotune(g, o.scheme, o.clamp)) != HJ_OK)
    return st;
  double dt = o.dt > 0.0 ? o.dt : hja::cfl_dt(g, o.cfl);
  // order the grid's own stream before the batch stream
  if (g->stream != stream_) HJ_CU(cudaStreamSynchronize(g->stream));
  hjd::DevGrid d = hja::devgrid(g);
  HJ_CU(hjk::launch_init(d, g->W, g->snap, mode == HJ_WARM ? 1 : 0, stream_));
  g->has_value = true;
  Slot& s = slots_[k];
  s = Slot();
  s.g = g;
  s.used = true;
  s.scheme = o.scheme;
  s.clamp = o.clamp;
  s.band = (float)o.band;
  s.margin = o.band_margin;
  s.dt = dt;
  s.max_wall_ms = o.max_wall_ms;
  s.t0 = std::chrono::steady_clock::now();
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  c.active = dt > 0.0 ? 1 : 0;
  c.status = dt > 0.0 ? S_RUNNING : S_CONVERGED;
  if (o.fixed_steps > 0) {
    s.fixed = true;
    c.per = o.fixed_steps;
    c.max_steps = o.fixed_steps;
    c.tol = -1.0;
  } else {
    long long per = (long long)std::ceil(o.check_dt / std::max(dt, 1e-300) - 1e-9);
    c.per = std::max(per, 1ll);
    c.max_steps = o.max_steps > 0 ? o.max_steps : (1ll << 62);
    c.tol = o.tol;
  }
  c.check_next = (1 % c.per == 0 || 1 >= c.max_steps) ? 1 : 0;
  host_ctl_[k] = c;
  HJ_CU(cudaMemcpyAsync(dev_ctl_ + k, &host_ctl_[k], sizeof(Ctl), cudaMemcpyHostToDevice, stream_));
  HJ_CU(cudaStreamSynchronize(stream_));
  if (!c.active) {
    s.done = true;
  }
  dirty_ = true;
  if (slot_out) *slot_out = k;
  return HJ_OK;
}

hj_status Runner::cancel(int k) {
  if (k < 0 || k >= cap_ || !slots_[k].used) return hja::fail(HJ_ERR_ARG, "bad slot");
  if (slots_[k].done) return HJ_OK;
  hja::DeviceGuard dg(device_);
  // written between rounds only, so no kernel of this runner reads it concurrently
  HJ_CU(cudaStreamSynchronize(stream_));
  host_ctl_[k].active = 0;
  host_ctl_[k].status = S_CANCELLED;
  HJ_CU(cudaMemcpyAsync(dev_ctl_ + k, &host_ctl_[k], sizeof(Ctl), cudaMemcpyHostToDevice, stream_));
  HJ_CU(cudaStreamSynchronize(stream_));
  slots_[k].done = true;
  slots_[k].wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                                slots_[k].t0).count();
  dirty_ = true;
  return HJ_OK;
}

hj_status Runner::rebuild() {
  order_.clear();
  groups_.clear();
  // grids of one kind share fused launches of up to kPackItems grids each
  std::vector<std::pair<int, int>> by_kind;  // (kind, slot)
  for (int k = 0; k < cap_; ++k) {
    Slot& s = slots_[k];
    if (!s.used || s.done) continue;
    by_kind.emplace_back(kind_code(s.g->model, s.g->ndim, s.scheme), k);
  }
  std::stable_sort(by_kind.begin(), by_kind.end(),
                   [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
                     return a.first < b.first;
                   });
  for (size_t j = 0; j < by_kind.size(); ++j) {
    int k = by_kind[j].second;
    Slot& s = slots_[k];
    hj_grid g = s.g;
    if (groups_.empty() || groups_.back().kind != by_kind[j].first ||
        groups_.back().pack.count == kPackItems ||
        groups_.back().pack.items[0].g.npts >= kSoloNodes) {
      groups_.emplace_back();
      Group& ng = groups_.back();
      std::memset(&ng.pack, 0, sizeof(ng.pack));
      ng.kind = by_kind[j].first;
      ng.blocks = 0;
    }
    // a grid that fills the GPU by itself gains nothing from fusion; it keeps
    // its own single-grid launch (a group of one)
    if (g->npts >= kSoloNodes && groups_.back().pack.count > 0) {
      groups_.emplace_back();
      Group& ng = groups_.back();
      std::memset(&ng.pack, 0, sizeof(ng.pack));
      ng.kind = by_kind[j].first;
      ng.blocks = 0;
    }
    Group& gr = groups_.back();
    Item& it = gr.pack.items[gr.pack.count];
    it.g = hja::devgrid(g);
    float dt = (float)s.dt;
    it.a[0] = hjd::StageArgs{g->W, g->W, g->A, nullptr, nullptr, dt, 0, s.clamp, s.band, s.margin};
    it.a[1] = hjd::StageArgs{g->A, g->W, g->B, nullptr, nullptr, dt, 0, s.clamp, s.band, s.margin};
    it.a[2] = hjd::StageArgs{g->B, g->W, g->W, g->snap, nullptr, dt, 1, s.clamp, s.band, s.margin};
    it.kind = by_kind[j].first;
    it.slot = k;
    it.bx = (it.g.plane + kThreads - 1) / kThreads;
    it.by = g->ndim == 4 ? g->n[0] : 1;
    if (it.bx >= 2) hjd::div_consts((unsigned)it.bx, it.bx_m, it.bx_s);
    it.block_begin = gr.blocks;
    gr.pack.block_begin[gr.pack.count] = gr.blocks;
    gr.blocks += it.bx * it.by;
    gr.pack.count += 1;
    gr.pack.block_begin[gr.pack.count] = gr.blocks;
    order_.push_back(k);
  }
  nitems_ = (int)order_.size();
  plan_group();
  if (nitems_ > item_cap_) {
    hja::dev_free(alloc_, dev_slots_);
    dev_slots_ = nullptr;
    item_cap_ = std::max(nitems_, 2 * item_cap_);
    HJ_CU(hja::dev_malloc(alloc_, (void**)&dev_slots_, sizeof(int) * item_cap_));
  }
  if (nitems_) {
    HJ_CU(cudaMemcpyAsync(dev_slots_, order_.data(), sizeof(int) * nitems_, cudaMemcpyHostToDevice,
                          stream_));
    HJ_CU(cudaStreamSynchronize(stream_));
  }
  drop_graphs();
  dirty_ = false;
  return HJ_OK;
}

// The group launch of the current membership: every active grid in blocks
// of kGroupThreads nodes of its flat mapping, at a position of the group
// kernel compiled for a grid of its kind, shape and model constants.  A
// loaded kernel keeps serving while grids retire from the batch: each grid
// keeps a position of its own code, and positions left without a grid get
// no blocks.  Otherwise the current membership's kernel is compiled in the
// background, and group mode starts once it is loaded.
bool Runner::plan_group() {
  std::vector<std::string> keys(nitems_);
  std::vector<hjd::DevGrid> grids(nitems_);
  bool ok = group_allowed_ && nitems_ >= 1 && nitems_ <= kGroupItems;
  for (int i = 0; ok && i < nitems_; ++i) {
    const Slot& s = slots_[order_[i]];
    grids[i] = hja::devgrid(s.g);
    grids[i].tile_rows = 0;
    keys[i] = hjk::code_key(grids[i], s.scheme);
  }
  std::vector<int> pos(nitems_, -1);
  bool reuse = ok && group_mode_ && group_handle_ != nullptr;
  if (reuse) {
    std::vector<bool> taken(gkeys_.size(), false);
    for (int i = 0; i < nitems_ && reuse; ++i) {
      for (size_t p = 0; p < gkeys_.size(); ++p)
        if (!taken[p] && gkeys_[p] == keys[i]) {
          pos[i] = (int)p;
          taken[p] = true;
          break;
        }
      reuse = pos[i] >= 0;
    }
  }
  if (!reuse) {
    group_mode_ = false;
    group_pending_ = false;
    group_handle_ = nullptr;
    gkeys_.clear();
    gcodes_.clear();
    gschemes_.clear();
    if (!ok) return false;
    gkeys_ = keys;
    gcodes_ = grids;
    for (int i = 0; i < nitems_; ++i) {
      gschemes_.push_back(slots_[order_[i]].scheme);
      pos[i] = i;
    }
  }
  // the pack: position p holds current item i with pos[i] == p, or nothing
  std::memset(&gpack_, 0, sizeof(gpack_));
  int npos = (int)gkeys_.size();
  std::vector<int> at(npos, -1);
  for (int i = 0; i < nitems_; ++i) at[pos[i]] = i;
  unsigned blocks = 0;
  for (int p = 0; p < npos; ++p) {
    GroupItem& it = gpack_.items[p];
    gpack_.block_begin[p] = (int)blocks;
    if (at[p] < 0) continue;  // no grid here: no blocks
    int k = order_[at[p]];
    const Slot& s = slots_[k];
    hj_grid g = s.g;
    it.g = grids[at[p]];
    float dt = (float)s.dt;
    it.a[0] = hjd::StageArgs{g->W, g->W, g->A, nullptr, nullptr, dt, 0, s.clamp, s.band, s.margin};
    it.a[1] = hjd::StageArgs{g->A, g->W, g->B, nullptr, nullptr, dt, 0, s.clamp, s.band, s.margin};
    it.a[2] = hjd::StageArgs{g->B, g->W, g->W, g->snap, nullptr, dt, 0, s.clamp, s.band, s.margin};
    it.slot = k;
    it.bx = (it.g.plane + kGroupThreads - 1) / kGroupThreads;
    if (it.bx >= 2) hjd::div_consts((unsigned)it.bx, it.bx_m, it.bx_s);
    blocks += (unsigned)it.bx * (unsigned)(it.g.ndim == 4 ? it.g.n[0] : 1);
  }
  gpack_.count = npos;
  gpack_.block_begin[npos] = (int)blocks;
  gblocks_ = blocks;
  if (reuse) return true;
  group_mode_ = hjk::group_prepare(gcodes_, gschemes_, kGroupThreads, &group_handle_);
  group_pending_ = !group_mode_ && hjk::jit_enabled();
  return group_mode_;
}

// R steps: per step, the three stage launches of every kind group, then the
// control kernel over all grids.  A group holding a single grid uses the
// single-grid kernel, whose descriptor is a plain kernel parameter.  Rounds
// end at the first window boundary of any grid, so such a grid can check only
// at the round's last step, and only when its own window ends there.
cudaError_t Runner::enqueue_round(long long R, cudaStream_t s) {
  if (group_mode_) {
    for (long long i = 0; i < R; ++i) {
      for (int stage = 1; stage <= 3; ++stage) {
        cudaError_t e = hjk::group_launch(group_handle_, stage, &gpack_, dev_ctl_, gblocks_,
                                          kGroupThreads, s);
        if (e != cudaSuccess) return e;
      }
      batch_control<<<1, 256, 0, s>>>(dev_slots_, nitems_, dev_ctl_);
    }
    return cudaGetLastError();
  }
  for (long long i = 0; i < R; ++i) {
    for (int stage = 1; stage <= 3; ++stage) {
      for (const Group& gr : groups_) {
        if (gr.pack.count == 1) {
          const Item& it = gr.pack.items[0];
          hjd::StageArgs a = it.a[stage - 1];
          const Ctl& c = host_ctl_[it.slot];
          long long s1 = c.steps + i + 1;
          a.check = (stage == 3 && (s1 % c.per == 0 || s1 >= c.max_steps)) ? 1 : 0;
          a.resid = &dev_ctl_[it.slot].resid;
          cudaError_t e = hjk::launch_stage(it.g, it.kind % 10, stage, a, s,
                                            slots_[it.slot].g->threads);
          if (e != cudaSuccess) return e;
        } else if (!launch_kind(gr.kind, gr.pack, gr.blocks, dev_ctl_, s, stage)) {
          return cudaErrorInvalidValue;
        }
      }
    }
    batch_control<<<1, 256, 0, s>>>(dev_slots_, nitems_, dev_ctl_);
  }
  return cudaGetLastError();
}

hj_status Runner::sync_ctl() {
  HJ_CU(cudaMemcpyAsync(host_ctl_, dev_ctl_, sizeof(Ctl) * cap_, cudaMemcpyDeviceToHost, stream_));
  HJ_CU(cudaStreamSynchronize(stream_));
  auto now = std::chrono::steady_clock::now();
  for (int k : order_) {
    Slot& s = slots_[k];
    if (s.done) continue;
    if (!host_ctl_[k].active) {
      s.done = true;
      s.wall_ms = std::chrono::duration<double, std::milli>(now - s.t0).count();
      dirty_ = true;
    }
  }
  return HJ_OK;
}

hj_status Runner::round(bool use_graph) {
  hja::DeviceGuard dg(device_);
  hj_status st;
  // the group kernels of the current membership finished compiling: switch
  if (!dirty_ && group_pending_ && !group_mode_) {
    group_mode_ = hjk::group_prepare(gcodes_, gschemes_, kGroupThreads, &group_handle_);
    if (group_mode_) {
      group_pending_ = false;
      drop_graphs();
    }
  }
  bool changed = dirty_;
  if (dirty_ && (st = rebuild()) != HJ_OK) return st;
  if (nitems_ == 0) return HJ_OK;
  // capture only a membership that repeats: a fresh set runs its first round
  // with direct launches
  use_graph = use_graph && !changed;
  // run to the next window boundary of any active grid
  long long R = 1ll << 62;
  for (int k : order_) {
    const Ctl& c = host_ctl_[k];
    long long to_window = c.per - (c.steps % c.per);
    long long to_cap = c.max_steps - c.steps;
    R = std::min(R, std::min(to_window, to_cap));
  }
  // bound a round to about 1e8 grid-point updates (a few ms) so that new
  // arrivals join and finished grids leave promptly
  long long active_nodes = 0;
  for (int k : order_) active_nodes += slots_[k].g->npts;
  long long r_work = std::max(16ll, 100000000ll / std::max(1ll, active_nodes));
  R = std::max(1ll, std::min(R, std::min(r_work, 4096ll)));
  // a single-grid group bakes its check step into the launch, so the graph
  // key holds each such grid's phase within its window
  std::string key = std::to_string(R) + (group_mode_ ? "G" : "");
  static const std::vector<Group> kNoGroups;
  const std::vector<Group>& solo = group_mode_ ? kNoGroups : groups_;
  for (const Group& gr : solo)
    if (gr.pack.count == 1) {
      const Ctl& c = host_ctl_[gr.pack.items[0].slot];
      long long to_cap = c.max_steps - c.steps;
      key += "," + std::to_string(c.steps % c.per) + ":" + std::to_string(to_cap <= R ? to_cap : -1);
    }
  // grids launched on their own may use shape-specialised kernels: they
  // load outside the capture, and a round graph records whether it has them
  for (const Group& gr : solo)
    if (gr.pack.count == 1)
      key += hjk::jit_prepare(gr.pack.items[0].g, gr.pack.items[0].kind % 10,
                              slots_[gr.pack.items[0].slot].g->threads)
                 ? "j"
                 : "p";
  unsigned long long before = hjk::g_launches.load();
  if (use_graph) {
    auto it = graphs_.find(key);
    if (it == graphs_.end()) {
      cudaGraph_t graph = nullptr;
      HJ_CU(cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = enqueue_round(R, cap_stream_);
      cudaError_t e2 = cudaStreamEndCapture(cap_stream_, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return hja::fail(HJ_ERR_CUDA, "batch capture: %s",
                         cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      cudaGraphExec_t ex = nullptr;
      cudaError_t e3 = cudaGraphInstantiate(&ex, graph, 0);
      cudaGraphDestroy(graph);
      if (e3 != cudaSuccess) return hja::fail(HJ_ERR_CUDA, "batch instantiate: %s", cudaGetErrorString(e3));
      if (graphs_.size() > 64) drop_graphs();
      it = graphs_.emplace(key, ex).first;
    }
    HJ_CU(cudaGraphLaunch(it->second, stream_));
  } else {
    HJ_CU(enqueue_round(R, stream_));
  }
  // every kernel of the round counted once: single-grid launches counted
  // themselves while enqueued (also during capture), so top up to the total
  unsigned long long counted = hjk::g_launches.load() - before;
  unsigned long long total =
      (3ull * (group_mode_ ? 1ull : groups_.size()) + 1ull) * (unsigned long long)R;
  if (total > counted) hjk::g_launches.fetch_add(total - counted);
  if ((st = sync_ctl()) != HJ_OK) return st;
  // wall-time caps are host-side and apply between rounds
  auto now = std::chrono::steady_clock::now();
  for (int k : order_) {
    Slot& s = slots_[k];
    if (s.done || s.max_wall_ms <= 0.0) continue;
    double ms = std::chrono::duration<double, std::milli>(now - s.t0).count();
    if (ms > s.max_wall_ms) {
      if ((st = cancel(k)) != HJ_OK) return st;
      s.wall_capped = true;
    }
  }
  return HJ_OK;
}

hj_status Runner::collect(int k, hj_solve_stats* out) {
  if (k < 0 || k >= cap_ || !slots_[k].used || !slots_[k].done)
    return hja::fail(HJ_ERR_ARG, "slot not finished");
  Slot& s = slots_[k];
  const Ctl& c = host_ctl_[k];
  hj_solve_stats st;
  std::memset(&st, 0, sizeof(st));
  st.steps = c.steps;
  st.dt = s.dt;
  st.t = s.dt * (double)c.steps;
  st.residual = c.last_resid;
  st.windows = c.windows;
  st.wall_ms = s.wall_ms;
  st.converged = c.status == S_CONVERGED;
  st.stepped = 1.0;
  hj_status rc = HJ_OK;
  if (s.fixed) {
    st.converged = 0;
    if (c.status == S_NONFINITE) rc = hja::fail(HJ_ERR_DIVERGED, "non-finite value");
  } else if (c.status == S_NONFINITE) {
    rc = hja::fail(HJ_ERR_DIVERGED, "non-finite value after %lld steps", c.steps);
  } else if (c.status == S_CAP || s.wall_capped) {
    rc = hja::fail(HJ_ERR_NOT_CONVERGED, "step or time cap reached (residual %g)", (double)c.last_resid);
  } else if (c.status == S_CANCELLED) {
    rc = hja::fail(HJ_ERR_ABORTED, "cancelled");
  }
  if (out) *out = st;
  s = Slot();
  return rc;
}

}  // namespace hjb

extern "C" hj_status hj_solve_batch(hj_grid* gs, int ngrids, const int* modes,
                                    const hj_solve_opts* opts, int opts_count,
                                    hj_solve_stats* stats, int* status_out) {
  if (!gs || ngrids < 1 || !modes) return hja::fail(HJ_ERR_ARG, "bad batch arguments");
  if (opts && opts_count != 1 && opts_count != ngrids)
    return hja::fail(HJ_ERR_ARG, "opts_count must be 1 or ngrids");
  for (int i = 0; i < ngrids; ++i) {
    if (!gs[i]) return hja::fail(HJ_ERR_ARG, "grid %d is NULL", i);
    for (int j = 0; j < i; ++j)
      if (gs[j] == gs[i]) return hja::fail(HJ_ERR_ARG, "grid %d appears twice", i);
  }
  hjb::Runner r(gs[0]->device, gs[0]->stream, std::max(ngrids, 1));
  r.allow_group(true);
  hj_status st = r.init();
  if (st != HJ_OK) return st;
  std::vector<int> slot(ngrids, -1);
  bool graph = true;
  for (int i = 0; i < ngrids; ++i) {
    hj_solve_opts o;
    hj_default_opts(&o);
    if (opts) o = opts[opts_count == 1 ? 0 : i];
    graph = graph && o.use_graph;
    st = r.add(gs[i], modes[i], o, &slot[i]);
    if (st != HJ_OK) return st;
  }
  while (r.active() > 0) {
    st = r.round(graph);
    if (st != HJ_OK) return st;
  }
  hj_status first = HJ_OK;
  for (int i = 0; i < ngrids; ++i) {
    hj_solve_stats s;
    hj_status si = r.collect(slot[i], &s);
    if (stats) stats[i] = s;
    if (status_out) status_out[i] = si;
    if (first == HJ_OK && si != HJ_OK) first = si;
  }
  return first;
}
