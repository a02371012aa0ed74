// hj_server.cu -- continuous-batching server for safety-update solves.
//
// In the paper's runtime (Sec. II-C, Sec. III), every new disturbance bound
// from the GP triggers an update of the affected subsystem's safe set, warm
// started from the previous value function when that is valid (Sec. III-B).
// Here one worker thread owns a batch Runner.  Each loop it:
//   1. admits queued requests (arrival order, first fit) while active slots
//      and the HBM budget allow; a request with a dominated resident prior
//      for its key warm-starts from it, every other request starts cold; a
//      request with coarse initialisation (Sec. III-C) first steps a coarse
//      grid, is migrated to its own grid, and then steps that grid warm;
//   2. advances all admitted grids by one round (fused launches, per-grid
//      stop decisions on the device);
//   3. retires finished grids, records latency, and makes each converged
//      value the resident prior of its key.
// Callers submit, poll, wait and read results from any thread.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "hj_batch.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

enum ReqState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2 };

struct Req {
  long long ticket = 0;
  hj_request r{};
  size_t bytes = 0;          // fine grid bytes (plus the coarse grids while they live)
  size_t coarse_bytes = 0;   // current coarse level
  long long npts = 0;
  long long coarse_npts = 0; // current coarse level
  int phase = 0;             // 0: single solve; 1: coarse phase; 2: fine phase after migration
  hj_grid gc = nullptr;      // grid of the current coarse level
  int nlev = 0, lev = 0;     // coarse levels, and the one stepping now
  int lev_n[2] = {0, 0};     // nodes per axis of each coarse level
  long long lev_npts[2] = {0, 0};
  size_t lev_bytes[2] = {0, 0};
  long long coarse_steps = 0;
  Clock::time_point t_submit, t_done;
  int state = Q_QUEUED;
  hj_grid g = nullptr;
  int slot = -1;
  hj_status result = HJ_OK;
  hj_solve_stats stats{};
  bool released = false;
  bool resident = false;   // this grid is the current prior of its key
  bool cancel = false;
  Clock::time_point last_use;
};

size_t grid_bytes(long long npts) {
  size_t f = ((size_t)npts * sizeof(float) + 255) & ~(size_t)255;
  return 4 * f + 64 * sizeof(unsigned) + 4096;
}

bool same_geometry(const hj_request& a, const hj_request& b) {
  if (a.ndim != b.ndim || a.model != b.model || a.nparams != b.nparams) return false;
  for (int i = 0; i < a.ndim; ++i)
    if (a.n[i] != b.n[i] || a.lo[i] != b.lo[i] || a.hi[i] != b.hi[i]) return false;
  for (int i = 0; i < a.nparams; ++i)
    if (a.params[i] != b.params[i]) return false;
  return a.opts.scheme == b.opts.scheme;
}

// The prior's fixed point dominates the new one (so a warm start reaches the
// new fixed point exactly): disturbance box inside the new one, constraint
// box containing the new one (l_prior >= l_new everywhere).
bool dominates(const hj_request& prior, const hj_request& req) {
  if (!same_geometry(prior, req) || prior.nd != req.nd) return false;
  for (int i = 0; i < req.nd; ++i)
    if (prior.d_lo[i] < req.d_lo[i] || prior.d_hi[i] > req.d_hi[i]) return false;
  if (prior.con_ball != req.con_ball) return false;
  if (!req.con_ball) {
    for (int i = 0; i < req.ndim; ++i)
      if (prior.con_a[i] > req.con_a[i] || prior.con_b[i] < req.con_b[i]) return false;
  } else {
    for (int i = 0; i < req.ndim; ++i)
      if (prior.con_a[i] != req.con_a[i]) return false;
    if (prior.con_b[0] > req.con_b[0]) return false;  // smaller obstacle = larger margin
  }
  return true;
}

// Dominance modulo a translation (hj_translate): along axes the dynamics do
// not depend on (the position axis of the quadcopter blocks, every axis of a
// drift) the prior's constraint may be moved by *shift; it must then contain
// the new one.  The shift centres the prior's box on the new one.  False when
// no translation is needed (plain dominance covers that).
bool dominates_translated(const hj_request& prior, const hj_request& req, double* shift) {
  if (!same_geometry(prior, req) || prior.nd != req.nd) return false;
  for (int i = 0; i < req.nd; ++i)
    if (prior.d_lo[i] < req.d_lo[i] || prior.d_hi[i] > req.d_hi[i]) return false;
  if (prior.con_ball != req.con_ball) return false;
  bool moved = false;
  for (int i = 0; i < req.ndim; ++i) {
    shift[i] = 0.0;
    bool invariant = req.model == HJ_DRIFT || i == 0;
    double pa = prior.con_a[i], pb = prior.con_b[i], ra = req.con_a[i], rb = req.con_b[i];
    if (!req.con_ball) {
      if (invariant && std::isfinite(pa) && std::isfinite(pb) && std::isfinite(ra) &&
          std::isfinite(rb))
        shift[i] = 0.5 * ((ra + rb) - (pa + pb));
      double tol = 1e-9 * (1.0 + std::fabs(ra) + std::fabs(rb));
      if (pa + shift[i] > ra + tol || pb + shift[i] < rb - tol) return false;
    } else {
      if (invariant) shift[i] = ra - pa;
      else if (pa != ra) return false;
    }
    moved = moved || shift[i] != 0.0;
  }
  if (req.con_ball && prior.con_b[0] > req.con_b[0]) return false;
  return moved;
}

// Solve options of the coarse levels: the request's, with its coarse scheme.
hj_solve_opts coarse_opts(const hj_request& r) {
  hj_solve_opts o = r.opts;
  if (r.coarse_scheme) o.scheme = r.coarse_scheme;
  return o;
}

hj_status make_grid(const hj_request& r, cudaStream_t s, hj_grid* out) {
  hj_grid g = nullptr;
  hj_status st = hj_grid_create(&g, r.ndim, r.n, r.lo, r.hi, s);
  if (st != HJ_OK) return st;
  if ((st = hj_set_dynamics(g, r.model, r.params, r.nparams)) == HJ_OK &&
      (st = hj_set_disturbance_bound(g, r.d_lo, r.d_hi, r.nd)) == HJ_OK) {
    st = r.con_ball ? hj_set_constraint_ball(g, r.con_a, r.con_b[0])
                    : hj_set_constraint(g, r.con_a, r.con_b);
  }
  if (st != HJ_OK) {
    hj_grid_destroy(g);
    return st;
  }
  *out = g;
  return HJ_OK;
}

}  // namespace

struct hj_server_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  int max_active = 0;
  hjb::Runner* runner = nullptr;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;

  long long next_ticket = 1;
  std::map<long long, Req> reqs;
  std::deque<long long> queue;
  std::map<long long, long long> resident_of_key;  // key -> ticket holding the prior
  size_t used = 0;
  int order = HJ_ORDER_FIFO;
  long long max_active_nodes = 0;
  bool translated_starts = false;  // warm starts from translated priors (opt-in)
  long long active_nodes = 0;
  hj_server_stats st{};
  std::vector<double> latencies;
  bool first_submit_seen = false;
  Clock::time_point t_first, t_last_done;

  void run();
  void admit_locked(std::vector<long long>& admitted);
  bool evict_locked(size_t need);
  void free_req_locked(Req& q);
};

void hj_server_s::free_req_locked(Req& q) {
  if (q.g) {
    hj_grid_destroy(q.g);
    q.g = nullptr;
    used -= q.bytes;
  }
}

// Free released grids that are only kept as priors, least recently used first.
bool hj_server_s::evict_locked(size_t need) {
  while (used + need > budget) {
    Req* victim = nullptr;
    for (auto& kv : reqs) {
      Req& q = kv.second;
      if (q.state == Q_DONE && q.released && q.g &&
          (!victim || q.last_use < victim->last_use))
        victim = &q;
    }
    if (!victim) return false;
    if (victim->resident) {
      resident_of_key.erase(victim->r.key);
      victim->resident = false;
    }
    free_req_locked(*victim);
    st.evictions++;
  }
  return true;
}

// Estimated work of a request: nodes x largest axis length (steps ~ 1 / h).
static double est_work(const Req& q) {
  int m = 1;
  for (int i = 0; i < q.r.ndim; ++i) m = std::max(m, q.r.n[i]);
  return (double)q.npts * (double)m;
}

void hj_server_s::admit_locked(std::vector<long long>& admitted) {
  if (order == HJ_ORDER_SHORTEST && queue.size() > 1) {
    std::stable_sort(queue.begin(), queue.end(), [&](long long a, long long b) {
      return est_work(reqs[a]) < est_work(reqs[b]);
    });
  }
  for (auto it = queue.begin(); it != queue.end();) {
    if (runner->active() >= max_active) break;
    Req& q = reqs[*it];
    if (q.cancel) {
      q.state = Q_DONE;
      q.result = HJ_ERR_ABORTED;
      q.t_done = Clock::now();
      st.failed++;
      it = queue.erase(it);
      cv_done.notify_all();
      continue;
    }
    // the node cap keeps large grids from time-slicing each other; grids
    // below 1/64 of it ride along regardless (they barely load the GPU)
    if (max_active_nodes > 0 && runner->active() > 0 && q.npts * 64 > max_active_nodes &&
        active_nodes + q.npts > max_active_nodes) {
      ++it;
      continue;
    }
    if (used + q.bytes > budget && !evict_locked(q.bytes)) {
      ++it;  // first fit: a later, smaller request may still fit
      continue;
    }
    hj_grid g = nullptr;
    hj_status s = make_grid(q.r, stream, &g);
    int mode = HJ_COLD;
    bool coarse_first = q.coarse_npts > 0;
    if (s == HJ_OK && coarse_first) {
      // coarse initialisation: the coarse grid steps first; the fine grid
      // waits for the migrated value
      hj_request rc = q.r;
      for (int i = 0; i < rc.ndim; ++i) rc.n[i] = q.lev_n[0];
      s = make_grid(rc, stream, &q.gc);
      int slot = -1;
      if (s == HJ_OK) s = runner->add(q.gc, HJ_COLD, coarse_opts(q.r), &slot);
      if (s != HJ_OK) {
        if (q.gc) hj_grid_destroy(q.gc);
        q.gc = nullptr;
        hj_grid_destroy(g);
        q.state = Q_DONE;
        q.result = s;
        q.t_done = Clock::now();
        st.failed++;
        it = queue.erase(it);
        cv_done.notify_all();
        continue;
      }
      q.g = g;
      q.slot = slot;
      q.phase = 1;
      q.state = Q_RUNNING;
      used += q.bytes;
      active_nodes += q.coarse_npts;
      st.peak_bytes = std::max<long long>(st.peak_bytes, (long long)used);
      st.admitted++;
      st.cold_starts++;
      admitted.push_back(q.ticket);
      it = queue.erase(it);
      continue;
    }
    // Only the VI clamp (Eq. 2) reaches the same fixed point from every
    // dominating start.  Under the monotone clamp the limit depends on the
    // start, so such a request always solves cold.
    if (s == HJ_OK && q.r.mode == HJ_WARM && q.r.key != 0 && q.r.opts.clamp == HJ_CLAMP_VI) {
      auto rk = resident_of_key.find(q.r.key);
      if (rk != resident_of_key.end()) {
        Req& p = reqs[rk->second];
        double shift[HJ_MAX_DIM];
        if (p.g && dominates(p.r, q.r)) {
          cudaError_t e = cudaMemcpyAsync(g->W, p.g->W, (size_t)q.npts * sizeof(float),
                                          cudaMemcpyDeviceToDevice, stream);
          if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
          if (e == cudaSuccess) {
            g->has_value = true;
            mode = HJ_WARM;
            p.last_use = Clock::now();
          }
        } else if (translated_starts && p.g && dominates_translated(p.r, q.r, shift)) {
          if (hj_translate(p.g, g, shift) == HJ_OK) {
            mode = HJ_WARM;
            st.translated_starts++;
            p.last_use = Clock::now();
          }
        }
      }
    }
    int slot = -1;
    if (s == HJ_OK) s = runner->add(g, mode, q.r.opts, &slot);
    if (s != HJ_OK) {
      if (g) hj_grid_destroy(g);
      q.state = Q_DONE;
      q.result = s;
      q.t_done = Clock::now();
      st.failed++;
      it = queue.erase(it);
      cv_done.notify_all();
      continue;
    }
    q.g = g;
    q.slot = slot;
    q.state = Q_RUNNING;
    used += q.bytes;
    active_nodes += q.npts;
    st.peak_bytes = std::max<long long>(st.peak_bytes, (long long)used);
    st.admitted++;
    if (mode == HJ_WARM) st.warm_starts++; else st.cold_starts++;
    admitted.push_back(q.ticket);
    it = queue.erase(it);
  }
}

void hj_server_s::run() {
  hja::DeviceGuard dg(device);
  std::vector<long long> running;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      std::vector<long long> admitted;
      admit_locked(admitted);
      running.insert(running.end(), admitted.begin(), admitted.end());
      // cancellations of running requests
      for (long long t : running) {
        Req& q = reqs[t];
        if (q.cancel && q.state == Q_RUNNING && !runner->finished(q.slot)) runner->cancel(q.slot);
      }
      if (running.empty()) {
        if (stop && queue.empty()) return;
        cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        continue;
      }
    }
    hj_status rs = runner->round(true);
    std::lock_guard<std::mutex> lk(mu);
    st.rounds++;
    auto now = Clock::now();
    for (auto it = running.begin(); it != running.end();) {
      Req& q = reqs[*it];
      if (rs == HJ_OK && q.phase == 1 && runner->finished(q.slot)) {
        // coarse phase done: migrate to the fine grid and step it from there
        hj_solve_stats cs{};
        hj_status r = runner->collect(q.slot, &cs);
        q.coarse_steps += cs.steps;
        st.updates += (double)q.coarse_npts * (double)cs.steps;
        int slot = -1;
        if (q.lev + 1 < q.nlev) {
          // next coarse level: migrate up one level and step it warm
          hj_request rn = q.r;
          for (int i = 0; i < rn.ndim; ++i) rn.n[i] = q.lev_n[q.lev + 1];
          hj_grid gn = nullptr;
          if (r == HJ_OK || r == HJ_ERR_NOT_CONVERGED) r = make_grid(rn, stream, &gn);
          if (r == HJ_OK) r = hj_prolong(q.gc, gn);
          if (r == HJ_OK) r = runner->add(gn, HJ_WARM, coarse_opts(q.r), &slot);
          hj_grid_destroy(q.gc);
          q.gc = nullptr;
          used -= q.coarse_bytes;
          q.bytes -= q.coarse_bytes;
          active_nodes -= q.coarse_npts;
          if (r == HJ_OK) {
            q.lev++;
            q.gc = gn;
            q.slot = slot;
            q.coarse_npts = q.lev_npts[q.lev];
            q.coarse_bytes = q.lev_bytes[q.lev];
            active_nodes += q.coarse_npts;
            ++it;
            continue;
          }
          if (gn) hj_grid_destroy(gn);
          // the remaining coarse level's reservation goes with the failure
          used -= q.lev_bytes[q.lev + 1];
          q.bytes -= q.lev_bytes[q.lev + 1];
          q.coarse_npts = 0;
          q.coarse_bytes = 0;
        } else {
          if (r == HJ_OK || r == HJ_ERR_NOT_CONVERGED) r = hj_prolong(q.gc, q.g);
          if (r == HJ_OK) r = runner->add(q.g, HJ_WARM, q.r.opts, &slot);
          hj_grid_destroy(q.gc);
          q.gc = nullptr;
          used -= q.coarse_bytes;
          q.bytes -= q.coarse_bytes;
          active_nodes -= q.coarse_npts;
          q.coarse_npts = 0;
          q.coarse_bytes = 0;
        }
        if (r == HJ_OK) {
          q.slot = slot;
          q.phase = 2;
          active_nodes += q.npts;
          ++it;
          continue;
        }
        q.result = r;
        q.state = Q_DONE;
        q.t_done = now;
        q.last_use = now;
        t_last_done = now;
        st.failed++;
        latencies.push_back(ms_since(q.t_submit, now));
        it = running.erase(it);
        continue;
      }
      if (rs != HJ_OK || runner->finished(q.slot)) {
        hj_solve_stats s{};
        hj_status r = rs != HJ_OK ? rs : runner->collect(q.slot, &s);
        q.result = r;
        s.wall_ms = ms_since(q.t_submit, now);
        q.stats = s;
        q.state = Q_DONE;
        q.t_done = now;
        q.last_use = now;
        t_last_done = now;
        active_nodes -= q.phase == 1 ? q.coarse_npts : q.npts;
        if (q.gc) {
          hj_grid_destroy(q.gc);
          q.gc = nullptr;
          // this level and any level not reached yet
          size_t left = 0;
          for (int l = q.lev; l < q.nlev; ++l) left += q.lev_bytes[l];
          used -= left;
          q.bytes -= left;
        }
        latencies.push_back(s.wall_ms);
        // grid-point updates count for every request that stepped, converged or not
        st.updates += (double)q.npts * (double)s.steps;
        if (r == HJ_OK) {
          st.completed++;
          if (q.r.key != 0) {
            auto rk = resident_of_key.find(q.r.key);
            if (rk != resident_of_key.end() && rk->second != q.ticket) {
              Req& old = reqs[rk->second];
              old.resident = false;
              if (old.released) free_req_locked(old);
            }
            resident_of_key[q.r.key] = q.ticket;
            q.resident = true;
          }
        } else {
          st.failed++;
        }
        if (q.released && !q.resident) free_req_locked(q);
        it = running.erase(it);
      } else {
        ++it;
      }
    }
    cv_done.notify_all();
  }
}

extern "C" {

hj_status hj_server_create(hj_server* out, long long hbm_budget_bytes, int max_active,
                           void* cuda_stream) {
  if (!out) return hja::fail(HJ_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes <= 0 || max_active < 1 || max_active > 1024)
    return hja::fail(HJ_ERR_ARG, "need a positive budget and 1..1024 active slots");
  int count = 0;
  cudaError_t ce = cudaGetDeviceCount(&count);
  if (ce != cudaSuccess || count == 0)
    return hja::fail(HJ_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(ce));
  hj_server s = new (std::nothrow) hj_server_s();
  if (!s) return hja::fail(HJ_ERR_OOM, "host allocation failed");
  HJ_CU(cudaGetDevice(&s->device));
  s->budget = (size_t)hbm_budget_bytes;
  s->max_active = max_active;
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete s;
      return hja::fail(HJ_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    }
    s->own_stream = true;
  }
  s->runner = new hjb::Runner(s->device, s->stream, max_active);
  hj_status st = s->runner->init();
  if (st != HJ_OK) {
    delete s->runner;
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return st;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return HJ_OK;
}

void hj_server_destroy(hj_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (long long t : s->queue) s->reqs[t].cancel = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  {
    hja::DeviceGuard dg(s->device);
    delete s->runner;
    for (auto& kv : s->reqs)
      if (kv.second.g) hj_grid_destroy(kv.second.g);
    if (s->own_stream) cudaStreamDestroy(s->stream);
  }
  delete s;
}

hj_status hj_server_submit(hj_server s, const hj_request* r, long long* ticket) {
  if (!s || !r || !ticket) return hja::fail(HJ_ERR_ARG, "NULL argument");
  if (r->ndim < 1 || r->ndim > HJ_MAX_DIM) return hja::fail(HJ_ERR_ARG, "bad ndim");
  long long npts = 1;
  for (int i = 0; i < r->ndim; ++i) {
    if (r->n[i] < 3) return hja::fail(HJ_ERR_ARG, "axis %d has fewer than 3 nodes", i);
    npts *= r->n[i];
    if (npts >= (1ll << 31)) return hja::fail(HJ_ERR_ARG, "grid too large");
  }
  if (r->mode != HJ_COLD && r->mode != HJ_WARM) return hja::fail(HJ_ERR_ARG, "bad mode");
  int lev_n[2] = {0, 0};
  int nlev = 0;
  if (r->coarse_n != 0) {
    if (r->coarse_n < 3) return hja::fail(HJ_ERR_ARG, "coarse_n must be 0 or >= 3");
    lev_n[nlev++] = r->coarse_n;
  }
  if (r->coarse_n2 != 0) {
    if (!r->coarse_n || r->coarse_n2 <= r->coarse_n)
      return hja::fail(HJ_ERR_ARG, "coarse_n2 needs coarse_n < coarse_n2");
    lev_n[nlev++] = r->coarse_n2;
  }
  if (r->coarse_scheme != 0 && r->coarse_scheme != HJ_FIRST &&
      r->coarse_scheme != HJ_ENO2 && r->coarse_scheme != HJ_WENO5)
    return hja::fail(HJ_ERR_ARG, "bad coarse_scheme");
  long long lev_npts[2] = {0, 0};
  size_t lev_bytes[2] = {0, 0};
  for (int l = 0; l < nlev; ++l) {
    lev_npts[l] = 1;
    for (int i = 0; i < r->ndim; ++i) {
      if (lev_n[l] > r->n[i]) return hja::fail(HJ_ERR_ARG, "coarse level exceeds axis %d", i);
      lev_npts[l] *= lev_n[l];
    }
    lev_bytes[l] = grid_bytes(lev_npts[l]);
  }
  size_t cbytes = lev_bytes[0] + lev_bytes[1];
  size_t bytes = grid_bytes(npts) + cbytes;
  std::lock_guard<std::mutex> lk(s->mu);
  if (bytes > s->budget) {
    s->st.rejected++;
    return hja::fail(HJ_ERR_OOM, "request needs %zu bytes, budget is %zu", bytes, s->budget);
  }
  Req q;
  q.ticket = s->next_ticket++;
  q.r = *r;
  q.bytes = bytes;
  q.nlev = nlev;
  for (int l = 0; l < 2; ++l) {
    q.lev_n[l] = lev_n[l];
    q.lev_npts[l] = lev_npts[l];
    q.lev_bytes[l] = lev_bytes[l];
  }
  q.coarse_bytes = lev_bytes[0];
  q.npts = npts;
  q.coarse_npts = lev_npts[0];
  q.t_submit = Clock::now();
  q.last_use = q.t_submit;
  if (!s->first_submit_seen) {
    s->first_submit_seen = true;
    s->t_first = q.t_submit;
  }
  s->reqs[q.ticket] = q;
  s->queue.push_back(q.ticket);
  s->st.submitted++;
  *ticket = q.ticket;
  s->cv_work.notify_all();
  return HJ_OK;
}

hj_status hj_server_poll(hj_server s, long long ticket, int* done, hj_status* result,
                         hj_solve_stats* st) {
  if (!s || !done) return hja::fail(HJ_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return hja::fail(HJ_ERR_ARG, "unknown ticket %lld", ticket);
  *done = it->second.state == Q_DONE;
  if (*done) {
    if (result) *result = it->second.result;
    if (st) *st = it->second.stats;
  }
  return HJ_OK;
}

hj_status hj_server_wait(hj_server s, long long ticket, double timeout_ms, hj_status* result,
                         hj_solve_stats* st) {
  if (!s) return hja::fail(HJ_ERR_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return hja::fail(HJ_ERR_ARG, "unknown ticket %lld", ticket);
  auto pred = [&] { return s->reqs[ticket].state == Q_DONE; };
  if (timeout_ms > 0.0) {
    if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred))
      return hja::fail(HJ_ERR_NOT_CONVERGED, "timeout waiting for ticket %lld", ticket);
  } else {
    s->cv_done.wait(lk, pred);
  }
  Req& q = s->reqs[ticket];
  if (result) *result = q.result;
  if (st) *st = q.stats;
  return HJ_OK;
}

hj_status hj_server_get_value(hj_server s, long long ticket, float* dst, int on_device) {
  if (!s || !dst) return hja::fail(HJ_ERR_ARG, "NULL argument");
  hj_grid g = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return hja::fail(HJ_ERR_ARG, "unknown ticket %lld", ticket);
    Req& q = it->second;
    if (q.state != Q_DONE) return hja::fail(HJ_ERR_STATE, "ticket %lld not finished", ticket);
    if (q.released || !q.g) return hja::fail(HJ_ERR_STATE, "ticket %lld released", ticket);
    g = q.g;
    // the worker only frees released grids, so g stays valid for this copy
    q.last_use = Clock::now();
    return hj_get_value(g, dst, on_device);
  }
}

hj_status hj_server_release(hj_server s, long long ticket) {
  if (!s) return hja::fail(HJ_ERR_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return hja::fail(HJ_ERR_ARG, "unknown ticket %lld", ticket);
  Req& q = it->second;
  q.released = true;
  if (q.state == Q_DONE && !q.resident) s->free_req_locked(q);
  return HJ_OK;
}

hj_status hj_server_cancel(hj_server s, long long ticket) {
  if (!s) return hja::fail(HJ_ERR_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return hja::fail(HJ_ERR_ARG, "unknown ticket %lld", ticket);
  it->second.cancel = true;
  s->cv_work.notify_all();
  return HJ_OK;
}

hj_status hj_server_set_policy(hj_server s, int order, long long max_active_nodes) {
  if (!s) return hja::fail(HJ_ERR_ARG, "NULL server");
  if (order != HJ_ORDER_FIFO && order != HJ_ORDER_SHORTEST) return hja::fail(HJ_ERR_ARG, "bad order");
  if (max_active_nodes < 0) return hja::fail(HJ_ERR_ARG, "max_active_nodes must be >= 0");
  std::lock_guard<std::mutex> lk(s->mu);
  s->order = order;
  s->max_active_nodes = max_active_nodes;
  s->cv_work.notify_all();
  return HJ_OK;
}

hj_status hj_server_set_translated_starts(hj_server s, int enable) {
  if (!s) return hja::fail(HJ_ERR_ARG, "NULL server");
  if (enable != 0 && enable != 1) return hja::fail(HJ_ERR_ARG, "enable must be 0 or 1");
  std::lock_guard<std::mutex> lk(s->mu);
  s->translated_starts = enable != 0;
  return HJ_OK;
}

hj_status hj_server_get_stats(hj_server s, hj_server_stats* out) {
  if (!s || !out) return hja::fail(HJ_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  hj_server_stats r = s->st;
  r.bytes_in_use = (long long)s->used;
  r.queued = (long long)s->queue.size();
  long long act = 0;
  for (auto& kv : s->reqs)
    if (kv.second.state == Q_RUNNING) act++;
  r.active = act;
  std::vector<double> l = s->latencies;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
      double idx = p * (double)(l.size() - 1);
      size_t i = (size_t)std::floor(idx);
      size_t j = std::min(i + 1, l.size() - 1);
      double f = idx - (double)i;
      return l[i] * (1.0 - f) + l[j] * f;
    };
    r.p50_ms = pct(0.50);
    r.p99_ms = pct(0.99);
  }
  r.busy_ms = s->first_submit_seen && r.completed + r.failed > 0 ? ms_since(s->t_first, s->t_last_done)
                                                                  : 0.0;
  *out = r;
  return HJ_OK;
}

}  // extern "C"
