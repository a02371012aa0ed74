// hj_batch.h -- fused multi-grid stepping shared by hj_solve_batch and the server.
#pragma once

#include <chrono>
#include <map>
#include <string>
#include <vector>

#include "hj_grid.h"
#include "hj_group.cuh"

namespace hjb {

// One grid inside a fused launch (device memory; copied to shared memory per block).
struct Item {
  hjd::DevGrid g;
  hjd::StageArgs a[3];  // stage 1..3 arguments (check is decided on the device)
  int kind;             // model * 100 + ndim * 10 + scheme
  int slot;             // index into the control array
  int block_begin;      // first block of this grid in the fused launch
  int bx, by;           // blocks per slab; slabs (first-axis nodes of a 4-D grid, else 1)
  unsigned bx_m;        // bx as a multiply-shift reciprocal (bx >= 2)
  int bx_s;
};

// Grids of one fused launch, passed as a __grid_constant__ kernel parameter.
// A block finds its grid from the block offsets.  Every later descriptor
// read is then a uniform constant-bank load, as in the single-grid kernel,
// rather than a shared-memory load per use.
constexpr int kPackItems = 24;
struct ItemPack {
  int count;
  int block_begin[kPackItems + 1];
  Item items[kPackItems];
};
static_assert(sizeof(ItemPack) <= 32000, "kernel parameters are limited to 32764 bytes");

static_assert(sizeof(GroupPack) <= 32000, "kernel parameters are limited to 32764 bytes");

enum { S_RUNNING = 0, S_CONVERGED = 1, S_CAP = 2, S_NONFINITE = 3, S_CANCELLED = 4 };

// Steps a changing set of grids together.  Grids join with add() and leave
// when their control state says so.  Every round advances all active grids by
// the same number of steps.  Each step is one fused launch per RK stage and
// per grid kind (model, ndim, scheme), plus one control launch.
class Runner {
 public:
  Runner(int device, cudaStream_t stream, int capacity = 1024);
  ~Runner();
  hj_status init();
  // Validate, run the init kernel and set up the control slot.  Returns the slot.
  hj_status add(hj_grid g, int mode, const hj_solve_opts& o, int* slot);
  // Advance every active grid until the next window boundary of any of them.
  hj_status round(bool use_graph);
  // Ask an active slot to stop at the next round boundary.
  hj_status cancel(int slot);
  int active() const;
  bool finished(int slot) const { return slots_[slot].done; }
  // Final state of a finished slot; frees the slot for reuse.
  hj_status collect(int slot, hj_solve_stats* st);
  long long steps_of(int slot) const { return host_ctl_[slot].steps; }
  // Allow group launches (one launch per stage over all grids, compiled per
  // membership).  Worth it for a membership that steps many rounds, as in
  // hj_solve_batch; a server whose membership changes every few rounds
  // would only start compiles it never uses.  Off by default.
  void allow_group(bool on) {
    group_allowed_ = on;
    dirty_ = true;
  }
  cudaStream_t stream() const { return stream_; }

 private:
  struct Slot {
    hj_grid g = nullptr;
    bool used = false, done = false, fixed = false, wall_capped = false;
    int scheme = 5, clamp = 0;
    float band = 0.f;
    int margin = 0;
    double dt = 0.0, max_wall_ms = 0.0;
    std::chrono::steady_clock::time_point t0;
    double wall_ms = 0.0;
  };
  struct Group {
    int kind;      // model * 100 + ndim * 10 + scheme
    ItemPack pack; // up to kPackItems grids of that kind
    int blocks;    // blocks of one fused stage launch over the pack
  };
  hj_status rebuild();
  hj_status sync_ctl();
  void drop_graphs();
  cudaError_t enqueue_round(long long R, cudaStream_t s);

  int device_;
  cudaStream_t stream_;
  int cap_;
  std::vector<Slot> slots_;
  hja::Allocator alloc_;  // serves the control arrays
  Ctl* dev_ctl_ = nullptr;
  Ctl* host_ctl_ = nullptr;  // pinned mirror
  int* dev_slots_ = nullptr;   // control slots of the current items, in launch order
  int item_cap_ = 0;
  int nitems_ = 0;
  std::vector<Group> groups_;
  bool dirty_ = true;
  std::vector<int> order_;  // slots in the current item list
  std::map<std::string, cudaGraphExec_t> graphs_;  // round shape -> graph
  cudaStream_t cap_stream_ = nullptr;
  // Group mode: one launch per RK stage over the blocks of every active
  // grid, with the kernels compiled for this composition (hj_group.cuh).
  // Until they are compiled the per-kind launches above run.
  bool group_allowed_ = false;
  bool group_mode_ = false;
  bool group_pending_ = false;  // a compile of the current composition is running
  void* group_handle_ = nullptr;
  GroupPack gpack_;
  unsigned gblocks_ = 0;
  std::vector<hjd::DevGrid> gcodes_;
  std::vector<int> gschemes_;
  std::vector<std::string> gkeys_;  // code keys of the kernels in group_handle_
  bool plan_group();
};

}  // namespace hjb
