// hj_group.cuh -- device-side structures of batched stepping: the per-grid
// control state, and the pack of a group launch (one launch per RK stage
// over the row tiles of every active grid of a batch, whatever its kind).
#pragma once

#include "hj_stage.cuh"

namespace hjb {

// Per-grid stepping state, written only by the control kernel between steps.
struct Ctl {
  int active;         // 1 while the grid is stepping
  int status;         // 0 running, 1 converged, 2 step cap, 3 non-finite, 4 cancelled
  long long per;      // steps per check window
  long long steps;    // steps done
  long long max_steps;
  long long windows;
  double tol;         // stop when the window residual drops below (negative: never)
  unsigned resid;     // running window residual (float bits)
  float last_resid;
};

// One grid of a group launch: bx blocks of kGroupThreads nodes per slab of
// the flat mapping (by slabs: the first axis of a 4-D grid, else one);
// `code` selects the body of the group kernel compiled for its kind, shape
// and model constants.
struct GroupItem {
  hjd::DevGrid g;
  hjd::StageArgs a[3];  // stage 1..3 arguments (check and resid are set on the device)
  int slot;             // index into the control array
  int code;
  int bx;
};

constexpr int kGroupItems = 16;
constexpr int kGroupThreads = 256;
struct GroupPack {
  int count;
  int block_begin[kGroupItems + 1];
  GroupItem items[kGroupItems];
};

// The block's item of a group launch: its index (binary search over the
// block offsets), its block (bx, yb) in the item's flat mapping, and its
// stage arguments with the window check of stage 3 decided from the control
// state.  -1 when the grid no longer steps (the whole block returns).
template <int STAGE>
__device__ __forceinline__ int group_find(const GroupPack& pack, Ctl* ctl, hjd::StageArgs& a,
                                          int& bx, int& yb, bool& check) {
  int lo = 0, hi = pack.count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pack.block_begin[mid] <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const GroupItem& it = pack.items[lo];
  const Ctl& c = ctl[it.slot];
  if (!c.active) return -1;
  int lb = (int)blockIdx.x - pack.block_begin[lo];
  yb = lb / it.bx;
  bx = lb - yb * it.bx;
  a = it.a[STAGE - 1];
  check = false;
  if (STAGE == 3) {
    long long s1 = c.steps + 1;
    check = (s1 % c.per == 0) || (s1 >= c.max_steps);
    a.check = check ? 1 : 0;
    a.resid = &ctl[it.slot].resid;
  }
  return lo;
}

}  // namespace hjb
