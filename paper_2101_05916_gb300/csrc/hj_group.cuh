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

// One position of a group launch: a grid with bx blocks of kGroupThreads
// nodes per slab of the flat mapping (slabs: the first axis of a 4-D grid,
// else one).  The group kernel holds one body per position, compiled for
// that grid's kind, shape and model constants.  A position without a grid
// has bx = 0 (no blocks).
struct GroupItem {
  hjd::DevGrid g;
  hjd::StageArgs a[3];  // stage 1..3 arguments (check and resid are set on the device)
  int slot;             // index into the control array
  int bx;
};

constexpr int kGroupItems = 16;
constexpr int kGroupThreads = 256;
struct GroupPack {
  int count;
  int block_begin[kGroupItems + 1];
  GroupItem items[kGroupItems];
};

// The block's position in a group launch: its index k (binary search over
// the block offsets; positions without blocks are never found), its block
// (bx, yb) in that grid's flat mapping, its control slot, and whether this
// stage-3 launch closes the grid's window.  -1 when the grid no longer
// steps (the whole block returns).  The kernel then reads the descriptor
// and stage arguments of position k with a literal index, so that they
// stay constant-bank operands as in the single-grid kernel.
template <int STAGE>
__device__ __forceinline__ int group_locate(const GroupPack& pack, const Ctl* ctl, int& bx,
                                            int& yb, bool& check, int& slot) {
  int lo = 0, hi = pack.count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (pack.block_begin[mid] <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  slot = pack.items[lo].slot;
  const Ctl& c = ctl[slot];
  if (!c.active) return -1;
  int per = pack.items[lo].bx;
  int lb = (int)blockIdx.x - pack.block_begin[lo];
  yb = lb / per;
  bx = lb - yb * per;
  check = false;
  if (STAGE == 3) {
    long long s1 = c.steps + 1;
    check = (s1 % c.per == 0) || (s1 >= c.max_steps);
  }
  return lo;
}

}  // namespace hjb
