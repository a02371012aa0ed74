// hj_group.cuh -- device-side structures of batched stepping: the per-grid
// control state, and the pack of a group launch (one launch per RK stage
// over the blocks of every active grid of a batch, whatever its kind).
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
  int check_next;     // 1 when the next step closes a window (or reaches the cap)
};

// One position of a group launch: a grid with bx blocks of kGroupThreads
// nodes per slab of the flat mapping (slabs: the first axis of a 4-D grid,
// else one).  The group kernel holds one body per position, compiled for
// that grid's kind, shape and model constants; a block finds its position
// by comparing its index with the positions' first blocks, and each body
// reads its position's fields with literal indices (constant-bank operands,
// as in the single-grid kernel).  A position without a grid has no blocks:
// its first block equals its successor's.
struct GroupItem {
  hjd::DevGrid g;
  hjd::StageArgs a[3];  // stage 1..3 arguments (check and resid are set on the device)
  int slot;             // index into the control array
  int bx;
  unsigned bx_m;        // bx as a multiply-shift reciprocal (hjd::fast_div), bx >= 2
  int bx_s;
};

constexpr int kGroupItems = 16;
constexpr int kGroupThreads = 256;
struct GroupPack {
  int count;
  int block_begin[kGroupItems + 1];
  GroupItem items[kGroupItems];
};

}  // namespace hjb
