// hj_stage.cuh -- one TVD-RK3 stage at one grid node, shared by the
// single-grid kernel and the fused multi-grid (batched) kernel.
#pragma once

#include "hj_device.cuh"

namespace hjd {

// Node handled by thread index q of slab yb.  A 4-D grid runs one slab per
// value of its first axis (yb), and q walks the other three axes.  A grid
// with ndim <= 3 is one slab (yb = 0) holding every node.  Flattening three
// axes keeps warps full whatever the axis lengths.  The divisions use
// precomputed multiply-shift reciprocals.
template <int D>
__device__ __forceinline__ bool node_of(const DevGrid& g, int q, int yb, int (&idx)[D], int& p) {
  if constexpr (D == 1) {
    idx[0] = q;
    p = q;
  } else {
    int a = fast_div(q, g.div_m[0], g.div_s[0]);
    idx[D - 1] = q - a * g.n[D - 1];
    if constexpr (D == 2) {
      idx[0] = a;
    } else {
      int b = fast_div(a, g.div_m[1], g.div_s[1]);
      idx[D - 2] = a - b * g.n[D - 2];
      idx[D - 3] = b;
    }
    p = q;
    if constexpr (D == 4) {
      idx[0] = yb;
      p += yb * g.stride[0];
    }
  }
  return q < g.plane;
}

template <int D>
__device__ __forceinline__ void coords(const DevGrid& g, const int (&idx)[D], float (&x)[D]) {
#pragma unroll
  for (int d = 0; d < D; ++d) x[d] = fmaf((float)idx[d], g.h[d], g.lo[d]);
}

// Stage STAGE of one TVD-RK3 step at node p with multi-index idx:
//   1: W1 = W + dt L(W)
//   2: W2 = 3/4 W + 1/4 (W1 + dt L(W1))
//   3: W3 = 1/3 W + 2/3 (W2 + dt L(W2)),  W <- min(W3, l)  [, W_prev]
// fast: the node's fastest-axis line in shared memory (see lf_rhs), or null.
// Returns the window-residual contribution |W_new - snap| as float bits
// (stage 3 with check; 0 otherwise).  LOCAL compiles in what a localized
// solve needs (frozen slabs, the slab residual in *raw, mid-window checks);
// plain solves run without it.
template <int D, int S, int M, int STAGE, bool LOCAL = false>
__device__ __forceinline__ unsigned stage_node(const DevGrid& g, const StageArgs& a,
                                               const int (&idx)[D], int p, bool check,
                                               const float* fast, unsigned* raw = nullptr) {
  float x[D];
  coords<D>(g, idx, x);
  float c;
  float L = lf_rhs<D, S, M>(g, a.src, p, idx, x, c, fast);
  float stepped = fmaf(a.dt, L, c);
  if constexpr (STAGE == 1) {
    a.dst[p] = stepped;
    return 0u;
  } else if constexpr (STAGE == 2) {
    float w = a.base[p];
    a.dst[p] = fmaf(0.75f, w, 0.25f * stepped);
    return 0u;
  } else {
    // a frozen slab of a localized solve keeps W and its snapshot
    if constexpr (LOCAL) {
      if (a.live && !a.live[slab_of<D>(g, idx)]) return 0u;
    }
    float w = a.base[p];
    float w3 = fmaf(1.f / 3.f, w, (2.f / 3.f) * stepped);
    float wn = fminf(w3, margin<D>(g, x, p));
    if (a.clamp) wn = fminf(wn, w);
    if (w3 != w3) wn = w3;  // keep a NaN visible to the stop test
    a.dst[p] = wn;
    if (!check) return 0u;
    float sv = a.snap[p];
    float r = fabsf(wn - sv);
    a.snap[p] = wn;
    if (a.margin > 0) {
      // only faces of unconstrained axes: on a constrained axis the margin l
      // decides the value next to the face
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (!((g.con_kind == C_BOX) && ((g.con_mask >> d) & 1u)) &&
            (idx[d] < a.margin || idx[d] > g.n[d] - 1 - a.margin))
          r = 0.f;
    }
    // the slab residual of a localized solve: every node away from the
    // faces the margin excludes, inside the band or not
    if constexpr (LOCAL) {
      if (raw) *raw = __float_as_uint(r);
    }
    if (a.band > 0.f && fminf(fabsf(wn), fabsf(sv)) > a.band) r = 0.f;
    if (wn != wn) r = wn;  // NaN always reaches the stop test
    return __float_as_uint(r);
  }
}

// The flat mapping: thread q of slab yb, one node per thread.
template <int D, int S, int M, int STAGE>
__device__ __forceinline__ unsigned stage_point(const DevGrid& g, const StageArgs& a, int q, int yb,
                                                bool check) {
  int idx[D];
  int p;
  if (!node_of<D>(g, q, yb, idx, p)) return 0u;
  return stage_node<D, S, M, STAGE>(g, a, idx, p, check, nullptr);
}

// What one thread's node gives back to its block: the stop-test residual
// bits (band and margin rules applied), the node's change for its slab's
// residual, and its slab (-1 for a thread without a node).
struct NodeOut {
  unsigned resid;
  unsigned raw;
  int slab;
};

// Per-slab maximum of v into out[slab], one atomic per run of lanes that
// share a slab (slab < 0: no node).  Every lane of the warp must call it.
__device__ __forceinline__ void slab_max_bits(int slab, unsigned v, unsigned* out) {
  unsigned m = __match_any_sync(0xffffffffu, slab);
  unsigned w = __reduce_max_sync(m, v);
  if (slab >= 0 && w && (int)(threadIdx.x & 31) == __ffs(m) - 1) atomicMax(out + slab, w);
}

// Blocks of the flat mapping per slab yb.
__device__ __forceinline__ int flat_blocks_per_slab(const DevGrid& g) {
  return (g.plane + (int)blockDim.x - 1) / (int)blockDim.x;
}

// Body of a flat stage kernel.  Block (x, y) covers nodes x * blockDim ..
// of slab y; stage 3 with check folds the stop-test residual of the block
// into *a.resid.  The LOCAL variant (localized solves) also takes a tile
// list, where block b runs flat tile tiles[b] = y * (blocks per slab) + x,
// and folds every node's change into its slab's entry of a.slab_resid.
template <int D, int S, int M, int STAGE, bool LOCAL>
__device__ __forceinline__ void flat_body(const DevGrid& g, const StageArgs& a) {
  if constexpr (!LOCAL) {
    unsigned r = stage_point<D, S, M, STAGE>(g, a, blockIdx.x * blockDim.x + threadIdx.x,
                                             blockIdx.y, a.check != 0);
    if constexpr (STAGE == 3) {
      if (a.check) block_max_bits(r, a.resid);
    }
    return;
  }
  int bx = (int)blockIdx.x, yb = (int)blockIdx.y;
  if (a.tiles) {
    int t = a.tiles[blockIdx.x];
    int per = flat_blocks_per_slab(g);
    yb = t / per;
    bx = t - yb * per;
  }
  NodeOut o{0u, 0u, -1};
  int idx[D];
  int p;
  if (node_of<D>(g, bx * (int)blockDim.x + (int)threadIdx.x, yb, idx, p)) {
    o.slab = slab_of<D>(g, idx);
    o.resid = stage_node<D, S, M, STAGE, true>(g, a, idx, p, a.check != 0, nullptr, &o.raw);
  }
  if constexpr (STAGE == 3) {
    if (a.check) {
      if (a.slab_resid) slab_max_bits(o.slab, o.raw, a.slab_resid);
      block_max_bits(o.resid, a.resid);
    }
  }
}

// Shared-memory floats of one row tile: tile_rows rows of n + 2 R values.
template <int S>
__host__ __device__ constexpr int tile_row_pitch(int n) {
  return n + 2 * Slopes<S>::R;
}

// The row-tile mapping.  Block `tile` owns the g.tile_rows consecutive lines
// along the fastest axis starting at line tile * g.tile_rows (the last tile
// may hold fewer).  These lines are one contiguous run of nodes in memory.
//   1. The run is staged in shared memory with 16-byte loads over its
//      16-byte-aligned cover (fields start 16-byte aligned and carry guard
//      floats, so the cover never leaves the allocation), each line padded
//      by R values on both sides: the linear continuation of the line
//      through its two outermost nodes.  The differences that reach into
//      the padding are replaced by the end rule (edge_diffs), as in the
//      flat mapping, so the padding only keeps every shared-memory read
//      defined.
//   2. Thread t < (lines in the tile) * n then computes node t of the run;
//      its fastest-axis stencil reads the staged line, the other axes read
//      global memory as in the flat mapping.
// sm holds g.tile_rows * tile_row_pitch<S>(n) floats.  All threads of the
// block must call this (it synchronises the block once).
struct TileOut {
  unsigned resid;  // stop-test residual bits of the node (band and margin rules applied)
  unsigned raw;    // |W - snap| bits of the node, for the slab residual
  int slab;        // the node's slab, -1 for a thread without a node
};

template <int D, int S, int M, int STAGE>
__device__ __forceinline__ TileOut stage_tile(const DevGrid& g, const StageArgs& a, int tile,
                                              bool check, float* sm) {
  constexpr int R = Slopes<S>::R;
  TileOut out{0u, 0u, -1};
  const int n = g.n[D - 1];
  const int P = tile_row_pitch<S>(n);
  const int row0 = tile * g.tile_rows;
  const int nr = min(g.tile_rows, g.nrows - row0);
  const int base = row0 * n;
  const int len = nr * n;
  const int a0 = base & ~3;
  const int nvec = (base + len - a0 + 3) >> 2;
  const float4* src4 = reinterpret_cast<const float4*>(a.src + a0);
  for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
    float4 q4 = __ldg(src4 + v);
    const float e[4] = {q4.x, q4.y, q4.z, q4.w};
    int k = a0 - base + 4 * v;  // run-local index of q4.x (>= -3)
    int r = (k >= 0) ? fast_div(k, g.div_m[0], g.div_s[0]) : -1;
    int c = k - r * n;          // in [0, n) for k >= 0; k + n for k < 0
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (k + j >= 0 && k + j < len) sm[r * P + R + c] = e[j];
      if (++c == n) {
        c = 0;
        ++r;
      }
    }
  }
  for (int t = threadIdx.x; t < nr * 2 * R; t += blockDim.x) {
    int r = t / (2 * R), j = t - r * (2 * R);
    const float* row = a.src + base + r * n;
    if (j < R) {
      float w0 = __ldg(row), w1 = __ldg(row + 1);
      sm[r * P + j] = fmaf((float)(R - j), w0 - w1, w0);
    } else {
      float wn = __ldg(row + (n - 1)), wm = __ldg(row + (n - 2));
      sm[r * P + R + n + (j - R)] = fmaf((float)(j - R + 1), wn - wm, wn);
    }
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t >= len) return out;
  const int r = fast_div(t, g.div_m[0], g.div_s[0]);
  int idx[D];
  idx[D - 1] = t - r * n;
  if constexpr (D >= 2) {
    int line = row0 + r;
    if constexpr (D == 2) {
      idx[0] = line;
    } else {
      int a1 = fast_div(line, g.div_m[1], g.div_s[1]);
      idx[D - 2] = line - a1 * g.n[D - 2];
      if constexpr (D == 3) {
        idx[0] = a1;
      } else {
        int a2 = fast_div(a1, g.div_m[2], g.div_s[2]);
        idx[1] = a1 - a2 * g.n[1];
        idx[0] = a2;
      }
    }
  }
  out.slab = slab_of<D>(g, idx);
  out.resid = stage_node<D, S, M, STAGE, true>(g, a, idx, base + t, check,
                                               sm + r * P + R + idx[D - 1],
                                         &out.raw);
  return out;
}

// Body of a row-tile stage kernel: the block's tile comes from the tile list
// when there is one; stage 3 with check folds the stop-test residual of the
// block into *a.resid and, in a localized solve, every node's change into
// its slab's entry of a.slab_resid.
template <int D, int S, int M, int STAGE>
__device__ __forceinline__ void tile_body(const DevGrid& g, const StageArgs& a, float* sm) {
  int tile = a.tiles ? a.tiles[blockIdx.x] : (int)blockIdx.x;
  TileOut o = stage_tile<D, S, M, STAGE>(g, a, tile, a.check != 0, sm);
  if constexpr (STAGE == 3) {
    if (a.check) {
      if (a.slab_resid) slab_max_bits(o.slab, o.raw, a.slab_resid);
      block_max_bits(o.resid, a.resid);
    }
  }
}

}  // namespace hjd
