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

// Stage STAGE of one TVD-RK3 step at the node of (q, yb):
//   1: W1 = W + dt L(W)
//   2: W2 = 3/4 W + 1/4 (W1 + dt L(W1))
//   3: W3 = 1/3 W + 2/3 (W2 + dt L(W2)),  W <- min(W3, l)  [, W_prev]
// Returns the window-residual contribution |W_new - snap| as float bits
// (stage 3 with check; 0 otherwise).
template <int D, int S, int M, int STAGE>
__device__ __forceinline__ unsigned stage_point(const DevGrid& g, const StageArgs& a, int q, int yb,
                                                bool check) {
  int idx[D];
  int p;
  if (!node_of<D>(g, q, yb, idx, p)) return 0u;
  float x[D];
  coords<D>(g, idx, x);
  float c;
  float L = lf_rhs<D, S, M>(g, a.src, p, idx, x, c);
  float stepped = fmaf(a.dt, L, c);
  if constexpr (STAGE == 1) {
    a.dst[p] = stepped;
    return 0u;
  } else if constexpr (STAGE == 2) {
    float w = a.base[p];
    a.dst[p] = fmaf(0.75f, w, 0.25f * stepped);
    return 0u;
  } else {
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
    if (a.band > 0.f && fminf(fabsf(wn), fabsf(sv)) > a.band) r = 0.f;
    if (a.margin > 0) {
      // only faces of unconstrained axes: on a constrained axis the margin l
      // decides the value next to the face
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (!((g.con_kind == C_BOX) && ((g.con_mask >> d) & 1u)) &&
            (idx[d] < a.margin || idx[d] > g.n[d] - 1 - a.margin))
          r = 0.f;
    }
    if (wn != wn) r = wn;  // NaN always reaches the stop test
    return __float_as_uint(r);
  }
}

}  // namespace hjd
