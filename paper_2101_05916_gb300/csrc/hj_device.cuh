// hj_device.cuh -- per-grid-point device arithmetic of the HJ level-set solve
// (sm_103a, FP32).
//
// One time step advances dW/ds = H(x, grad W) (Eq. 2 of the paper, written
// for W = -V) by TVD-RK3.  The right-hand side at a node is the global
// Lax-Friedrichs numerical Hamiltonian
//
//     L(W) = H(x, (p- + p+)/2) + sum_i a_i (p+_i - p-_i) / 2,
//
// where p-/p+ are one-sided slopes (first-order, ENO2 or WENO5) and
// H(x, p) = max_u min_d p . f(x, u, d) is taken in closed form: each input
// enters one component of f linearly, so the optimal control and the
// worst-case disturbance sit at the ends of their intervals (bang-bang).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace hjd {

constexpr int MAXD = 4;
enum { M_DRIFT = 0, M_QUAD_Z = 1, M_QUAD_X4 = 2 };
enum { C_BOX = 0, C_BALL_OUT = 1 };

// Everything a kernel needs to know about one grid, passed by value.
struct DevGrid {
  int ndim;
  int n[MAXD];
  int stride[MAXD];    // row-major, last axis fastest
  int npts;
  int plane;           // nodes in the flattened last-two-axes plane (all nodes if ndim <= 2)
  float lo[MAXD];
  float h[MAXD];
  double lo_d[MAXD];   // the same box in double, for interpolation
  double h_d[MAXD];
  float ih[MAXD];      // 1 / h
  float ih6[MAXD];     // 1 / (6 h), folds the 1/6 of the WENO candidates
  float wfloor[MAXD];  // WENO epsilon floor on undivided differences: 1e-18 h^2
  int model;
  float prm[8];
  float dlo[MAXD], dhi[MAXD];
  int con_kind;
  unsigned con_mask;   // constrained axes of a box constraint
  float ca[MAXD], cb[MAXD];
  float alpha[MAXD];   // Lax-Friedrichs coefficients
  const float* tab;    // quad_x4: g * tan(th_j) per th index
};

// Arguments of one Runge-Kutta stage launch.
struct StageArgs {
  const float* src;    // field whose slopes are taken (W, W1 or W2)
  const float* base;   // W at the start of the step (stages 2 and 3)
  float* dst;          // W1, W2, or W itself (stage 3 updates W in place)
  float* snap;         // window snapshot (stage 3 with check)
  unsigned* resid;     // max |W - snap| as float bits (stage 3 with check)
  float dt;
  int check;
  int clamp;           // 0: min(W3, l); 1: min(W3, l, W)
  float band;          // > 0: residual only where min(|W|, |snap|) <= band
};

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------- geometry

// Margin l = -c to the constraint set: distance to the nearest face inside a
// box, minus the Euclidean distance outside it; or distance outside a ball.
template <int D>
__device__ __forceinline__ float margin(const DevGrid& g, const float (&x)[D]) {
  if (g.con_kind == C_BALL_OUT) {
    float s = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      float e = x[d] - g.ca[d];
      s = fmaf(e, e, s);
    }
    return sqrtf(s) - g.cb[0];
  }
  bool inside = true;
  float m = CUDART_INF_F, o2 = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    if (!((g.con_mask >> d) & 1u)) continue;
    float below = g.ca[d] - x[d], above = x[d] - g.cb[d];
    float e = fmaxf(fmaxf(below, above), 0.f);
    inside = inside && (e <= 0.f);
    o2 = fmaf(e, e, o2);
    m = fminf(m, fminf(x[d] - g.ca[d], g.cb[d] - x[d]));
  }
  return inside ? m : -sqrtf(o2);
}

// ------------------------------------------------------------- dynamics

// H(x, p) = max_u min_d p . f(x, u, d) in closed (bang-bang) form.
template <int M, int D>
__device__ __forceinline__ float hamiltonian(const DevGrid& g, const float (&x)[D],
                                             const int (&idx)[D], const float (&p)[D]) {
  if constexpr (M == M_QUAD_Z) {
    // f = (vz, kT u - g + d); prm = (kT, g, u_lo, u_hi)
    float a = p[1] * g.prm[0];
    float H = fmaf(p[0], x[1], -p[1] * g.prm[1]);
    H += fmaxf(a * g.prm[2], a * g.prm[3]);
    H += fminf(p[1] * g.dlo[0], p[1] * g.dhi[0]);
    return H;
  } else if constexpr (M == M_QUAD_X4) {
    // f = (v, g tan th, -d1 th + w, -d0 th + n0 u) + d e_axis
    // prm = (g, d1, d0, n0, u_lo, u_hi, axis)
    float gt = __ldg(g.tab + idx[2]);
    float a = p[3] * g.prm[3];
    float H = p[0] * x[1];
    H = fmaf(p[1], gt, H);
    H = fmaf(p[2], fmaf(-g.prm[1], x[2], x[3]), H);
    H = fmaf(-p[3] * g.prm[2], x[2], H);
    H += fmaxf(a * g.prm[4], a * g.prm[5]);
    float pa = (g.prm[6] != 0.f) ? p[1] : p[0];
    H += fminf(pa * g.dlo[0], pa * g.dhi[0]);
    return H;
  } else {
    // drift: f = d, one interval per axis
    float H = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) H += fminf(p[d] * g.dlo[d], p[d] * g.dhi[d]);
    return H;
  }
}

// Per-axis max over the input box vertices of |f_i(x, u, d)| at one node.
template <int M, int D>
__device__ __forceinline__ void abs_f_max(const DevGrid& g, const float (&x)[D],
                                          const int (&idx)[D], float (&m)[D]) {
  if constexpr (M == M_QUAD_Z) {
    m[0] = fmaxf(m[0], fabsf(x[1]));
    float kT = g.prm[0], gg = g.prm[1];
    float e = 0.f;
    e = fmaxf(e, fabsf(kT * g.prm[2] - gg + g.dlo[0]));
    e = fmaxf(e, fabsf(kT * g.prm[2] - gg + g.dhi[0]));
    e = fmaxf(e, fabsf(kT * g.prm[3] - gg + g.dlo[0]));
    e = fmaxf(e, fabsf(kT * g.prm[3] - gg + g.dhi[0]));
    m[1] = fmaxf(m[1], e);
  } else if constexpr (M == M_QUAD_X4) {
    float gt = __ldg(g.tab + idx[2]);
    bool ax1 = g.prm[6] != 0.f;
    float dl = g.dlo[0], dh = g.dhi[0];
    float f0 = ax1 ? fabsf(x[1]) : fmaxf(fabsf(x[1] + dl), fabsf(x[1] + dh));
    float f1 = ax1 ? fmaxf(fabsf(gt + dl), fabsf(gt + dh)) : fabsf(gt);
    float f2 = fabsf(fmaf(-g.prm[1], x[2], x[3]));
    float f3 = fmaxf(fabsf(fmaf(g.prm[3], g.prm[4], -g.prm[2] * x[2])),
                     fabsf(fmaf(g.prm[3], g.prm[5], -g.prm[2] * x[2])));
    m[0] = fmaxf(m[0], f0);
    m[1] = fmaxf(m[1], f1);
    m[2] = fmaxf(m[2], f2);
    m[3] = fmaxf(m[3], f3);
  } else {
#pragma unroll
    for (int d = 0; d < D; ++d) m[d] = fmaxf(m[d], fmaxf(fabsf(g.dlo[d]), fabsf(g.dhi[d])));
  }
}

// ---------------------------------------------------------- grid lines

// The 2R+1 values of the grid line through node p along one axis; ghost
// nodes beyond either end continue the line linearly through its two
// outermost nodes.
template <int R>
__device__ __forceinline__ void load_line(const float* __restrict__ src, int p, int stride, int i,
                                          int n, float (&v)[2 * R + 1]) {
  if (i >= R && i < n - R) {
#pragma unroll
    for (int k = -R; k <= R; ++k) v[k + R] = __ldg(src + p + k * stride);
    return;
  }
#pragma unroll
  for (int k = -R; k <= R; ++k) {
    int j = min(max(i + k, 0), n - 1);
    v[k + R] = __ldg(src + p + (j - i) * stride);
  }
  if (i < R) {
    float w0 = __ldg(src + p - i * stride);
    float s = w0 - __ldg(src + p + (1 - i) * stride);
#pragma unroll
    for (int k = -R; k <= R; ++k)
      if (i + k < 0) v[k + R] = fmaf((float)(-(i + k)), s, w0);
  }
  if (i > n - 1 - R) {
    float wn = __ldg(src + p + (n - 1 - i) * stride);
    float s = wn - __ldg(src + p + (n - 2 - i) * stride);
#pragma unroll
    for (int k = -R; k <= R; ++k)
      if (i + k > n - 1) v[k + R] = fmaf((float)(i + k - (n - 1)), s, wn);
  }
}

// ------------------------------------------------------------- slopes

// WENO5 of Jiang & Peng on undivided differences q1..q5 in upwind order.
// Returns 6 * h * slope (the caller multiplies by 1 / (6 h)).
//
// The nonlinear weights a_k = c_k / (S_k + eps)^2 are normalised, so any
// common factor cancels.  Multiplying every S_k + eps by 1 / eps and then
// every a_k by the product of all three squares gives weights
// c_1 s_2^2 s_3^2, c_2 s_1^2 s_3^2, c_3 s_1^2 s_2^2 with s_k = S_k / eps + 1.
// Since S_k <= 34 max q^2 and eps >= 1e-6 max q^2, every s_k lies in
// [1, 3.4e7], so these products stay inside FP32 range.  The rewrite needs
// two reciprocals instead of four.
__device__ __forceinline__ float weno5_6h(float q1, float q2, float q3, float q4, float q5,
                                          float floor_) {
  const float k1312 = 13.f / 12.f;
  float t1 = fmaf(-2.f, q2, q1 + q3);
  float u1 = fmaf(3.f, q3, fmaf(-4.f, q2, q1));
  float t2 = fmaf(-2.f, q3, q2 + q4);
  float u2 = q2 - q4;
  float t3 = fmaf(-2.f, q4, q3 + q5);
  float u3 = fmaf(3.f, q3, fmaf(-4.f, q4, q5));
  float S1 = fmaf(k1312 * t1, t1, 0.25f * u1 * u1);
  float S2 = fmaf(k1312 * t2, t2, 0.25f * u2 * u2);
  float S3 = fmaf(k1312 * t3, t3, 0.25f * u3 * u3);
  float m = fmaxf(fmaxf(fmaxf(fabsf(q1), fabsf(q2)), fmaxf(fabsf(q3), fabsf(q4))), fabsf(q5));
  float ie = rcp_approx(fmaf(1e-6f * m, m, floor_));
  float s1 = fmaf(S1, ie, 1.f), s2 = fmaf(S2, ie, 1.f), s3 = fmaf(S3, ie, 1.f);
  float a1 = s1 * s1, a2 = s2 * s2, a3 = s3 * s3;
  float w1 = 0.1f * (a2 * a3), w2 = 0.6f * (a1 * a3), w3 = 0.3f * (a1 * a2);
  float phi1 = fmaf(2.f, q1, fmaf(-7.f, q2, 11.f * q3));
  float phi2 = fmaf(5.f, q3, fmaf(2.f, q4, -q2));
  float phi3 = fmaf(2.f, q3, fmaf(5.f, q4, -q5));
  float num = fmaf(w1, phi1, fmaf(w2, phi2, w3 * phi3));
  return num * rcp_approx(w1 + w2 + w3);
}

template <int S>
struct Slopes;

template <>
struct Slopes<1> {
  static constexpr int R = 1;
  __device__ __forceinline__ static void eval(const float (&v)[3], const DevGrid& g, int d,
                                              float& pm, float& pp) {
    pm = (v[1] - v[0]) * g.ih[d];
    pp = (v[2] - v[1]) * g.ih[d];
  }
};

// ENO2: first difference plus half the smaller (in magnitude) of the two
// adjacent second differences; ties take the left one.
template <>
struct Slopes<2> {
  static constexpr int R = 2;
  __device__ __forceinline__ static void eval(const float (&v)[5], const DevGrid& g, int d,
                                              float& pm, float& pp) {
    float a = fmaf(-2.f, v[1], v[2] + v[0]);
    float b = fmaf(-2.f, v[2], v[3] + v[1]);
    float c = fmaf(-2.f, v[3], v[4] + v[2]);
    float m1 = (fabsf(a) <= fabsf(b)) ? a : b;
    float m2 = (fabsf(b) <= fabsf(c)) ? b : c;
    pm = fmaf(0.5f, m1, v[2] - v[1]) * g.ih[d];
    pp = fmaf(-0.5f, m2, v[3] - v[2]) * g.ih[d];
  }
};

template <>
struct Slopes<5> {
  static constexpr int R = 3;
  __device__ __forceinline__ static void eval(const float (&v)[7], const DevGrid& g, int d,
                                              float& pm, float& pp) {
    float D0 = v[1] - v[0], D1 = v[2] - v[1], D2 = v[3] - v[2];
    float D3 = v[4] - v[3], D4 = v[5] - v[4], D5 = v[6] - v[5];
    float f = g.wfloor[d];
    pm = weno5_6h(D0, D1, D2, D3, D4, f) * g.ih6[d];
    pp = weno5_6h(D5, D4, D3, D2, D1, f) * g.ih6[d];
  }
};

// L(src) at node p with multi-index idx; also returns src[p] in `center`.
template <int D, int S, int M>
__device__ __forceinline__ float lf_rhs(const DevGrid& g, const float* __restrict__ src, int p,
                                        const int (&idx)[D], const float (&x)[D], float& center) {
  constexpr int R = Slopes<S>::R;
  float pbar[D];
  float diss = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    float v[2 * R + 1];
    load_line<R>(src, p, g.stride[d], idx[d], g.n[d], v);
    if (d == 0) center = v[R];
    float pm, pp;
    Slopes<S>::eval(v, g, d, pm, pp);
    pbar[d] = 0.5f * (pm + pp);
    diss = fmaf(0.5f * g.alpha[d], pp - pm, diss);
  }
  return hamiltonian<M, D>(g, x, idx, pbar) + diss;
}

// Maximum of non-negative float bit patterns across the block, then one
// atomicMax into *out.  Works on bits so that NaN and +inf are kept (they
// compare above every finite value).
__device__ __forceinline__ void block_max_bits(unsigned v, unsigned* out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ unsigned warp_max[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_max[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int nw = (blockDim.x + 31) >> 5;
    v = (lane < nw) ? warp_max[lane] : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0 && v) atomicMax(out, v);
  }
}

}  // namespace hjd
