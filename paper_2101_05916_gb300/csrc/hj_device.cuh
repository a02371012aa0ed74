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

#ifdef __CUDACC_RTC__
// compiled at run time (shape-specialised stage kernels): no host headers
#define CUDART_INF_F __int_as_float(0x7f800000)
#else
#include <cuda_runtime.h>
#include <math_constants.h>
#endif

namespace hjd {

constexpr int MAXD = 4;
enum { M_DRIFT = 0, M_QUAD_Z = 1, M_QUAD_X4 = 2 };
enum { C_BOX = 0, C_BALL_OUT = 1, C_FIELD = 2 };

// Everything a kernel needs to know about one grid, passed by value.
struct DevGrid {
  int ndim;
  int n[MAXD];
  int stride[MAXD];    // row-major, last axis fastest
  int npts;
  int plane;           // nodes of one thread slab: all axes but the first of a 4-D grid,
                       // every node of a grid with ndim <= 3
  unsigned div_m[3];   // n[ndim-1], n[ndim-2], n[ndim-3] as multiply-shift reciprocals
  int div_s[3];
  int nrows;           // lines along the fastest axis: npts / n[ndim-1]
  int tile_rows;       // > 0: row-tile kernels, this many fastest-axis lines per block;
                       // 0: one node per thread over flattened slabs
  float lo[MAXD];
  float h[MAXD];
  double lo_d[MAXD];   // the same box in double, for interpolation
  double h_d[MAXD];
  double ih_d[MAXD];   // 1 / h in double
  double ih2_d[MAXD];  // 1 / (2 h) in double
  float ih[MAXD];      // 1 / h
  float hih[MAXD];     // 0.5 / h
  float haih[MAXD];    // 0.5 a / h
  float wfloor[MAXD];  // WENO epsilon floor on undivided differences: 1e-18 h^2, times 3/4
  int model;
  float prm[8];
  float dlo[MAXD], dhi[MAXD];
  int con_kind;
  unsigned con_mask;   // constrained axes of a box constraint
  float ca[MAXD], cb[MAXD];
  float alpha[MAXD];   // Lax-Friedrichs coefficients
  const float* tab;    // quad_x4: g * tan(th_j) per th index
  const float* dflo;   // state-dependent disturbance box, input-major nd x npts
  const float* dfhi;   // (nullptr: the uniform box dlo/dhi)
  const float* lfield; // C_FIELD: the margin l at every node
};

// Arguments of one Runge-Kutta stage launch.
struct StageArgs {
  const float* src;    // field whose slopes are taken (W, W1 or W2)
  const float* base;   // W at the start of the step (stages 2 and 3)
  float* dst;          // W1, W2, or W itself (stage 3 updates W in place)
  float* snap;         // window snapshot (stage 3 with check)
  unsigned* resid;     // max |W - snap| as float bits (stage 3 with check)
  float dt;
  int check;           // stage 3: fold the window residual, move the snapshot on
  int clamp;           // 0: min(W3, l); 1: min(W3, l, W)
  float band;          // > 0: residual only where min(|W|, |snap|) <= band
  int margin;          // residual only at nodes >= margin cells from every face
  // Localized stepping (row-tile kernels only; all null in a plain solve):
  const int* tiles;          // block b runs row tile tiles[b] (null: tile b)
  int ntiles;                // entries of tiles (host side: the launch's block count)
  const unsigned char* live; // stage 3: nonzero where the node's slab steps (null: all)
  unsigned* slab_resid;      // stage 3 with check: per-slab max |W - snap| over every
                             // node, as float bits (null: not kept)
};

// Slabs of a grid, the units of localized stepping: the lines of the two
// slowest axes of a 4-D grid (index i0 n1 + i1), the first axis of a 2-D or
// 3-D grid, the whole of a 1-D grid.  A slab spans every node of the axes it
// leaves free.
template <int D>
__device__ __forceinline__ int slab_of(const DevGrid& g, const int (&idx)[D]) {
  if constexpr (D == 4) return idx[0] * g.n[1] + idx[1];
  else if constexpr (D >= 2) return idx[0];
  else return 0;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Quotient of q < 2^31 by the divisor encoded as (m, s) with s = ceil(log2 d) - 1
// and m = ceil(2^(31 + s + 1) / d): floor(q m / 2^(32 + s)).  For divisors
// d >= 2 the rounding error q (m - 2^(32+s)/d) / 2^(32+s) < 1/d never crosses
// an integer.
__device__ __forceinline__ int fast_div(int q, unsigned m, int s) {
  return (int)(__umulhi((unsigned)q, m) >> s);
}

// The (m, s) of a divisor d >= 2 for fast_div.
__host__ __device__ inline void div_consts(unsigned d, unsigned& m, int& s) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  unsigned long long num = 1ull << (31 + l);
  m = (unsigned)((num + d - 1) / d);
  s = l - 1;
}

// ---------------------------------------------------------------- geometry

// Margin l = -c to the constraint set at node p, coordinates x: distance to
// the nearest face inside a box, minus the Euclidean distance outside it;
// distance outside a ball; or the caller's value at the node.
template <int D>
__device__ __forceinline__ float margin(const DevGrid& g, const float (&x)[D], int p) {
  if (g.con_kind == C_FIELD) return __ldg(g.lfield + p);
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
// Disturbance interval of input j at node `node`: the state-dependent field
// when one is set (a GP confidence band, Sec. II-C), else the uniform box.
__device__ __forceinline__ void dist_box(const DevGrid& g, int j, int node, float& lo, float& hi) {
  if (g.dflo) {
    lo = __ldg(g.dflo + (long long)j * g.npts + node);
    hi = __ldg(g.dfhi + (long long)j * g.npts + node);
  } else {
    lo = g.dlo[j];
    hi = g.dhi[j];
  }
}

template <int M, int D>
__device__ __forceinline__ float hamiltonian(const DevGrid& g, const float (&x)[D],
                                             const int (&idx)[D], const float (&p)[D], int node) {
  if constexpr (M == M_QUAD_Z) {
    // f = (vz, kT u - g + d); prm = (kT, g, u_lo, u_hi)
    float a = p[1] * g.prm[0];
    float H = fmaf(p[0], x[1], -p[1] * g.prm[1]);
    H += fmaxf(a * g.prm[2], a * g.prm[3]);
    float dl, dh;
    dist_box(g, 0, node, dl, dh);
    H += fminf(p[1] * dl, p[1] * dh);
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
    float dl, dh;
    dist_box(g, 0, node, dl, dh);
    H += fminf(pa * dl, pa * dh);
    return H;
  } else {
    // drift: f = d, one interval per axis
    float H = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      float dl, dh;
      dist_box(g, d, node, dl, dh);
      H += fminf(p[d] * dl, p[d] * dh);
    }
    return H;
  }
}

// Per-axis max over the input box vertices of |f_i(x, u, d)| at one node.
template <int M, int D>
__device__ __forceinline__ void abs_f_max(const DevGrid& g, const float (&x)[D],
                                          const int (&idx)[D], float (&m)[D], int node) {
  if constexpr (M == M_QUAD_Z) {
    m[0] = fmaxf(m[0], fabsf(x[1]));
    float kT = g.prm[0], gg = g.prm[1];
    float dl, dh;
    dist_box(g, 0, node, dl, dh);
    float e = 0.f;
    e = fmaxf(e, fabsf(kT * g.prm[2] - gg + dl));
    e = fmaxf(e, fabsf(kT * g.prm[2] - gg + dh));
    e = fmaxf(e, fabsf(kT * g.prm[3] - gg + dl));
    e = fmaxf(e, fabsf(kT * g.prm[3] - gg + dh));
    m[1] = fmaxf(m[1], e);
  } else if constexpr (M == M_QUAD_X4) {
    float gt = __ldg(g.tab + idx[2]);
    bool ax1 = g.prm[6] != 0.f;
    float dl, dh;
    dist_box(g, 0, node, dl, dh);
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
    for (int d = 0; d < D; ++d) {
      float dl, dh;
      dist_box(g, d, node, dl, dh);
      m[d] = fmaxf(m[d], fmaxf(fabsf(dl), fabsf(dh)));
    }
  }
}

// ------------------------------------------------------- interpolation

// Coarse cell and fractional offset of coordinate xv along axis d of grid c.
__device__ __forceinline__ bool locate(const DevGrid& c, int d, double xv, int& i0, double& fr) {
  double t = (xv - c.lo_d[d]) * c.ih_d[d];
  double tol = 1e-9;
  if (t < -tol || t > (double)(c.n[d] - 1) + tol) return false;
  int i = (int)floor(t);
  i = min(max(i, 0), c.n[d] - 2);
  double f = t - (double)i;
  fr = fmin(fmax(f, 0.0), 1.0);
  i0 = i;
  return true;
}

// Twice the node gradient along axis d, times h: the central difference
// inside, twice the one-sided difference at the ends.  Times 1 / (2 h) it is
// the node gradient.
template <int D>
__device__ __forceinline__ double node_diff2(const DevGrid& g, const float* W, int off, int i,
                                             int d) {
  int s = g.stride[d];
  if (i == 0) return 2.0 * ((double)W[off + s] - (double)W[off]);
  if (i == g.n[d] - 1) return 2.0 * ((double)W[off] - (double)W[off - s]);
  return (double)W[off + s] - (double)W[off - s];
}

// ---------------------------------------------------------- grid lines

// A grid line around node i (of n along one axis) is handled as its 2R
// first differences Dk[k] = W(i + k - R + 1) - W(i + k - R), k = 0 .. 2R-1.
// Ghost nodes beyond either end continue the line linearly through its two
// outermost nodes, so every difference that reaches past an end equals the
// line's edge difference there: W(1) - W(0) at the start, W(n-1) - W(n-2)
// at the end.
//
// edge_diffs applies that rule to differences that are right wherever both
// nodes of a slot lie on the line (whatever they hold elsewhere).  The
// start's edge difference sits in slot R - i when i < R, the end's in slot
// R - 1 + (n-1-i) when n-1-i < R; both are read before any slot is
// replaced.  Selects, not branches: lanes away from the ends keep every
// slot.  n >= 2 keeps the two replaced ranges apart.
template <int R>
__host__ __device__ __forceinline__ void edge_diffs(float (&Dk)[2 * R], int i, int n) {
  const int r = n - 1 - i;
  float dl = Dk[R], dr = Dk[R - 1];
#pragma unroll
  for (int j = 1; j < R; ++j) {
    dl = (i == j) ? Dk[R - j] : dl;
    dr = (r == j) ? Dk[R - 1 + j] : dr;
  }
#pragma unroll
  for (int k = 0; k < R; ++k) Dk[k] = (k + i < R) ? dl : Dk[k];
#pragma unroll
  for (int k = R; k < 2 * R; ++k) Dk[k] = (k - r >= R) ? dr : Dk[k];
}

template <int R>
__host__ __device__ __forceinline__ void diffs_of(const float (&v)[2 * R + 1], float (&Dk)[2 * R]) {
#pragma unroll
  for (int k = 0; k < 2 * R; ++k) Dk[k] = v[k + 1] - v[k];
}

// The differences of the line through node p along an axis of stride
// `stride` (a slower axis).  Nodes R or more from both ends load their
// 2R+1 values at offsets that are the same for the whole warp; the others
// load with the index clamped to the line (so every address stays inside
// the field) and replace the differences past an end.
template <int R>
__device__ __forceinline__ void line_diffs(const float* __restrict__ src, int p, int stride, int i,
                                           int n, float (&Dk)[2 * R]) {
  float v[2 * R + 1];
  if (i >= R && i < n - R) {
    // one per-thread base address plus offsets that are the same for the
    // whole warp: 64-bit integer adds instead of a multiply-add per load
    const char* c = reinterpret_cast<const char*>(src + p);
    const long long sb = (long long)stride * (long long)sizeof(float);
#pragma unroll
    for (int k = -R; k <= R; ++k) v[k + R] = __ldg(reinterpret_cast<const float*>(c + k * sb));
    diffs_of<R>(v, Dk);
    return;
  }
#pragma unroll
  for (int k = -R; k <= R; ++k) {
    int j = min(max(i + k, 0), n - 1);
    v[k + R] = __ldg(src + p + (j - i) * stride);
  }
  diffs_of<R>(v, Dk);
  edge_diffs<R>(Dk, i, n);
}

// The same along the fastest axis (stride 1), from the 2R+1 line values v
// around the node: loaded unclamped at immediate offsets by the caller
// (near a row end some of them come from the neighbouring row, or from the
// guard floats every field carries before its first and after its last
// node), or read from a shared-memory copy of the row.  Returns the node's
// own value.  Only a warp that holds a node within R of a line end applies
// the end rule; the others (about half the warps at 81 nodes per line)
// skip it.  The vote runs over the lanes still active here, which is
// warp-uniform in outcome.
template <int R>
__device__ __forceinline__ float fast_line_diffs(const float (&v)[2 * R + 1], int i, int n,
                                                 float (&Dk)[2 * R]) {
  diffs_of<R>(v, Dk);
  if (__any_sync(__activemask(), i < R || i > n - 1 - R)) edge_diffs<R>(Dk, i, n);
  return v[R];
}

// ------------------------------------------------------------- slopes

// Packed FP32 pairs (Blackwell FFMA2 / FMUL2 / FADD2): one instruction
// issues the same operation on both lanes, each lane rounded exactly like
// the scalar fmaf / mul / add.
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Both one-sided WENO5 slopes (Jiang & Peng) at a node, from the six
// undivided differences D_k = v[k+1] - v[k] of the line values v at offsets
// -3..3.  The left-biased slope uses D0..D4; the right-biased slope uses
// D5..D1 in upwind order.  Returns h p- and h p+; the caller folds in 1 / h.
//
// The right-biased slope is the left-biased formula applied to the mirrored
// differences, so both run as the two lanes of packed FP32 pairs: lane x
// holds the left side's operand, lane y the right side's.  Packed pairs
// halve the issue slots of the arithmetic.
//
// Lane y runs on its second differences with the sign flipped.  Mirrored,
// they are (D4 - D5, D3 - D4, D2 - D3, D1 - D2); flipped, the two lanes share
// the five second differences of the line (D1 - D0 .. D5 - D4), and C is one
// value in both lanes.  The indicators are even in them and the candidate
// offsets odd, and rounding to nearest is symmetric in sign, so lane y ends
// with exactly the negated offset N / M: its X2 slot holds -D3 and the
// result is negated once more.  The slopes are bit for bit those of the
// unflipped form.
//
// The arithmetic is the textbook scheme, rewritten in the second
// differences A, B, C, E of the five upwind differences X0..X4 (A = X1 - X0,
// B = X2 - X1, C = X3 - X2, E = X4 - X3) to save operations:
//   - Smoothness indicators.  13/12 t^2 + 1/4 u^2 of each candidate equals
//     4/3 of a sum of two squares:
//       S1 = (A - 11/8 B)^2 + 39/64 B^2,
//       S2 = (B - 5/8 C)^2 + 39/64 C^2,
//       S3 = (E - 11/8 C)^2 + 39/64 C^2.
//     The epsilon gets the same factor 3/4, so every S_k + eps scales by
//     one common factor, which normalised weights cancel.  No term can
//     cancel another.
//   - Nonlinear weights a_k = c_k / (S_k + eps)^2 are evaluated as
//     c_1 s_2^2 s_3^2, c_2 s_1^2 s_3^2, c_3 s_1^2 s_2^2 with
//     s_k = S_k / eps + 1: the same normalised set, multiplied through by a
//     common factor.  Since S_k <= 34 max D^2 and eps >= 1e-6 max D^2, every
//     s_k lies in [1, 3.4e7], so the products stay inside FP32 range.
//   - Candidates.  The three third-order candidates times their linear
//     weights (1/10, 6/10, 3/10) sum to X2 times the weight sum plus
//     (B - 2A/5)/2, (B/2 + C) 6/5 and (C - E/4) 6/5 times the weights.  With
//     s_1^2 scaled by 12/5, the slope is X2 + N / M where
//       N = Q1 (B - 2A/5) + Q2 (B/2 + C) + Q3 (C - E/4),
//       M = 6/5 Q1 + 3 Q2 + 3/2 Q3,
//       Q1 = s_2^2 s_3^2, Q2 = 12/5 s_1^2 s_3^2, Q3 = 12/5 s_1^2 s_2^2.
//     It takes one reciprocal per side.
__device__ __forceinline__ void weno5_pair(float D0, float D1, float D2, float D3, float D4,
                                           float D5, float floor_, float& pm_h, float& pp_h) {
  const float a = D1 - D0, b = D2 - D1, c = D3 - D2, d = D4 - D3, f = D5 - D4;
  const float2 A = make_float2(a, f), B = make_float2(b, d);
  const float2 C = make_float2(c, c), E = make_float2(d, b);
  const float2 X2 = make_float2(D2, -D3);
  const float2 k = f2s(39.f / 64.f);
  float2 kB2 = mul2(mul2(k, B), B);
  // C holds one value in both lanes: its square term is one scalar product
  const float kc = (39.f / 64.f) * c * c;
  const float2 kC2 = make_float2(kc, kc);
  float2 q1 = fma2(f2s(-1.375f), B, A);
  float2 q2 = fma2(f2s(-0.625f), C, B);
  float2 q3 = fma2(f2s(-1.375f), C, E);
  float2 S1 = fma2(q1, q1, kB2);
  float2 S2 = fma2(q2, q2, kC2);
  float2 S3 = fma2(q3, q3, kC2);
  // epsilon = 3/4 (1e-6 max D^2 + floor), the factor of the indicators
  float mid = fmaxf(fmaxf(fabsf(D1), fabsf(D2)), fmaxf(fabsf(D3), fabsf(D4)));
  float2 m = make_float2(fmaxf(mid, fabsf(D0)), fmaxf(mid, fabsf(D5)));
  float2 e = fma2(mul2(f2s(0.75e-6f), m), m, f2s(floor_));
  float2 ie = make_float2(rcp_approx(e.x), rcp_approx(e.y));
  float2 s1 = fma2(S1, ie, f2s(1.f)), s2 = fma2(S2, ie, f2s(1.f)), s3 = fma2(S3, ie, f2s(1.f));
  s1 = mul2(mul2(f2s(2.4f), s1), s1);
  s2 = mul2(s2, s2);
  s3 = mul2(s3, s3);
  float2 Q1 = mul2(s2, s3), Q2 = mul2(s1, s3), Q3 = mul2(s1, s2);
  float2 h1 = fma2(f2s(-0.4f), A, B);
  float2 h2 = fma2(f2s(0.5f), B, C);
  float2 h3 = fma2(f2s(-0.25f), E, C);
  float2 num = fma2(Q1, h1, fma2(Q2, h2, mul2(Q3, h3)));
  float2 den = fma2(f2s(1.2f), Q1, fma2(f2s(3.f), Q2, mul2(f2s(1.5f), Q3)));
  float2 w = fma2(num, make_float2(rcp_approx(den.x), rcp_approx(den.y)), X2);
  pm_h = w.x;
  pp_h = -w.y;
}

// Per scheme: the stencil radius R and raw one-sided slopes, from the 2R
// first differences Dk of the node's line (Dk[k] spans offsets k-R and
// k-R+1), whose scale the caller removes with folded per-axis constants
// (half and half-alpha times 1/h for first order and ENO2, times 1/(6h) for
// WENO5).
template <int S>
struct Slopes;

template <>
struct Slopes<1> {
  static constexpr int R = 1;
  __device__ __forceinline__ static void eval(const float (&Dk)[2], const DevGrid&, int,
                                              float& pm, float& pp) {
    pm = Dk[0];
    pp = Dk[1];
  }
  __device__ __forceinline__ static float half(const DevGrid& g, int d) { return g.hih[d]; }
  __device__ __forceinline__ static float half_alpha(const DevGrid& g, int d) { return g.haih[d]; }
};

// ENO2: first difference plus half the smaller (in magnitude) of the two
// adjacent second differences; ties take the left one.  The second
// differences are differences of the first ones.
template <>
struct Slopes<2> {
  static constexpr int R = 2;
  __device__ __forceinline__ static void eval(const float (&Dk)[4], const DevGrid&, int,
                                              float& pm, float& pp) {
    float a = Dk[1] - Dk[0];
    float b = Dk[2] - Dk[1];
    float c = Dk[3] - Dk[2];
    float m1 = (fabsf(a) <= fabsf(b)) ? a : b;
    float m2 = (fabsf(b) <= fabsf(c)) ? b : c;
    pm = fmaf(0.5f, m1, Dk[1]);
    pp = fmaf(-0.5f, m2, Dk[2]);
  }
  __device__ __forceinline__ static float half(const DevGrid& g, int d) { return g.hih[d]; }
  __device__ __forceinline__ static float half_alpha(const DevGrid& g, int d) { return g.haih[d]; }
};

template <>
struct Slopes<5> {
  static constexpr int R = 3;
  __device__ __forceinline__ static void eval(const float (&Dk)[6], const DevGrid& g, int d,
                                              float& pm, float& pp) {
    weno5_pair(Dk[0], Dk[1], Dk[2], Dk[3], Dk[4], Dk[5], g.wfloor[d], pm, pp);
  }
  __device__ __forceinline__ static float half(const DevGrid& g, int d) { return g.hih[d]; }
  __device__ __forceinline__ static float half_alpha(const DevGrid& g, int d) { return g.haih[d]; }
};

// L(src) at node p with multi-index idx; also returns src[p] in `center`.
// The last axis is the fastest (stride 1).  Its line values come either
// from `fast`, a shared-memory copy of the node's row (fast[k] is the line
// value at offset k, k = -R..R), or, when fast is null, from global memory
// at immediate offsets; src then needs at least 3 readable guard floats
// before its first and after its last node.  Both give the same
// differences (fast_line_diffs).
template <int D, int S, int M>
__device__ __forceinline__ float lf_rhs(const DevGrid& g, const float* __restrict__ src, int p,
                                        const int (&idx)[D], const float (&x)[D], float& center,
                                        const float* fast = nullptr) {
  constexpr int R = Slopes<S>::R;
  float pbar[D];
  float diss = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    float Dk[2 * R];
    if (d == D - 1) {
      float v[2 * R + 1];
#pragma unroll
      for (int k = -R; k <= R; ++k) v[k + R] = fast ? fast[k] : __ldg(src + p + k);
      center = fast_line_diffs<R>(v, idx[d], g.n[d], Dk);
    } else {
      line_diffs<R>(src, p, g.stride[d], idx[d], g.n[d], Dk);
    }
    float pm, pp;
    Slopes<S>::eval(Dk, g, d, pm, pp);
    pbar[d] = Slopes<S>::half(g, d) * (pm + pp);
    diss = fmaf(Slopes<S>::half_alpha(g, d), pp - pm, diss);
  }
  return hamiltonian<M, D>(g, x, idx, pbar, p) + diss;
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
