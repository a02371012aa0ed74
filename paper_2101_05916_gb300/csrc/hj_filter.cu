// hj_filter.cu -- the safety filter of the safe-learning loop (Sec. II-B,
// II-C) over a system decomposed into independent subsystem grids
// (Sec. III-A).
//
// Per query state and subsystem grid k: W_k and grad W_k by multilinear
// interpolation (node gradients: central differences, one-sided at the
// ends), the optimal safety control u*_k = argmax_u min_d <grad W_k, f_k>
// (bang-bang on the subsystem's one input), and the switch: u*_k replaces
// the performance control where W_k <= level.  The decomposed value is
// W = min_k W_k.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include <math_constants.h>

#include "hj.h"
#include "hj_device.cuh"
#include "hj_grid.h"
#include "hj_internal.h"

namespace {

using hjd::DevGrid;

// Where one subsystem sits in the full state and control vectors, and its
// single input: f depends on u only through axis gain_axis, as gain * u.
struct FilterMap {
  int axes[HJ_MAX_DIM];  // state index of each grid axis
  int ctrl;              // control index driven by this subsystem, -1 for none
  int bit;               // bit of this subsystem in the active mask
  int gain_axis;         // axis whose dynamics the input enters (-1: no input)
  double gain;           // d f_{gain_axis} / d u
  double ulo, uhi;       // input box
};

// Up to kPack subsystems per launch, as one __grid_constant__ parameter.
constexpr int kPack = 4;
struct FilterPack {
  int n;
  int first;                 // 1: this launch starts the outputs (w = +inf, active = 0)
  DevGrid g[kPack];
  FilterMap m[kPack];
  const float* W[kPack];
};

// W_k and grad W_k at one state; min into w, the switch into u and act.
template <int D>
__device__ __forceinline__ bool filter_point(const DevGrid& g, const float* __restrict__ W,
                                             const double* __restrict__ x, const FilterMap& m,
                                             double level, double* __restrict__ u, double& w,
                                             int& act) {
  int i0[D];
  double fr[D];
#pragma unroll
  for (int d = 0; d < D; ++d)
    if (!hjd::locate(g, d, x[m.axes[d]], i0[d], fr[d])) return false;
  double wk = 0.0, grad[D];
#pragma unroll
  for (int d = 0; d < D; ++d) grad[d] = 0.0;
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    double wgt = 1.0;
    int off = 0, ci[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      int bit = (c >> d) & 1;
      wgt *= bit ? fr[d] : 1.0 - fr[d];
      ci[d] = i0[d] + bit;
      off += ci[d] * g.stride[d];
    }
    wk += wgt * (double)__ldg(W + off);
#pragma unroll
    for (int d = 0; d < D; ++d) grad[d] += wgt * hjd::node_diff2<D>(g, W, off, ci[d], d);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) grad[d] *= g.ih2_d[d];
  w = fmin(w, wk);
  if (m.gain_axis >= 0 && m.ctrl >= 0 && wk <= level) {
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d)
      if (d == m.gain_axis) s = grad[d] * m.gain;
    double* uc = u + m.ctrl;
    // W is maximised by the input: the upper bound where the gain is
    // positive, the lower where it is negative; on a tie the performance
    // control stays, kept inside the input box
    *uc = s > 0.0 ? m.uhi : (s < 0.0 ? m.ulo : fmin(fmax(*uc, m.ulo), m.uhi));
    act |= 1 << m.bit;
  }
  return true;
}

__global__ void filter_kernel(const __grid_constant__ FilterPack P, long long nq,
                              const double* __restrict__ states, int state_dim, int ctrl_dim,
                              double level, double* __restrict__ u_out,
                              double* __restrict__ w_out, int* __restrict__ active, int* bad) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const double* x = states + q * state_dim;
  double* u = u_out + q * ctrl_dim;
  double w = P.first ? CUDART_INF : w_out[q];
  int act = P.first ? 0 : active[q];
  bool ok = true;
  for (int k = 0; k < P.n && ok; ++k) {
    switch (P.g[k].ndim) {
      case 1: ok = filter_point<1>(P.g[k], P.W[k], x, P.m[k], level, u, w, act); break;
      case 2: ok = filter_point<2>(P.g[k], P.W[k], x, P.m[k], level, u, w, act); break;
      case 3: ok = filter_point<3>(P.g[k], P.W[k], x, P.m[k], level, u, w, act); break;
      default: ok = filter_point<4>(P.g[k], P.W[k], x, P.m[k], level, u, w, act); break;
    }
  }
  if (!ok) {
    *bad = 1;
    return;
  }
  w_out[q] = w;
  active[q] = act;
}

}  // namespace

using hja::fail;

extern "C" {

hj_status hj_safety_filter(const hj_grid* grids, int ngrids, const int* axes,
                           const int* ctrl_index, int state_dim, int ctrl_dim, long long nq,
                           const double* states, const double* u_perf, double level,
                           double* u_out, double* w_out, int* active_out, int on_device) {
  if (!grids || !axes || !ctrl_index || ngrids < 1 || ngrids > 30)
    return fail(HJ_ERR_ARG, "need 1..30 grids with their axes and control indices");
  if (state_dim < 1 || ctrl_dim < 0 || nq < 0 || !std::isfinite(level))
    return fail(HJ_ERR_ARG, "bad dimensions or level");
  if (nq > 0 && (!states || !w_out || !active_out || (ctrl_dim > 0 && (!u_perf || !u_out))))
    return fail(HJ_ERR_ARG, "NULL buffer");
  unsigned used_ctrl = 0;
  for (int k = 0; k < ngrids; ++k) {
    hj_grid g = grids[k];
    if (!g) return fail(HJ_ERR_ARG, "grid %d is NULL", k);
    if (!g->has_value) return fail(HJ_ERR_STATE, "grid %d holds no value yet", k);
    if (g->model < 0) return fail(HJ_ERR_STATE, "grid %d has no dynamics", k);
    if (g->device != grids[0]->device) return fail(HJ_ERR_ARG, "grids on different devices");
    for (int d = 0; d < g->ndim; ++d)
      if (axes[k * HJ_MAX_DIM + d] < 0 || axes[k * HJ_MAX_DIM + d] >= state_dim)
        return fail(HJ_ERR_ARG, "grid %d axis %d: state index out of range", k, d);
    int c = ctrl_index[k];
    if (c >= ctrl_dim || c < -1) return fail(HJ_ERR_ARG, "grid %d: control index out of range", k);
    if (c >= 0) {
      if (c < 32 && (used_ctrl >> c) & 1u)
        return fail(HJ_ERR_ARG, "control %d is driven by two grids", c);
      if (c < 32) used_ctrl |= 1u << c;
    }
  }
  if (nq == 0) return HJ_OK;
  if (nq > (1ll << 31)) return fail(HJ_ERR_ARG, "at most 2^31 states per call");
  hj_grid g0 = grids[0];
  hja::DeviceGuard dg(g0->device);
  cudaStream_t s = g0->stream;
  size_t n_s = (size_t)nq * state_dim, n_u = (size_t)nq * ctrl_dim, n_w = (size_t)nq;
  const double* dx = states;
  double *du = u_out, *dw = w_out;
  int* da = active_out;
  int* dbad = (int*)(g0->dscal + 5);
  unsigned* hbad = g0->hscal + 5;
  if (!on_device) {
    // host buffers: one persistent device block and its pinned mirror, laid
    // out as [states | u | w | active | flag]; one copy in, one copy out
    size_t n_a = (n_w + 1) / 2;
    size_t need = n_s + n_u + n_w + n_a + 1;
    if (need > g0->fcap) {
      hja::dev_free(g0->alloc, g0->fdev);
      if (g0->fhost) cudaFreeHost(g0->fhost);
      g0->fdev = nullptr;
      g0->fhost = nullptr;
      g0->fcap = 0;
      HJ_CU(hja::dev_malloc(g0->alloc, (void**)&g0->fdev, need * sizeof(double)));
      HJ_CU(cudaMallocHost(&g0->fhost, need * sizeof(double)));
      g0->fcap = need;
    }
    double* h = g0->fhost;
    std::memcpy(h, states, n_s * sizeof(double));
    if (n_u) std::memcpy(h + n_s, u_perf, n_u * sizeof(double));
    std::memset(h + n_s + n_u + n_w + n_a, 0, sizeof(double));
    double* d = g0->fdev;
    dx = d;
    du = d + n_s;
    dw = du + n_u;
    da = (int*)(dw + n_w);
    dbad = (int*)(dw + n_w + n_a);
    hbad = (unsigned*)(h + n_s + n_u + n_w + n_a);
    // states, performance controls and the cleared flag in one copy
    HJ_CU(cudaMemcpyAsync(d, h, need * sizeof(double), cudaMemcpyHostToDevice, s));
  } else {
    if (n_u && du != u_perf)
      HJ_CU(cudaMemcpyAsync(du, u_perf, n_u * sizeof(double), cudaMemcpyDeviceToDevice, s));
    HJ_CU(cudaMemsetAsync(dbad, 0, sizeof(int), s));
  }
  unsigned nb = (unsigned)((nq + 127) / 128);
  for (int k0 = 0; k0 < ngrids; k0 += kPack) {
    FilterPack P;
    std::memset(&P, 0, sizeof(P));
    P.n = std::min(kPack, ngrids - k0);
    P.first = k0 == 0;
    for (int j = 0; j < P.n; ++j) {
      int k = k0 + j;
      FilterMap& m = P.m[j];
      for (int d = 0; d < grids[k]->ndim; ++d) m.axes[d] = axes[k * HJ_MAX_DIM + d];
      m.ctrl = ctrl_index[k];
      m.bit = k;
      m.gain_axis = -1;
      const double* prm = grids[k]->params;
      if (grids[k]->model == HJ_QUAD_Z) {  // dv/dt = kT u - g + d
        m.gain_axis = 1;
        m.gain = prm[0];
        m.ulo = prm[2];
        m.uhi = prm[3];
      } else if (grids[k]->model == HJ_QUAD_X4) {  // dw/dt = -d0 th + n0 u
        m.gain_axis = 3;
        m.gain = prm[3];
        m.ulo = prm[4];
        m.uhi = prm[5];
      }
      P.g[j] = hja::devgrid(grids[k]);
      P.W[j] = grids[k]->W;
    }
    filter_kernel<<<nb, 128, 0, s>>>(P, nq, dx, state_dim, ctrl_dim, level, du, dw, da, dbad);
    hjk::g_launches.fetch_add(1, std::memory_order_relaxed);
    HJ_CU(cudaGetLastError());
  }
  if (!on_device) {
    // u, w, active and the flag are contiguous after the states
    size_t n_out = n_u + n_w + (n_w + 1) / 2 + 1;
    HJ_CU(cudaMemcpyAsync(g0->fhost + n_s, du, n_out * sizeof(double), cudaMemcpyDeviceToHost,
                          s));
  } else {
    HJ_CU(cudaMemcpyAsync(hbad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  HJ_CU(cudaStreamSynchronize(s));
  if (*hbad) return fail(HJ_ERR_ARG, "a query state lies outside a grid box");
  if (!on_device) {
    const double* h = g0->fhost + n_s;
    if (n_u) std::memcpy(u_out, h, n_u * sizeof(double));
    std::memcpy(w_out, h + n_u, n_w * sizeof(double));
    std::memcpy(active_out, h + n_u + n_w, n_w * sizeof(int));
  }
  return HJ_OK;
}

}  // extern "C"
