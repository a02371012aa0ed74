// hj_kernels.cu -- sm_103a kernels of the HJ level-set solve.
//
//  stage_kernel   one TVD-RK3 stage: slopes on every axis, Lax-Friedrichs
//                 Hamiltonian, the RK combination, and in stage 3 the clamp
//                 W <- min(W3, l) of Eq. 2 plus the window residual.
//  alpha_kernel   max-reduction of |f_i| over the grid for the LF
//                 coefficients and the CFL dt.
//  init_kernel    cold start W = l, or warm start W = min(prior, l) (Sec. III-B).
//  prolong_kernel coarse-to-fine migration (Sec. III-C).
//  query_kernel   value / gradient read-out for the safety controller (Sec. II-A).
//
// The stencil is bound by FP32 instruction issue: about 450 FP32
// instructions per node and stage for WENO5 in 4-D, against 8-12 bytes of
// compulsory traffic.  So threads map one-to-one onto nodes.  A 4-D grid runs
// one slab of its last three axes per blockIdx.y; lower ranks are a single
// slab.  That keeps warps fully populated whatever the axis lengths.  Line
// neighbours come through the read-only (L1) path.  The warps of a block
// cover adjacent rows, so the +-3 neighbours along the two fast axes are L1
// hits.
#include <algorithm>
#include <cstdint>
#include <cstdio>

#include "hj_internal.h"
#include "hj_stage.cuh"

namespace hjk {

std::atomic<unsigned long long> g_launches{0};

using hjd::DevGrid;
using hjd::StageArgs;

template <int D, int S, int M, int STAGE, int THREADS, bool LOCAL>
__global__ void __launch_bounds__(THREADS) stage_kernel(const DevGrid g, const StageArgs a) {
  hjd::flat_body<D, S, M, STAGE, LOCAL>(g, a);
}

// Whether a stage launch is part of a localized solve.
static bool is_local(const StageArgs& a) { return a.tiles || a.live || a.slab_resid; }

// Row-tile variant: block b stages lines [b R, b R + R) of the fastest axis
// in shared memory (hjd::stage_tile) and computes their nodes.
template <int D, int S, int M, int STAGE, int MAXT>
__global__ void __launch_bounds__(MAXT) tile_kernel(const DevGrid g, const StageArgs a) {
  extern __shared__ float sm[];
  hjd::tile_body<D, S, M, STAGE>(g, a, sm);
}

template <int D>
__device__ __forceinline__ void unravel(const DevGrid& g, int pt, int (&idx)[D]) {
#pragma unroll
  for (int d = D - 1; d > 0; --d) {
    int q = pt / g.n[d];
    idx[d] = pt - q * g.n[d];
    pt = q;
  }
  idx[0] = pt;
}

using hjd::coords;
using hjd::locate;
using hjd::node_diff2;

template <int D, int M>
__global__ void alpha_kernel(const DevGrid g, unsigned* out) {
  float m[D];
#pragma unroll
  for (int d = 0; d < D; ++d) m[d] = 0.f;
  for (int pt = blockIdx.x * blockDim.x + threadIdx.x; pt < g.npts; pt += gridDim.x * blockDim.x) {
    int idx[D];
    float x[D];
    unravel<D>(g, pt, idx);
    coords<D>(g, idx, x);
    hjd::abs_f_max<M, D>(g, x, idx, m, pt);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    hjd::block_max_bits(__float_as_uint(m[d]), out + d);
    __syncthreads();
  }
}

template <int D>
__global__ void init_kernel(const DevGrid g, float* W, float* snap, int warm) {
  for (int pt = blockIdx.x * blockDim.x + threadIdx.x; pt < g.npts; pt += gridDim.x * blockDim.x) {
    int idx[D];
    float x[D];
    unravel<D>(g, pt, idx);
    coords<D>(g, idx, x);
    float l = hjd::margin<D>(g, x, pt);
    float w = warm ? fminf(W[pt], l) : l;
    W[pt] = w;
    snap[pt] = w;
  }
}


template <int D>
__global__ void prolong_kernel(const DevGrid c, const float* __restrict__ Wc, const DevGrid f,
                               float* Wf, hjk::Shift sh, int* bad) {
  for (int pt = blockIdx.x * blockDim.x + threadIdx.x; pt < f.npts; pt += gridDim.x * blockDim.x) {
    int idx[D];
    unravel<D>(f, pt, idx);
    int i0[D];
    double fr[D];
    float xf[D];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      double xv = f.lo_d[d] + (double)idx[d] * f.h_d[d];
      xf[d] = (float)xv;
      ok = ok && locate(c, d, xv - sh.s[d], i0[d], fr[d]);
    }
    float l = hjd::margin<D>(f, xf, pt);
    if (!ok) {
      // outside the source box: the cold start there, or an error
      if (sh.fill_outside) Wf[pt] = l;
      else *bad = 1;
      continue;
    }
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < (1 << D); ++k) {
      double wgt = 1.0;
      int off = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        int bit = (k >> d) & 1;
        wgt *= bit ? fr[d] : 1.0 - fr[d];
        off += (i0[d] + bit) * c.stride[d];
      }
      acc += wgt * (double)__ldg(Wc + off);
    }
    Wf[pt] = fminf((float)acc, l);
  }
}


template <int D>
__global__ void query_kernel(const DevGrid g, const float* __restrict__ W, int npts,
                             const double* __restrict__ xs, double* out, int* bad, int grad) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npts) return;
  int i0[D];
  double fr[D];
  bool ok = true;
#pragma unroll
  for (int d = 0; d < D; ++d) ok = ok && locate(g, d, xs[k * D + d], i0[d], fr[d]);
  if (!ok) {
    *bad = 1;
    return;
  }
  double acc[D + 1];
#pragma unroll
  for (int e = 0; e <= D; ++e) acc[e] = 0.0;
#pragma unroll
  for (int c = 0; c < (1 << D); ++c) {
    double wgt = 1.0;
    int off = 0;
    int ci[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      int bit = (c >> d) & 1;
      wgt *= bit ? fr[d] : 1.0 - fr[d];
      ci[d] = i0[d] + bit;
      off += ci[d] * g.stride[d];
    }
    if (grad) {
#pragma unroll
      for (int d = 0; d < D; ++d) acc[d] += wgt * node_diff2<D>(g, W, off, ci[d], d);
    } else {
      acc[0] += wgt * (double)W[off];
    }
  }
  if (grad) {
#pragma unroll
    for (int d = 0; d < D; ++d) out[k * D + d] = acc[d] * g.ih2_d[d];
  } else {
    out[k] = acc[0];
  }
}

// ------------------------------------------------------------- dispatch

static dim3 stage_grid(const DevGrid& g, int threads) {
  unsigned bx = (unsigned)((g.plane + threads - 1) / threads);
  unsigned by = g.ndim == 4 ? (unsigned)g.n[0] : 1u;
  return dim3(bx, by, 1u);
}

template <int D, int S, int M, int T, bool LOCAL>
static void stage_launch(const DevGrid& g, int stage, const StageArgs& a, cudaStream_t s) {
  dim3 grid = a.tiles ? dim3((unsigned)a.ntiles, 1u, 1u) : stage_grid(g, T), block(T);
  switch (stage) {
    case 1: stage_kernel<D, S, M, 1, T, LOCAL><<<grid, block, 0, s>>>(g, a); break;
    case 2: stage_kernel<D, S, M, 2, T, LOCAL><<<grid, block, 0, s>>>(g, a); break;
    default: stage_kernel<D, S, M, 3, T, LOCAL><<<grid, block, 0, s>>>(g, a); break;
  }
}

template <int D, int S, int M, int MAXT>
static void tile_launch(const DevGrid& g, int stage, const StageArgs& a, const TileShape& ts,
                        cudaStream_t s) {
  dim3 grid(a.tiles ? (unsigned)a.ntiles : ts.blocks), block(ts.threads);
  if (grid.x == 0) return;
  switch (stage) {
    case 1: tile_kernel<D, S, M, 1, MAXT><<<grid, block, ts.smem, s>>>(g, a); break;
    case 2: tile_kernel<D, S, M, 2, MAXT><<<grid, block, ts.smem, s>>>(g, a); break;
    default: tile_kernel<D, S, M, 3, MAXT><<<grid, block, ts.smem, s>>>(g, a); break;
  }
}

template <int D, int S, int M>
static cudaError_t stage_dispatch(const DevGrid& g, int stage, const StageArgs& a, int threads,
                                  cudaStream_t s) {
  if (g.tile_rows > 0) {
    TileShape ts = tile_shape(g, S);
    if (ts.threads <= 256) tile_launch<D, S, M, 256>(g, stage, a, ts, s);
    else if (ts.threads <= 512) tile_launch<D, S, M, 512>(g, stage, a, ts, s);
    else tile_launch<D, S, M, 1024>(g, stage, a, ts, s);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
  }
  if (is_local(a)) {
    // localized solves launch 256-thread blocks of the flat mapping
    stage_launch<D, S, M, 256, true>(g, stage, a, s);
  } else {
    switch (threads) {
      case 128: stage_launch<D, S, M, 128, false>(g, stage, a, s); break;
      case 512: stage_launch<D, S, M, 512, false>(g, stage, a, s); break;
      default: stage_launch<D, S, M, 256, false>(g, stage, a, s); break;
    }
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <int D, int M>
static cudaError_t stage_by_scheme(const DevGrid& g, int scheme, int stage, const StageArgs& a,
                                   int threads, cudaStream_t s) {
  switch (scheme) {
    case 1: return stage_dispatch<D, 1, M>(g, stage, a, threads, s);
    case 2: return stage_dispatch<D, 2, M>(g, stage, a, threads, s);
    case 5: return stage_dispatch<D, 5, M>(g, stage, a, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

bool stage_supported(int model, int ndim, int scheme) {
  if (scheme != 1 && scheme != 2 && scheme != 5) return false;
  if (model == hjd::M_QUAD_Z) return ndim == 2;
  if (model == hjd::M_QUAD_X4) return ndim == 4;
  if (model == hjd::M_DRIFT) return ndim >= 1 && ndim <= 4;
  return false;
}

TileShape tile_shape(const DevGrid& g, int scheme) {
  TileShape t;
  int radius = scheme == 5 ? 3 : (scheme == 2 ? 2 : 1);
  int n = g.n[g.ndim - 1];
  int rows = g.tile_rows < g.nrows ? g.tile_rows : g.nrows;
  t.threads = (rows * n + 31) / 32 * 32;
  t.blocks = (unsigned)((g.nrows + g.tile_rows - 1) / g.tile_rows);
  t.smem = (size_t)g.tile_rows * (size_t)(n + 2 * radius) * sizeof(float);
  return t;
}

bool tile_ok(const DevGrid& g, int tile_rows, const void* const* fields, int nfields) {
  if (tile_rows <= 0) return false;
  long long nodes = (long long)tile_rows * g.n[g.ndim - 1];
  if (nodes > kTileMaxThreads || (long long)tile_rows > (long long)g.nrows) return false;
  for (int i = 0; i < nfields; ++i)
    if (reinterpret_cast<uintptr_t>(fields[i]) & 15u) return false;
  return true;
}

cudaError_t launch_stage(const DevGrid& g, int scheme, int stage, const StageArgs& a, cudaStream_t s,
                         int threads, bool allow_jit) {
  if (threads != 128 && threads != 512) threads = 256;
  if (g.tile_rows <= 0 && is_local(a)) threads = 256;
  if (g.tile_rows > 0 && (reinterpret_cast<uintptr_t>(a.src) & 15u)) return cudaErrorInvalidValue;
  if (a.tiles && a.ntiles == 0) return cudaSuccess;
  if (allow_jit) {
    bool used = false;
    cudaError_t e = jit_launch(g, scheme, stage, a, s, threads, &used);
    if (used || e != cudaSuccess) return e;
  }
  switch (g.model) {
    case hjd::M_QUAD_Z: return stage_by_scheme<2, hjd::M_QUAD_Z>(g, scheme, stage, a, threads, s);
    case hjd::M_QUAD_X4: return stage_by_scheme<4, hjd::M_QUAD_X4>(g, scheme, stage, a, threads, s);
    default:
      switch (g.ndim) {
        case 1: return stage_by_scheme<1, hjd::M_DRIFT>(g, scheme, stage, a, threads, s);
        case 2: return stage_by_scheme<2, hjd::M_DRIFT>(g, scheme, stage, a, threads, s);
        case 3: return stage_by_scheme<3, hjd::M_DRIFT>(g, scheme, stage, a, threads, s);
        case 4: return stage_by_scheme<4, hjd::M_DRIFT>(g, scheme, stage, a, threads, s);
      }
  }
  return cudaErrorInvalidValue;
}

int num_sms() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = -1;
  if (dev >= 0) {
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev < 0 ? 0 : dev) !=
          cudaSuccess ||
      sms <= 0) {
    cudaGetLastError();
    sms = 1;
  }
  if (dev >= 0) cached[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

unsigned stride_blocks(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  // grid-stride loops: cap at a few waves of the device's SMs
  return (unsigned)std::max(1ll, std::min(b, 16ll * num_sms()));
}

static unsigned flat_blocks(int npts, int threads) { return stride_blocks(npts, threads); }

cudaError_t launch_alpha(const DevGrid& g, unsigned* out, cudaStream_t s) {
  unsigned nb = flat_blocks(g.npts, 256);
  switch (g.model) {
    case hjd::M_QUAD_Z: alpha_kernel<2, hjd::M_QUAD_Z><<<nb, 256, 0, s>>>(g, out); break;
    case hjd::M_QUAD_X4: alpha_kernel<4, hjd::M_QUAD_X4><<<nb, 256, 0, s>>>(g, out); break;
    default:
      switch (g.ndim) {
        case 1: alpha_kernel<1, hjd::M_DRIFT><<<nb, 256, 0, s>>>(g, out); break;
        case 2: alpha_kernel<2, hjd::M_DRIFT><<<nb, 256, 0, s>>>(g, out); break;
        case 3: alpha_kernel<3, hjd::M_DRIFT><<<nb, 256, 0, s>>>(g, out); break;
        case 4: alpha_kernel<4, hjd::M_DRIFT><<<nb, 256, 0, s>>>(g, out); break;
        default: return cudaErrorInvalidValue;
      }
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_init(const DevGrid& g, float* W, float* snap, int warm, cudaStream_t s) {
  unsigned nb = flat_blocks(g.npts, 256);
  switch (g.ndim) {
    case 1: init_kernel<1><<<nb, 256, 0, s>>>(g, W, snap, warm); break;
    case 2: init_kernel<2><<<nb, 256, 0, s>>>(g, W, snap, warm); break;
    case 3: init_kernel<3><<<nb, 256, 0, s>>>(g, W, snap, warm); break;
    case 4: init_kernel<4><<<nb, 256, 0, s>>>(g, W, snap, warm); break;
    default: return cudaErrorInvalidValue;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const DevGrid& c, const float* Wc, const DevGrid& f, float* Wf,
                           const Shift& sh, int* bad, cudaStream_t s) {
  unsigned nb = flat_blocks(f.npts, 256);
  switch (f.ndim) {
    case 1: prolong_kernel<1><<<nb, 256, 0, s>>>(c, Wc, f, Wf, sh, bad); break;
    case 2: prolong_kernel<2><<<nb, 256, 0, s>>>(c, Wc, f, Wf, sh, bad); break;
    case 3: prolong_kernel<3><<<nb, 256, 0, s>>>(c, Wc, f, Wf, sh, bad); break;
    case 4: prolong_kernel<4><<<nb, 256, 0, s>>>(c, Wc, f, Wf, sh, bad); break;
    default: return cudaErrorInvalidValue;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

// ------------------------------------------------- localized stepping

// Slab masks from the last window's per-slab changes.  A slab is raw-active
// when its change exceeds thr.  A slab
//   steps (live)          when a raw-active slab lies within k0 slabs along
//                         the first slab axis and k1 along the second;
//   gets stage 2 (ring2)  within k0 + R, k1 + R, so that stage 3 at live
//                         nodes reads valid W2 within its stencil radius R;
//   gets stage 1 (ring1)  within k0 + 2R, k1 + 2R, so that stage 2 on ring2
//                         reads valid W1.
// k0, k1 cover how far a change can travel in one window (the host derives
// them from the CFL speeds), so that a frozen slab wakes up before anything
// reaches it.
__global__ void local_masks_kernel(const unsigned* __restrict__ resid, int s0, int s1, float thr,
                                   int k0, int k1, int radius, unsigned char* live,
                                   unsigned char* ring2, unsigned char* ring1) {
  int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= s0 * s1) return;
  int i = sl / s1, j = sl - i * s1;
  int r0 = k0 + 2 * radius, r1 = k1 + 2 * radius;
  bool m_live = false, m2 = false, m1 = false;
  int i_lo = max(0, i - r0), i_hi = min(s0 - 1, i + r0);
  int j_lo = max(0, j - r1), j_hi = min(s1 - 1, j + r1);
  for (int a = i_lo; a <= i_hi; ++a)
    for (int b = j_lo; b <= j_hi; ++b)
      if (__uint_as_float(resid[a * s1 + b]) > thr) {
        int di = abs(a - i), dj = abs(b - j);
        m1 = true;
        m2 = m2 || (di <= k0 + radius && dj <= k1 + radius);
        m_live = m_live || (di <= k0 && dj <= k1);
      }
  live[sl] = m_live;
  ring2[sl] = m2;
  ring1[sl] = m1;
}

// Tile lists of the next window: list q (q = 0, 1, 2 for stages 1, 2, 3)
// gets every tile that holds a node of a slab in mask q (ring1, ring2,
// live).  Tile t covers the nodes [first(t), last(t)] of the flat node
// order: row tiles hold tile_rows lines of n_last nodes; flat tiles are the
// blocks of `threads` nodes of the flat mapping, `per` blocks per slab of
// `plane` nodes.  Slabs are runs of nodes_per_slab nodes.  counts[q] must be
// zero on entry; the order within a list does not matter.
__global__ void local_lists_kernel(int ntiles, int tile_rows, int n_last, int threads, int per,
                                   int plane, int npts, int nodes_per_slab,
                                   const unsigned char* __restrict__ ring1,
                                   const unsigned char* __restrict__ ring2,
                                   const unsigned char* __restrict__ live, int* lists,
                                   int* counts) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  long long first, last;
  if (tile_rows > 0) {
    first = (long long)t * tile_rows * n_last;
    last = min(first + (long long)tile_rows * n_last, (long long)npts) - 1;
  } else {
    int yb = t / per, bx = t - yb * per;
    long long q0 = (long long)bx * threads;
    first = (long long)yb * plane + q0;
    last = (long long)yb * plane + min(q0 + threads, (long long)plane) - 1;
  }
  int f = (int)(first / nodes_per_slab), l = (int)(last / nodes_per_slab);
  bool m1 = false, m2 = false, m3 = false;
  for (int sl = f; sl <= l; ++sl) {
    m1 = m1 || ring1[sl];
    m2 = m2 || ring2[sl];
    m3 = m3 || live[sl];
  }
  if (m1) lists[atomicAdd(counts + 0, 1)] = t;
  if (m2) lists[ntiles + atomicAdd(counts + 1, 1)] = t;
  if (m3) lists[2 * ntiles + atomicAdd(counts + 2, 1)] = t;
}

LocalLayout local_layout(const DevGrid& g, int threads) {
  LocalLayout L;
  if (g.ndim == 4) {
    L.s0 = g.n[0];
    L.s1 = g.n[1];
  } else if (g.ndim >= 2) {
    L.s0 = g.n[0];
    L.s1 = 1;
  }
  L.nslabs = L.s0 * L.s1;
  L.nodes_per_slab = g.npts / L.nslabs;
  L.threads = threads;
  if (g.tile_rows > 0) {
    L.ntiles = (g.nrows + g.tile_rows - 1) / g.tile_rows;
  } else {
    L.per = (g.plane + threads - 1) / threads;
    L.ntiles = L.per * (g.ndim == 4 ? g.n[0] : 1);
  }
  return L;
}

cudaError_t launch_local_lists(const DevGrid& g, int scheme, int threads,
                               const unsigned* slab_resid, float thr, int k0, int k1,
                               unsigned char* masks, int* lists, int* counts, cudaStream_t s) {
  LocalLayout L = local_layout(g, threads);
  int radius = scheme == 5 ? 3 : (scheme == 2 ? 2 : 1);
  unsigned char *live = masks, *ring2 = masks + L.nslabs, *ring1 = masks + 2 * L.nslabs;
  cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  local_masks_kernel<<<(L.nslabs + 255) / 256, 256, 0, s>>>(slab_resid, L.s0, L.s1, thr, k0,
                                                           L.s1 > 1 ? k1 : 0, radius, live,
                                                           ring2, ring1);
  local_lists_kernel<<<(L.ntiles + 255) / 256, 256, 0, s>>>(
      L.ntiles, g.tile_rows, g.n[g.ndim - 1], threads, L.per, g.plane, g.npts, L.nodes_per_slab,
      ring1, ring2, live, lists, counts);
  g_launches.fetch_add(2, std::memory_order_relaxed);
  return cudaGetLastError();
}

// *bad = 1 when some lo[k] > hi[k] or either is not finite.
__global__ void field_check_kernel(const float* __restrict__ lo, const float* __restrict__ hi,
                                   long long n, int* bad) {
  int found = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    float a = lo[k], b = hi[k];
    found |= !(isfinite(a) && isfinite(b) && a <= b);
  }
  if (__syncthreads_or(found) && threadIdx.x == 0) *bad = 1;
}

cudaError_t launch_field_check(const float* lo, const float* hi, long long n, int* bad,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  unsigned nb = stride_blocks(n, 256);
  field_check_kernel<<<nb, 256, 0, s>>>(lo, hi, n, bad);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_query(const DevGrid& g, const float* W, int npts, const double* x, double* out,
                         int* bad, int grad, cudaStream_t s) {
  unsigned nb = (unsigned)((npts + 127) / 128);
  if (nb == 0) return cudaSuccess;
  switch (g.ndim) {
    case 1: query_kernel<1><<<nb, 128, 0, s>>>(g, W, npts, x, out, bad, grad); break;
    case 2: query_kernel<2><<<nb, 128, 0, s>>>(g, W, npts, x, out, bad, grad); break;
    case 3: query_kernel<3><<<nb, 128, 0, s>>>(g, W, npts, x, out, bad, grad); break;
    case 4: query_kernel<4><<<nb, 128, 0, s>>>(g, W, npts, x, out, bad, grad); break;
    default: return cudaErrorInvalidValue;
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace hjk
