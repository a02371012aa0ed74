// hj_static.cu -- hj_solve_fixed_static: the fixed-horizon solve without any
// device allocation, for callers that cannot allocate after start-up (a
// real-time safety filter next to a controller, where cudaMalloc/cudaFree may
// synchronise the device; or a process whose device memory belongs to
// another framework's pool).
//
// The scratch lives in one file-scope device array (below), shared by every
// call and held by each GPU that loads the library until exit.  It holds the
// coefficient accumulator, the model table, a guarded working copy of the
// caller's W and the two Runge-Kutta stage fields.  Host code
// never passes the symbol itself to a kernel: on the host that name is only
// a stand-in, not a device address.  Instead, the first call on each device
// asks the runtime for the array's device address with that device current,
// caches it, and hands that pointer to the kernels.  Under lazy module
// loading (the CUDA default) that lookup is also the moment the driver loads
// this module on the device and reserves the array.
#include <cmath>
#include <cstring>
#include <mutex>

#include "hj_grid.h"
#include "hj_stage.cuh"

namespace {

constexpr size_t kHeadBytes = 256;                                    // alpha bits (4 x u32)
constexpr size_t kTabBytes = sizeof(float) * HJ_STATIC_MAX_AXIS;      // g tan(th) table
// one field: guard floats, HJ_STATIC_MAX_POINTS nodes, guard floats
constexpr size_t kGuardBytes = sizeof(float) * hja::kGuard;
constexpr size_t kFieldBytes = sizeof(float) * (size_t)HJ_STATIC_MAX_POINTS + 2 * kGuardBytes;
// three fields: the working copy of W and the two Runge-Kutta stages
constexpr size_t kScratchBytes = kHeadBytes + kTabBytes + 3 * kFieldBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
hj_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return hja::fail(HJ_ERR_CUDA, "device id %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return hja::fail(HJ_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return HJ_OK;
}

template <int D>
__global__ void static_init_kernel(const hjd::DevGrid g, float* W, int warm) {
  for (int pt = blockIdx.x * blockDim.x + threadIdx.x; pt < g.npts; pt += gridDim.x * blockDim.x) {
    int idx[D];
    int r = pt;
#pragma unroll
    for (int d = D - 1; d > 0; --d) {
      int q = r / g.n[d];
      idx[d] = r - q * g.n[d];
      r = q;
    }
    idx[0] = r;
    float x[D];
    hjd::coords<D>(g, idx, x);
    float l = hjd::margin<D>(g, x, pt);
    W[pt] = warm ? fminf(W[pt], l) : l;
  }
}

cudaError_t launch_static_init(const hjd::DevGrid& g, float* W, int warm, cudaStream_t s) {
  unsigned nb = hjk::stride_blocks(g.npts, 256);
  switch (g.ndim) {
    case 1: static_init_kernel<1><<<nb, 256, 0, s>>>(g, W, warm); break;
    case 2: static_init_kernel<2><<<nb, 256, 0, s>>>(g, W, warm); break;
    case 3: static_init_kernel<3><<<nb, 256, 0, s>>>(g, W, warm); break;
    case 4: static_init_kernel<4><<<nb, 256, 0, s>>>(g, W, warm); break;
    default: return cudaErrorInvalidValue;
  }
  hjk::g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace

extern "C" hj_status hj_solve_fixed_static(int ndim, const int* n, const double* lo,
                                           const double* hi, int model, const double* params,
                                           int nparams, const double* d_lo, const double* d_hi,
                                           int nd, const double* box_lo, const double* box_hi,
                                           int mode, int scheme, double dt, long long steps,
                                           int clamp, float* W, void* cuda_stream) {
  if (!W) return hja::fail(HJ_ERR_ARG, "W is NULL");
  if (ndim < 1 || ndim > HJ_MAX_DIM || !n || !lo || !hi)
    return hja::fail(HJ_ERR_ARG, "bad grid description");
  if (mode != HJ_COLD && mode != HJ_WARM) return hja::fail(HJ_ERR_ARG, "bad mode");
  if (clamp != HJ_CLAMP_VI && clamp != HJ_CLAMP_MONOTONE) return hja::fail(HJ_ERR_ARG, "bad clamp");
  // dt == 0 selects the CFL step; a negative or NaN dt is an argument error
  if (steps < 0 || !(dt >= 0.0)) return hja::fail(HJ_ERR_ARG, "need steps >= 0 and dt >= 0");
  if (!box_lo || !box_hi) return hja::fail(HJ_ERR_ARG, "box is NULL");
  // A handle on the stack: no allocation, only the description fields are used.
  hj_grid_s g;
  g.ndim = ndim;
  long long npts = 1;
  for (int i = 0; i < ndim; ++i) {
    if (n[i] < 3) return hja::fail(HJ_ERR_ARG, "axis %d has %d nodes (need >= 3)", i, n[i]);
    if (!(hi[i] > lo[i]) || !std::isfinite(lo[i]) || !std::isfinite(hi[i]))
      return hja::fail(HJ_ERR_ARG, "axis %d: need finite lo < hi", i);
    npts *= n[i];
    if (npts > HJ_STATIC_MAX_POINTS)
      return hja::fail(HJ_ERR_ARG,
                       "grid of %lld+ nodes exceeds the allocation-free limit of %d nodes", npts,
                       HJ_STATIC_MAX_POINTS);
    g.n[i] = n[i];
    g.lo[i] = lo[i];
    g.hi[i] = hi[i];
    g.h[i] = (hi[i] - lo[i]) / (double)(n[i] - 1);
  }
  g.npts = npts;
  if (nparams < 0 || nparams > 8 || (nparams > 0 && !params))
    return hja::fail(HJ_ERR_ARG, "bad parameter vector");
  if (model == HJ_QUAD_Z) {
    if (ndim != 2 || nparams < 4) return hja::fail(HJ_ERR_ARG, "HJ_QUAD_Z needs 2-D and 4 params");
  } else if (model == HJ_QUAD_X4) {
    if (ndim != 4 || nparams < 7) return hja::fail(HJ_ERR_ARG, "HJ_QUAD_X4 needs 4-D and 7 params");
    if (params[6] != 0.0 && params[6] != 1.0) return hja::fail(HJ_ERR_ARG, "axis must be 0 or 1");
    if (n[2] > HJ_STATIC_MAX_AXIS)
      return hja::fail(HJ_ERR_ARG, "theta axis of %d nodes exceeds the limit of %d", n[2],
                       HJ_STATIC_MAX_AXIS);
    if (std::max(std::fabs(lo[2]), std::fabs(hi[2])) >= 1.5)
      return hja::fail(HJ_ERR_ARG, "theta range must stay inside (-1.5, 1.5) rad");
  } else if (model != HJ_DRIFT) {
    return hja::fail(HJ_ERR_ARG, "unknown model %d", model);
  }
  g.model = model;
  for (int i = 0; i < nparams; ++i) g.params[i] = params[i];
  int need_nd = model == HJ_DRIFT ? ndim : 1;
  if (nd != need_nd || !d_lo || !d_hi)
    return hja::fail(HJ_ERR_ARG, "model needs %d disturbance intervals", need_nd);
  for (int i = 0; i < nd; ++i) {
    if (!std::isfinite(d_lo[i]) || !std::isfinite(d_hi[i]) || d_lo[i] > d_hi[i])
      return hja::fail(HJ_ERR_ARG, "input %d: need finite d_lo <= d_hi", i);
    g.d_lo[i] = d_lo[i];
    g.d_hi[i] = d_hi[i];
  }
  g.nd = nd;
  int constrained = 0;
  for (int i = 0; i < ndim; ++i) {
    if (std::isnan(box_lo[i]) || std::isnan(box_hi[i]) || !(box_lo[i] <= box_hi[i]))
      return hja::fail(HJ_ERR_ARG, "axis %d: need box_lo <= box_hi", i);
    if (!(std::isinf(box_lo[i]) && std::isinf(box_hi[i]))) constrained++;
    g.ca[i] = box_lo[i];
    g.cb[i] = box_hi[i];
  }
  if (!constrained) return hja::fail(HJ_ERR_ARG, "no axis is constrained");
  g.con_kind = hjd::C_BOX;
  hj_status st = hja::validate_ready(&g, scheme);
  if (st != HJ_OK) return st;

  int dev = 0;
  HJ_CU(cudaGetDevice(&dev));
  // W must be device (or managed) memory of the current device: a host
  // pointer, or memory of another GPU, would fault inside the kernels.
  // Asking for its attributes allocates nothing.
  cudaPointerAttributes pa;
  std::memset(&pa, 0, sizeof(pa));
  cudaError_t pe = cudaPointerGetAttributes(&pa, W);
  if (pe != cudaSuccess) {
    cudaGetLastError();
    return hja::fail(HJ_ERR_ARG, "W is not a CUDA pointer: %s", cudaGetErrorString(pe));
  }
  if (!(pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) || pa.device != dev)
    return hja::fail(HJ_ERR_ARG, "W must be device memory of the current device %d", dev);
  unsigned char* base = nullptr;
  if ((st = scratch_address(dev, &base)) != HJ_OK) return st;
  unsigned* alpha_bits = reinterpret_cast<unsigned*>(base);
  float* tab = reinterpret_cast<float*>(base + kHeadBytes);
  unsigned char* fields = base + kHeadBytes + kTabBytes;
  // the stencil reads a few floats past both ends of its source, so the
  // solve runs on a guarded working copy of the caller's W
  float* Wk = reinterpret_cast<float*>(fields + kGuardBytes);
  float* A = reinterpret_cast<float*>(fields + kFieldBytes + kGuardBytes);
  float* B = reinterpret_cast<float*>(fields + 2 * kFieldBytes + kGuardBytes);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t wbytes = (size_t)npts * sizeof(float);

  if (model == HJ_QUAD_X4) {
    float host_tab[HJ_STATIC_MAX_AXIS];
    for (int j = 0; j < n[2]; ++j)
      host_tab[j] = (float)(params[0] * std::tan(lo[2] + j * g.h[2]));
    HJ_CU(cudaMemcpyAsync(tab, host_tab, sizeof(float) * n[2], cudaMemcpyHostToDevice, s));
    g.tab = tab;
  }
  // the coefficient accumulator must start at zero; stage fields are fully
  // overwritten before they are read
  HJ_CU(cudaMemsetAsync(alpha_bits, 0, 4 * sizeof(unsigned), s));
  hjd::DevGrid d = hja::devgrid(&g);
  HJ_CU(hjk::launch_alpha(d, alpha_bits, s));
  unsigned host_bits[4] = {0, 0, 0, 0};
  HJ_CU(cudaMemcpyAsync(host_bits, alpha_bits, sizeof(host_bits), cudaMemcpyDeviceToHost, s));
  HJ_CU(cudaStreamSynchronize(s));
  for (int i = 0; i < ndim; ++i) std::memcpy(&g.alpha[i], &host_bits[i], 4);
  double step = dt > 0.0 ? dt : hja::cfl_dt(&g, 0.5);
  d = hja::devgrid(&g);
  if (mode == HJ_WARM) HJ_CU(cudaMemcpyAsync(Wk, W, wbytes, cudaMemcpyDeviceToDevice, s));
  HJ_CU(launch_static_init(d, Wk, mode == HJ_WARM ? 1 : 0, s));
  if (step > 0.0) {
    float fdt = (float)step;
    hjd::StageArgs a1{Wk, Wk, A, nullptr, nullptr, fdt, 0, clamp, 0.f, 0};
    hjd::StageArgs a2{A, Wk, B, nullptr, nullptr, fdt, 0, clamp, 0.f, 0};
    hjd::StageArgs a3{B, Wk, Wk, nullptr, nullptr, fdt, 0, clamp, 0.f, 0};
    for (long long k = 0; k < steps; ++k) {
      HJ_CU(hjk::launch_stage(d, scheme, 1, a1, s, hjk::kStageThreads, false));
      HJ_CU(hjk::launch_stage(d, scheme, 2, a2, s, hjk::kStageThreads, false));
      HJ_CU(hjk::launch_stage(d, scheme, 3, a3, s, hjk::kStageThreads, false));
    }
  }
  HJ_CU(cudaMemcpyAsync(W, Wk, wbytes, cudaMemcpyDeviceToDevice, s));
  HJ_CU(cudaStreamSynchronize(s));
  return HJ_OK;
}
