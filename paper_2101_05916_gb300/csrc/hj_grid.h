// hj_grid.h -- the grid handle shared by the C ABI translation units.
#pragma once

#include <cstdarg>
#include <cuda_runtime.h>

#include "hj.h"
#include "hj_internal.h"

namespace hja {
// The device allocator an object was created with (hj_set_allocator); both
// null: cudaMalloc / cudaFree.
struct Allocator {
  hj_alloc_fn alloc = nullptr;
  hj_free_fn free = nullptr;
  void* user = nullptr;
};
Allocator current_allocator();
// Device memory through the allocator (cudaErrorMemoryAllocation when it has
// none); release through it (a null pointer is ignored).
cudaError_t dev_malloc(const Allocator& a, void** p, size_t bytes);
void dev_free(const Allocator& a, void* p);
}  // namespace hja

struct hj_grid_s {
  int device = 0;
  hja::Allocator alloc;  // serves every device allocation of this grid
  int ndim = 0;
  int n[HJ_MAX_DIM] = {0, 0, 0, 0};
  double lo[HJ_MAX_DIM] = {0, 0, 0, 0};
  double hi[HJ_MAX_DIM] = {0, 0, 0, 0};
  double h[HJ_MAX_DIM] = {0, 0, 0, 0};
  long long npts = 0;
  cudaStream_t stream = nullptr;      // caller's stream (nullptr = legacy default)
  cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture

  int model = -1;
  double params[8] = {0};
  int nd = 0;
  double d_lo[HJ_MAX_DIM] = {0}, d_hi[HJ_MAX_DIM] = {0};
  int con_kind = -1;
  double ca[HJ_MAX_DIM] = {0}, cb[HJ_MAX_DIM] = {0};

  float* W = nullptr;      // value function (result, or prior for a warm start)
  float* A = nullptr;      // RK stage 1
  float* B = nullptr;      // RK stage 2
  float* snap = nullptr;   // W at the start of the current check window
  float* raw[4] = {nullptr, nullptr, nullptr, nullptr};  // allocations behind W, A, B, snap
  float* tab = nullptr;    // per-index coefficient table of the model
  float* dfield = nullptr; // state-dependent disturbance box: lo (nd x npts), then hi
  int dfield_nd = 0;       // inputs in dfield (0: the uniform box is in force)
  float* lfield = nullptr; // constraint margin l at every node (constraint kind C_FIELD)
  unsigned* dscal = nullptr;  // device scalars: [0..3] alpha bits, [4] residual bits, [5] flag
  unsigned* hscal = nullptr;  // pinned host mirror of dscal
  double* qbuf = nullptr;     // query staging (device)
  size_t qcap = 0;
  double* fdev = nullptr;     // safety-filter staging: device block ...
  double* fhost = nullptr;    // ... and its pinned host mirror
  size_t fcap = 0;            // doubles in each

  // localized stepping (allocated on first use): per-slab window change,
  // slab masks, the three stages' tile lists and their lengths
  unsigned* slab_resid = nullptr;
  unsigned char* slab_masks = nullptr;
  int* tile_lists = nullptr;
  int* tile_counts = nullptr;     // device, 3 ints
  int* tile_counts_h = nullptr;   // pinned host mirror
  long long local_slabs = 0, local_tiles = 0;  // sizes the buffers were made for

  bool has_value = false;
  bool alpha_valid = false;
  int threads = 256;        // stage-kernel block size of the flat mapping (hj_autotune may change it)
  int tile_rows = 0;        // > 0: row-tile stage kernels with this many lines per block
  int tuned_scheme = 0;     // scheme the block size was tuned for (0 = not tuned)
  float alpha[HJ_MAX_DIM] = {0, 0, 0, 0};

  cudaGraphExec_t gexec = nullptr;  // cached graph of one check window
  long long g_per = 0;
  float g_dt = 0.f;
  int g_scheme = 0, g_clamp = 0;
  float g_band = 0.f;
  int g_margin = 0;
  int g_threads = 0;
  int g_tile_rows = 0;
  bool g_jit = false;  // the cached graph holds shape-specialised kernels
};

namespace hja {

// Guard floats before the first and after the last node of every field.
// The stencil loads the fastest-axis line unclamped, up to 3 nodes past
// either end of the field.
constexpr size_t kGuard = 64;

hj_status fail(hj_status s, const char* fmt, ...);
hjd::DevGrid devgrid(const hj_grid g);
hj_status ensure_alpha(hj_grid g);
hj_status validate_ready(hj_grid g, int scheme);
hj_status autotune(hj_grid g, int scheme, int clamp);
double cfl_dt(const hj_grid g, double cfl);

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace hja

#define HJ_CU(call)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return hja::fail(e_ == cudaErrorMemoryAllocation ? HJ_ERR_OOM : HJ_ERR_CUDA,          \
                       "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)
