// hj_internal.h -- host-side launch interface between the C ABI layer and the
// kernels.  Not installed; not part of the public ABI.
#pragma once

#include <atomic>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "hj_device.cuh"

namespace hjk {

// kernels launched by this library so far (graph replays count every kernel node)
extern std::atomic<unsigned long long> g_launches;

// Threads per block of the stencil kernels.
constexpr int kStageThreads = 256;

// Launch shape of the row-tile stage kernels (DevGrid::tile_rows > 0):
// blocks of ceil(tile_rows * n_last / 32) warps, one block per tile_rows
// lines of the fastest axis, and the shared-memory bytes of one tile.
struct TileShape {
  int threads = 0;
  unsigned blocks = 0;
  size_t smem = 0;
};
constexpr int kTileMaxThreads = 1024;
TileShape tile_shape(const hjd::DevGrid& g, int scheme);
// Whether row tiles of tile_rows lines fit this grid (at most kTileMaxThreads
// nodes per tile, no more lines than the grid has) and every field is
// 16-byte aligned (the staging loads are 16 bytes wide).
bool tile_ok(const hjd::DevGrid& g, int tile_rows, const void* const* fields, int nfields);

// Localized stepping over slabs (hjd::slab_of): the slab lattice is
// s0 x s1, and every slab is a run of nodes_per_slab consecutive nodes.
// Tiles are the blocks of the stage launch: row tiles (g.tile_rows > 0), or
// blocks of `threads` nodes of the flat mapping, `per` of them per slab of
// the flat mapping's grid.
struct LocalLayout {
  int s0 = 1, s1 = 1, nslabs = 1, nodes_per_slab = 1, ntiles = 0, per = 0, threads = 0;
};
LocalLayout local_layout(const hjd::DevGrid& g, int threads);
// From the window's per-slab changes (float bits, nslabs entries): the slab
// masks (3 x nslabs bytes: live, ring2, ring1) and the row-tile lists of the
// three stages (3 x ntiles ints) with their lengths in counts[0..2].  A
// slab steps when one that changed by more than thr lies within k0 slabs
// along the first slab axis and k1 along the second.
cudaError_t launch_local_lists(const hjd::DevGrid& g, int scheme, int threads,
                               const unsigned* slab_resid, float thr, int k0, int k1,
                               unsigned char* masks, int* lists, int* counts, cudaStream_t s);

// Streaming multiprocessors of the current device (read once per device).
int num_sms();
// Blocks of a grid-stride launch over `work` items: enough to cover them,
// capped at 16 blocks per SM of the current device.
unsigned stride_blocks(long long work, int threads);

// One TVD-RK3 stage on one grid.  stage is 1, 2 or 3; scheme 1, 2 or 5;
// threads per block 128, 256 or 512 (other values use 256).  allow_jit:
// grids of at least kJitNodes nodes may run the shape-specialised kernel.
cudaError_t launch_stage(const hjd::DevGrid& g, int scheme, int stage, const hjd::StageArgs& a,
                         cudaStream_t s, int threads = kStageThreads, bool allow_jit = true);

// Shape-specialised stage kernels (hj_jit.cu), compiled at run time for
// grids of at least kJitNodes nodes.  The first sight of (grid shape,
// scheme, threads) starts a background compile; jit_prepare loads a
// finished one (outside any stream capture) and says whether the kernels
// are ready.  jit_launch sets *used when it launched; otherwise the caller
// launches the precompiled one.
constexpr long long kJitNodes = 1ll << 19;
bool jit_wanted(const hjd::DevGrid& g);
bool jit_prepare(const hjd::DevGrid& g, int scheme, int threads);
cudaError_t jit_launch(const hjd::DevGrid& g, int scheme, int stage, const hjd::StageArgs& a,
                       cudaStream_t s, int threads, bool* used);
// Group kernels of a batch (hj_group.cuh): codes[c] is a representative
// grid descriptor of code c, run with schemes[c]; threads per block are
// common to all codes.  The first sight of a composition starts its
// background compile; true (and *handle) once it is loaded.  Must not be
// called inside a stream capture.
bool group_prepare(const std::vector<hjd::DevGrid>& codes, const std::vector<int>& schemes,
                   int threads, void** handle);
// One group launch of stage 1..3 over `blocks` blocks; pack points at a
// hjb::GroupPack, ctl is the device control array.
cudaError_t group_launch(void* handle, int stage, const void* pack, void* ctl, unsigned blocks,
                         int threads, cudaStream_t s);
// Identity of a grid's specialised code: kind, shape, geometry, model
// constants, constraint kind and tile height (the folded fields).
std::string code_key(const hjd::DevGrid& g, int scheme);
bool jit_enabled();
long long jit_compiled();
long long jit_pending();
void jit_enable(int on);
// Per-axis max |f_i| over grid nodes and input vertices, as float bits into out[0..ndim).
// out must be zeroed first.
cudaError_t launch_alpha(const hjd::DevGrid& g, unsigned* out, cudaStream_t s);
// W = l (warm = 0) or W = min(W, l) (warm = 1); snap = W.
cudaError_t launch_init(const hjd::DevGrid& g, float* W, float* snap, int warm, cudaStream_t s);
// Offset of a migration: the target node x reads the source at x - s.
struct Shift {
  double s[4];
  int fill_outside;  // 1: a node whose source point leaves the source box gets l
};
// Wf = min(multilinear(Wc) at x - shift for every target node x, l_target).
// A source point outside the source box sets *bad = 1, or with fill_outside
// gives the node l_target.
cudaError_t launch_prolong(const hjd::DevGrid& c, const float* Wc, const hjd::DevGrid& f,
                           float* Wf, const Shift& sh, int* bad, cudaStream_t s);
// Multilinear value (grad = 0) or node-gradient interpolation (grad = 1) at npts
// points x (device, point-major doubles).  *bad is set to 1 when a point lies
// outside the box.
cudaError_t launch_query(const hjd::DevGrid& g, const float* W, int npts, const double* x,
                         double* out, int* bad, int grad, cudaStream_t s);

// *bad = 1 when some of the n pairs (lo[k], hi[k]) has lo > hi or a non-finite value.
cudaError_t launch_field_check(const float* lo, const float* hi, long long n, int* bad,
                               cudaStream_t s);

// Whether (model, ndim, scheme) has a compiled stencil.
bool stage_supported(int model, int ndim, int scheme);

}  // namespace hjk
