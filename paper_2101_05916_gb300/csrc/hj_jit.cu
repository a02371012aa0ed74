// hj_jit.cu -- stage kernels specialised to one grid shape at run time.
//
// About a third of the stage kernel's instructions are index, address and
// bounds arithmetic on the grid's axis lengths and strides.  For grids of at
// least kJitNodes nodes the library compiles (NVRTC), from the first use on,
// the same stage code with those integers folded in as constants, and keeps
// it for the process.  The compile runs on a background thread; until it is
// loaded the precompiled kernel runs, so no solve waits for it.  Every
// node's floating-point arithmetic is the one of the precompiled kernel;
// only integer index operations fold.  When NVRTC cannot be loaded or a
// compilation fails, the precompiled kernel runs.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hj.h"
#include "hj_grid.h"
#include "hj_internal.h"
#include "hj_group.cuh"

// kJitHeaderNames / kJitHeaders: the device headers as text (build.py)
#include "hj_jit_sources.inc"

#ifndef HJ_CUDA_LIB64
#define HJ_CUDA_LIB64 "/usr/local/cuda/lib64"
#endif

namespace hjk {
namespace {

// NVRTC entry points, loaded with dlopen so that the library does not need
// NVRTC to load.
struct Nvrtc {
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  bool ok = false;
};

const Nvrtc& nvrtc() {
  static Nvrtc n = [] {
    Nvrtc r;
    const char* names[] = {"libnvrtc.so.13", HJ_CUDA_LIB64 "/libnvrtc.so.13", "libnvrtc.so"};
    void* h = nullptr;
    for (const char* nm : names)
      if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!h) return r;
    r.create = (decltype(r.create))dlsym(h, "nvrtcCreateProgram");
    r.compile = (decltype(r.compile))dlsym(h, "nvrtcCompileProgram");
    r.log_size = (decltype(r.log_size))dlsym(h, "nvrtcGetProgramLogSize");
    r.log = (decltype(r.log))dlsym(h, "nvrtcGetProgramLog");
    r.cubin_size = (decltype(r.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
    r.cubin = (decltype(r.cubin))dlsym(h, "nvrtcGetCUBIN");
    r.destroy = (decltype(r.destroy))dlsym(h, "nvrtcDestroyProgram");
    r.ok = r.create && r.compile && r.log_size && r.log && r.cubin_size && r.cubin && r.destroy;
    return r;
  }();
  return n;
}

// Everything folded into a kernel set: the shape, and the geometry and
// model constants that stay fixed while a grid is updated (the disturbance
// bound, alpha and the constraint box stay run-time values).
struct Key {
  int device, ndim, model, scheme, threads, tile_rows, local, con_kind;
  unsigned con_mask;
  int n[hjd::MAXD];
  unsigned geom[5 * hjd::MAXD];  // float bits of lo, h, ih, hih, wfloor
  unsigned prm[8];               // float bits of the model parameters
  bool operator<(const Key& o) const {
    return std::memcmp(this, &o, sizeof(Key)) < 0;
  }
};

unsigned bits(float v) {
  unsigned u;
  std::memcpy(&u, &v, sizeof(u));
  return u;
}

// An exact float literal (hexadecimal).
std::string flit(float v) {
  char buf[64];
  std::snprintf(buf, sizeof(buf), "%af", (double)v);
  return buf;
}

// One kernel set: compiled on a background thread (NVRTC only, no CUDA
// calls there), then loaded on a caller's thread outside any capture.
struct Entry {
  std::atomic<int> state{0};  // 0 compiling, 1 cubin ready, 2 loaded, 3 failed
  std::vector<char> cubin;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t stage[3] = {nullptr, nullptr, nullptr};
};

std::mutex g_mu;
std::map<Key, std::shared_ptr<Entry>> g_cache;
std::atomic<long long> g_compiled{0};
std::atomic<long long> g_pending{0};
std::atomic<int> g_enabled{-1};  // -1: read HJ_JIT from the environment on first use

bool enabled() {
  int e = g_enabled.load();
  if (e < 0) {
    const char* v = std::getenv("HJ_JIT");
    e = (v && v[0] == '0') ? 0 : 1;
    g_enabled.store(e);
  }
  return e == 1;
}

Key key_of(const hjd::DevGrid& g, int scheme, int threads, bool local = false) {
  Key k;
  std::memset(&k, 0, sizeof(k));
  cudaGetDevice(&k.device);
  k.ndim = g.ndim;
  k.model = g.model;
  k.scheme = scheme;
  k.threads = threads;
  k.tile_rows = g.tile_rows;
  k.local = local && g.tile_rows <= 0 ? 1 : 0;
  k.con_kind = g.con_kind;
  k.con_mask = g.con_mask;
  for (int d = 0; d < g.ndim; ++d) {
    k.n[d] = g.n[d];
    k.geom[5 * d + 0] = bits(g.lo[d]);
    k.geom[5 * d + 1] = bits(g.h[d]);
    k.geom[5 * d + 2] = bits(g.ih[d]);
    k.geom[5 * d + 3] = bits(g.hih[d]);
    k.geom[5 * d + 4] = bits(g.wfloor[d]);
  }
  for (int i = 0; i < 8; ++i) k.prm[i] = bits(g.prm[i]);
  return k;
}

// A device function `name` that returns the grid descriptor with its shape,
// geometry, model constants and constraint kind replaced by literals.
std::string fixed_fn(const std::string& name, const hjd::DevGrid& g) {
  std::string s = "__device__ __forceinline__ hjd::DevGrid " + name +
                  "(const hjd::DevGrid& g) {\n  hjd::DevGrid c = g;\n";
  char buf[256];
  for (int d = 0; d < g.ndim; ++d) {
    std::snprintf(buf, sizeof(buf), "  c.n[%d] = %d; c.stride[%d] = %d;\n", d, g.n[d], d,
                  g.stride[d]);
    s += buf;
    s += "  c.lo[" + std::to_string(d) + "] = " + flit(g.lo[d]) + "; c.h[" + std::to_string(d) +
         "] = " + flit(g.h[d]) + "; c.ih[" + std::to_string(d) + "] = " + flit(g.ih[d]) + ";\n";
    s += "  c.hih[" + std::to_string(d) + "] = " + flit(g.hih[d]) + "; c.wfloor[" +
         std::to_string(d) + "] = " + flit(g.wfloor[d]) + ";\n";
  }
  for (int i = 0; i < 8; ++i)
    s += "  c.prm[" + std::to_string(i) + "] = " + flit(g.prm[i]) + ";\n";
  std::snprintf(buf, sizeof(buf), "  c.con_kind = %d; c.con_mask = %uu;\n", g.con_kind,
                g.con_mask);
  s += buf;
  std::snprintf(buf, sizeof(buf),
                "  c.npts = %d; c.plane = %d; c.nrows = %d; c.tile_rows = %d;\n"
                "  c.div_m[0] = %uu; c.div_s[0] = %d;\n"
                "  c.div_m[1] = %uu; c.div_s[1] = %d;\n  c.div_m[2] = %uu; c.div_s[2] = %d;\n"
                "  return c;\n}\n",
                g.npts, g.plane, g.nrows, g.tile_rows, g.div_m[0], g.div_s[0], g.div_m[1],
                g.div_s[1], g.div_m[2], g.div_s[2]);
  s += buf;
  return s;
}

int radius_of(int scheme) { return scheme == 5 ? 3 : (scheme == 2 ? 2 : 1); }

// The stage kernels of stage_kernel (hj_kernels.cu) with the shape fields
// of the grid descriptor replaced by literals.
std::string source(const hjd::DevGrid& g, int scheme, int threads, bool local) {
  std::string s = "#include \"hj_stage.cuh\"\n";
  s += fixed_fn("hj_fixed", g);
  char buf[256];
  if (g.tile_rows > 0) {
    // row tiles: the tile's shared memory is a static array of its exact size
    TileShape ts = tile_shape(g, scheme);
    int pitch = g.n[g.ndim - 1] + 2 * radius_of(scheme);
    for (int st = 1; st <= 3; ++st) {
      std::snprintf(buf, sizeof(buf),
                    "extern \"C\" __global__ void __launch_bounds__(%d)\n"
                    "hj_stage_%d(const hjd::DevGrid g, const hjd::StageArgs a) {\n"
                    "  __shared__ float sm[%d];\n",
                    ts.threads, st, g.tile_rows * pitch);
      s += buf;
      std::snprintf(buf, sizeof(buf), "  hjd::tile_body<%d, %d, %d, %d>(hj_fixed(g), a, sm);\n}\n",
                    g.ndim, scheme, g.model, st);
      s += buf;
    }
    return s;
  }
  // Resident threads per SM: 2048 (32 registers per thread, which the folded
  // kernels fit without spills in stages 1-2) for grids of 2^23 nodes and
  // more, 1536 (40 registers) below.  Measured per WENO5 stage launch: 61^4
  // and 81^4 run 1-1.3 % faster at 2048, 41^4 1.4 % faster at 1536.
  const int per_sm = g.npts >= (1 << 23) ? 2048 : 1536;
  for (int st = 1; st <= 3; ++st) {
    std::snprintf(buf, sizeof(buf),
                  "extern \"C\" __global__ void __launch_bounds__(%d, %d)\n"
                  "hj_stage_%d(const hjd::DevGrid g, const hjd::StageArgs a) {\n",
                  threads, std::max(1, per_sm / threads), st);
    s += buf;
    std::snprintf(buf, sizeof(buf), "  hjd::flat_body<%d, %d, %d, %d, %s>(hj_fixed(g), a);\n}\n",
                  g.ndim, scheme, g.model, st, local ? "true" : "false");
    s += buf;
  }
  return s;
}

// The group kernels of a batch: one kernel per RK stage over the blocks of
// every position of a hjb::GroupPack (the flat mapping, `threads` per
// block).  Position i holds a grid like grids[i] (kind, shape and model
// constants folded in) run with schemes[i]; its body reads the position's
// descriptor and stage arguments with a literal index.
std::string group_source(const std::vector<hjd::DevGrid>& grids, const std::vector<int>& schemes,
                         int threads) {
  std::string s = "#include \"hj_group.cuh\"\n";
  for (size_t c = 0; c < grids.size(); ++c) s += fixed_fn("hj_fixed_" + std::to_string(c), grids[c]);
  char buf[1024];
  const int npos = (int)grids.size();
  for (int st = 1; st <= 3; ++st) {
    // 2048 threads per SM at 32 registers, as the single-grid stage kernels
    // (without the bound the position switch of stage 3 takes 48 registers)
    std::snprintf(buf, sizeof(buf),
                  "extern \"C\" __global__ void __launch_bounds__(%d, %d)\n"
                  "hj_group_%d(const __grid_constant__ hjb::GroupPack pack, hjb::Ctl* ctl) {\n"
                  "  const int b = (int)blockIdx.x;\n  int k = 0;\n",
                  threads, std::max(1, 2048 / threads), st);
    s += buf;
    // the block's position: the last one whose first block is not after it
    // (positions without blocks share their successor's first block)
    for (int c = 1; c < npos; ++c) {
      std::snprintf(buf, sizeof(buf), "  if (b >= pack.block_begin[%d]) k = %d;\n", c, c);
      s += buf;
    }
    s += "  switch (k) {\n";
    for (int c = 0; c < npos; ++c) {
      std::snprintf(buf, sizeof(buf),
                    "    case %d: {\n"
                    "      const int slot = pack.items[%d].slot;\n"
                    "      if (!ctl[slot].active) return;\n"
                    "      const int lb = b - pack.block_begin[%d];\n"
                    "      const int yb = pack.items[%d].bx >= 2 ? hjd::fast_div(lb, pack.items[%d].bx_m,"
                    " pack.items[%d].bx_s) : lb;\n"
                    "      const int bx = lb - yb * pack.items[%d].bx;\n"
                    "      const bool check = %s;\n"
                    "      hjd::StageArgs a = pack.items[%d].a[%d];\n"
                    "      a.check = check ? 1 : 0;\n      a.resid = &ctl[slot].resid;\n",
                    c, c, c, c, c, c, c, st == 3 ? "ctl[slot].check_next != 0" : "false", c,
                    st - 1);
      s += buf;
      std::snprintf(buf, sizeof(buf),
                    "      unsigned r = hjd::stage_point<%d, %d, %d, %d>(hj_fixed_%d(pack.items[%d].g),"
                    " a, bx * %d + (int)threadIdx.x, yb, check);\n"
                    "      %s\n      return;\n    }\n",
                    grids[c].ndim, schemes[c], grids[c].model, st, c, c, threads,
                    st == 3 ? "if (check) hjd::block_max_bits(r, a.resid);" : "(void)r;");
      s += buf;
    }
    s += "  }\n}\n";
  }
  return s;
}

// NVRTC compile of one kernel set (no CUDA calls).  *log, when given,
// receives NVRTC's log.
// verbose: ptxas reports each kernel's registers and spills into the log.
std::vector<char> compile(const std::string& src, std::string* log = nullptr,
                          bool verbose = false) {
  std::vector<char> cubin;
  const Nvrtc& n = nvrtc();
  if (!n.ok) return cubin;
  nvrtcProgram prog = nullptr;
  int nh = (int)(sizeof(kJitHeaders) / sizeof(kJitHeaders[0]));
  if (n.create(&prog, src.c_str(), "hj_stage_jit.cu", nh, kJitHeaders, kJitHeaderNames) !=
      NVRTC_SUCCESS)
    return cubin;
  const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-ftz=true", "-lineinfo",
                        "--ptxas-options=-v"};
  size_t sz = 0;
  nvrtcResult rc = n.compile(prog, verbose ? 5 : 4, opts);
  if (log) {
    size_t ls = 0;
    if (n.log_size(prog, &ls) == NVRTC_SUCCESS && ls > 1) {
      std::vector<char> buf(ls);
      if (n.log(prog, buf.data()) == NVRTC_SUCCESS) log->assign(buf.data());
    }
  }
  if (rc == NVRTC_SUCCESS && n.cubin_size(prog, &sz) == NVRTC_SUCCESS && sz > 0) {
    cubin.resize(sz);
    if (n.cubin(prog, cubin.data()) != NVRTC_SUCCESS) cubin.clear();
  }
  n.destroy(&prog);
  return cubin;
}

// At most kMaxCompiles compiles run at once: a server that meets many new
// shapes must not take every host core from its own thread.
constexpr int kMaxCompiles = 4;
std::mutex g_slot_mu;
std::condition_variable g_slot_cv;
int g_slots_used = 0;

// Exit waits (bounded) for compiles still running, so that none is inside
// NVRTC while the process tears its libraries down.  Registered on the first
// compile, i.e. after NVRTC was loaded, so it runs before NVRTC's teardown.
void wait_pending_at_exit() {
  for (int i = 0; i < 6000 && g_pending.load() > 0; ++i)
    std::this_thread::sleep_for(std::chrono::milliseconds(10));
}

void compile_async(std::shared_ptr<Entry> e, std::string src) {
  static const bool registered = (std::atexit(wait_pending_at_exit), true);
  (void)registered;
  g_pending.fetch_add(1);
  std::thread([e, src] {
    {
      std::unique_lock<std::mutex> lk(g_slot_mu);
      g_slot_cv.wait(lk, [] { return g_slots_used < kMaxCompiles; });
      ++g_slots_used;
    }
    e->cubin = compile(src);
    e->state.store(e->cubin.empty() ? 3 : 1);
    {
      std::lock_guard<std::mutex> lk(g_slot_mu);
      --g_slots_used;
    }
    g_slot_cv.notify_one();
    g_pending.fetch_sub(1);
  }).detach();
}

// Load a compiled set on this thread (never inside a capture).
void load(Entry& e, const char* prefix = "hj_stage_") {
  if (cudaLibraryLoadData(&e.lib, e.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) !=
      cudaSuccess) {
    cudaGetLastError();
    e.lib = nullptr;
    e.state.store(3);
    return;
  }
  for (int st = 0; st < 3; ++st) {
    char name[32];
    std::snprintf(name, sizeof(name), "%s%d", prefix, st + 1);
    if (cudaLibraryGetKernel(&e.stage[st], e.lib, name) != cudaSuccess) {
      cudaGetLastError();
      cudaLibraryUnload(e.lib);
      e.lib = nullptr;
      e.state.store(3);
      return;
    }
  }
  e.cubin.clear();
  e.state.store(2);
  g_compiled.fetch_add(1);
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// The entry of (grid shape, scheme, threads): started on first sight,
// loaded once compiled when `may_load`.  Returns it when loaded.
Entry* lookup(const hjd::DevGrid& g, int scheme, int threads, bool may_load, bool local = false) {
  Key k = key_of(g, scheme, threads, local);
  std::shared_ptr<Entry> e;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(k);
    if (it == g_cache.end()) {
      e = std::make_shared<Entry>();
      g_cache.emplace(k, e);
      if (!nvrtc().ok) {
        e->state.store(3);
        return nullptr;
      }
      compile_async(e, source(g, scheme, threads, k.local != 0));
      return nullptr;
    }
    e = it->second;
  }
  int st = e->state.load();
  if (st == 1 && may_load) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (e->state.load() == 1) load(*e);
    st = e->state.load();
  }
  return st == 2 ? e.get() : nullptr;
}

std::map<std::string, std::shared_ptr<Entry>> g_group_cache;

}  // namespace

bool group_prepare(const std::vector<hjd::DevGrid>& codes, const std::vector<int>& schemes,
                   int threads, void** handle) {
  *handle = nullptr;
  if (!enabled() || codes.empty()) return false;
  std::string key = std::to_string(threads) + "/";
  for (size_t c = 0; c < codes.size(); ++c) {
    Key k = key_of(codes[c], schemes[c], threads);
    key.append(reinterpret_cast<const char*>(&k), sizeof(k));
  }
  std::shared_ptr<Entry> e;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_group_cache.find(key);
    if (it == g_group_cache.end()) {
      e = std::make_shared<Entry>();
      g_group_cache.emplace(key, e);
      if (!nvrtc().ok) {
        e->state.store(3);
        return false;
      }
      compile_async(e, group_source(codes, schemes, threads));
      return false;
    }
    e = it->second;
  }
  int st = e->state.load();
  if (st == 1) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (e->state.load() == 1) load(*e, "hj_group_");
    st = e->state.load();
  }
  if (st != 2) return false;
  *handle = e.get();
  return true;
}

cudaError_t group_launch(void* handle, int stage, const void* pack, void* ctl, unsigned blocks,
                         int threads, cudaStream_t s) {
  Entry* e = static_cast<Entry*>(handle);
  void* ctlp = ctl;
  void* args[] = {const_cast<void*>(pack), (void*)&ctlp};
  cudaError_t err = cudaLaunchKernel((const void*)e->stage[stage - 1], dim3(blocks, 1, 1),
                                     dim3(threads, 1, 1), args, 0, s);
  if (err == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
  return err;
}

std::string code_key(const hjd::DevGrid& g, int scheme) {
  Key k = key_of(g, scheme, 0);
  k.device = 0;
  return std::string(reinterpret_cast<const char*>(&k), sizeof(k));
}

bool jit_enabled() { return enabled(); }

bool jit_wanted(const hjd::DevGrid& g) {
  return (long long)g.npts >= kJitNodes && enabled();
}

bool jit_prepare(const hjd::DevGrid& g, int scheme, int threads) {
  if (!jit_wanted(g)) return false;
  return lookup(g, scheme, threads, true) != nullptr;
}

cudaError_t jit_launch(const hjd::DevGrid& g, int scheme, int stage, const hjd::StageArgs& a,
                       cudaStream_t s, int threads, bool* used) {
  *used = false;
  if (!jit_wanted(g)) return cudaSuccess;
  bool local = a.tiles || a.live || a.slab_resid;
  Entry* e = lookup(g, scheme, threads, !capturing(s), local);
  if (!e) return cudaSuccess;
  dim3 grid, block;
  if (g.tile_rows > 0) {
    TileShape ts = tile_shape(g, scheme);
    grid = dim3(a.tiles ? (unsigned)a.ntiles : ts.blocks, 1, 1);
    block = dim3(ts.threads, 1, 1);
  } else if (a.tiles) {
    grid = dim3((unsigned)a.ntiles, 1, 1);
    block = dim3(threads, 1, 1);
  } else {
    grid = dim3((unsigned)((g.plane + threads - 1) / threads), g.ndim == 4 ? (unsigned)g.n[0] : 1u,
                1);
    block = dim3(threads, 1, 1);
  }
  void* args[] = {(void*)&g, (void*)&a};
  cudaError_t err = cudaLaunchKernel((const void*)e->stage[stage - 1], grid, block, args, 0, s);
  if (err == cudaSuccess) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    *used = true;
  }
  return err;
}

long long jit_compiled() { return g_compiled.load(); }

long long jit_pending() { return g_pending.load(); }

void jit_enable(int on) { g_enabled.store(on ? 1 : 0); }

}  // namespace hjk

static hj_status jit_check(int ndim, const int* n, int model, int scheme, int threads,
                           int tile_rows, int* max_registers = nullptr,
                           int* max_spill_bytes = nullptr, unsigned con_axes = ~0u);

extern "C" hj_status hj_jit_check(int ndim, const int* n, int model, int scheme, int threads) {
  return jit_check(ndim, n, model, scheme, threads, 0);
}

extern "C" hj_status hj_jit_check_resources(int ndim, const int* n, int model, int scheme,
                                            int threads, unsigned con_axes, int* max_registers,
                                            int* max_spill_bytes) {
  if (!max_registers || !max_spill_bytes) return hja::fail(HJ_ERR_ARG, "NULL output");
  if (ndim < 1 || ndim > HJ_MAX_DIM || con_axes == 0u || (con_axes >> ndim) != 0u)
    return hja::fail(HJ_ERR_ARG, "con_axes must name at least one of the grid's axes");
  return jit_check(ndim, n, model, scheme, threads, 0, max_registers, max_spill_bytes, con_axes);
}

// The largest register count and spill-store size over the kernels of a
// ptxas -v log ("Used N registers", "N bytes spill stores").
static void parse_resources(const std::string& log, int* regs, int* spill) {
  *regs = -1;
  *spill = 0;
  size_t pos = 0;
  while ((pos = log.find("Used ", pos)) != std::string::npos) {
    int v = 0;
    if (std::sscanf(log.c_str() + pos, "Used %d registers", &v) == 1) *regs = std::max(*regs, v);
    pos += 5;
  }
  pos = 0;
  const std::string key = " bytes spill stores";
  while ((pos = log.find(key, pos)) != std::string::npos) {
    size_t b = pos;
    while (b > 0 && log[b - 1] >= '0' && log[b - 1] <= '9') --b;
    if (b < pos) *spill = std::max(*spill, std::atoi(log.c_str() + b));
    pos += key.size();
  }
}

extern "C" hj_status hj_jit_check_tiles(int ndim, const int* n, int model, int scheme,
                                        int tile_rows) {
  if (tile_rows <= 0) return hja::fail(HJ_ERR_ARG, "tile_rows must be > 0");
  return jit_check(ndim, n, model, scheme, 256, tile_rows);
}

static hj_status jit_check(int ndim, const int* n, int model, int scheme, int threads,
                           int tile_rows, int* max_registers, int* max_spill_bytes,
                           unsigned con_axes) {
  if (ndim < 1 || ndim > HJ_MAX_DIM || !n) return hja::fail(HJ_ERR_ARG, "bad grid shape");
  if (model != HJ_DRIFT && model != HJ_QUAD_Z && model != HJ_QUAD_X4)
    return hja::fail(HJ_ERR_ARG, "unknown model %d", model);
  if (scheme != HJ_FIRST && scheme != HJ_ENO2 && scheme != HJ_WENO5)
    return hja::fail(HJ_ERR_ARG, "unknown scheme %d", scheme);
  if (threads != 128 && threads != 256 && threads != 512)
    return hja::fail(HJ_ERR_ARG, "threads must be 128, 256 or 512");
  // a grid description on the stack over [0, 1]^ndim with a box constraint:
  // enough for the descriptor; no device memory is touched
  hj_grid_s g;
  g.ndim = ndim;
  long long npts = 1;
  for (int i = 0; i < ndim; ++i) {
    if (n[i] < 3) return hja::fail(HJ_ERR_ARG, "axis %d has fewer than 3 nodes", i);
    g.n[i] = n[i];
    g.lo[i] = 0.0;
    g.hi[i] = 1.0;
    g.h[i] = 1.0 / (double)(n[i] - 1);
    const bool con = (con_axes >> i) & 1u;
    g.ca[i] = con ? 0.25 : -INFINITY;
    g.cb[i] = con ? 0.75 : INFINITY;
    npts *= n[i];
  }
  if (npts >= (1ll << 31)) return hja::fail(HJ_ERR_ARG, "grid too large");
  g.npts = npts;
  g.model = model;
  g.con_kind = hjd::C_BOX;
  g.tile_rows = tile_rows;
  hjd::DevGrid d = hja::devgrid(&g);
  if (tile_rows > 0 && ((long long)tile_rows * n[ndim - 1] > hjk::kTileMaxThreads ||
                        tile_rows > d.nrows))
    return hja::fail(HJ_ERR_ARG, "row tile does not fit the grid");
  if (!hjk::nvrtc().ok) return hja::fail(HJ_ERR_CUDA, "NVRTC could not be loaded");
  std::string log;
  const bool verbose = max_registers != nullptr;
  std::vector<char> cubin = hjk::compile(hjk::source(d, scheme, threads, false), &log, verbose);
  if (cubin.empty()) return hja::fail(HJ_ERR_CUDA, "NVRTC: %.400s", log.c_str());
  if (verbose) {
    parse_resources(log, max_registers, max_spill_bytes);
    if (*max_registers < 0) return hja::fail(HJ_ERR_CUDA, "no ptxas resource report in the log");
  }
  return HJ_OK;
}

extern "C" hj_status hj_jit_check_group(int ngrids, const int* ndims, const int* shapes,
                                        const int* models, const int* schemes) {
  if (ngrids < 1 || ngrids > hjb::kGroupItems || !ndims || !shapes || !models || !schemes)
    return hja::fail(HJ_ERR_ARG, "bad group description");
  std::vector<hjd::DevGrid> codes;
  std::vector<int> sch;
  for (int k = 0; k < ngrids; ++k) {
    int nd = ndims[k];
    if (nd < 1 || nd > HJ_MAX_DIM) return hja::fail(HJ_ERR_ARG, "bad ndim");
    hj_grid_s g;
    g.ndim = nd;
    long long npts = 1;
    for (int i = 0; i < nd; ++i) {
      int n = shapes[4 * k + i];
      if (n < 3) return hja::fail(HJ_ERR_ARG, "axis with fewer than 3 nodes");
      g.n[i] = n;
      g.lo[i] = 0.0;
      g.hi[i] = 1.0;
      g.h[i] = 1.0 / (double)(n - 1);
      g.ca[i] = 0.25;
      g.cb[i] = 0.75;
      npts *= n;
    }
    if (npts >= (1ll << 31)) return hja::fail(HJ_ERR_ARG, "grid too large");
    g.npts = npts;
    g.model = models[k];
    g.con_kind = hjd::C_BOX;
    if (!hjk::stage_supported(models[k], nd, schemes[k]))
      return hja::fail(HJ_ERR_ARG, "model %d, %d-D, scheme %d has no stencil", models[k], nd,
                       schemes[k]);
    codes.push_back(hja::devgrid(&g));
    sch.push_back(schemes[k]);
  }
  if (!hjk::nvrtc().ok) return hja::fail(HJ_ERR_CUDA, "NVRTC could not be loaded");
  std::string log;
  std::vector<char> cubin = hjk::compile(hjk::group_source(codes, sch, hjb::kGroupThreads), &log);
  if (cubin.empty()) return hja::fail(HJ_ERR_CUDA, "NVRTC: %.400s", log.c_str());
  return HJ_OK;
}
