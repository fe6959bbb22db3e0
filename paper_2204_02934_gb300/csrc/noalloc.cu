// noalloc.cu -- mis2_run_noalloc: MIS-2 without any device or pinned-host
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: processes whose device memory is fully budgeted at start-up
// (a serving process, or a framework whose caching allocator owns the whole
// device), and latency-critical callers for whom a cudaMalloc/cudaFree (which
// may block or synchronise the device) is not acceptable.  The regular entry
// points allocate their scratch in mis2_ctx_create; this one takes its
// scratch from a fixed array in the library's own device image instead.
//
// The scratch below lives in every GPU that loads the library until the
// process exits.  All calls share it and it keeps the last call's contents:
// the counters are cleared at the start of each call, and calls that overlap
// on the GPU (two streams, two host threads) race on it.
#include <cuda.h>  // CUcontext / CUresult types only (see context_id below)

#include <cstring>
#include <mutex>

#include "internal.h"

namespace mis2 {

constexpr int64_t kNoAllocMaxN = MIS2_NOALLOC_MAX_N;
constexpr int64_t kNoAllocTiles = kNoAllocMaxN / 2048 + 4;
// T, M, 2 worklists x 2 buffers x 3 row classes, counters, traces, scan tiles
constexpr int64_t kOffT = 0;
constexpr int64_t kOffM = kOffT + 4 * kNoAllocMaxN;
constexpr int64_t kOffWl = kOffM + 4 * kNoAllocMaxN;
constexpr int64_t kOffCtr = kOffWl + 4 * kNoAllocMaxN * 2 * 2 * kClasses;
constexpr int64_t kOffTrace = kOffCtr + 4 * kCtrWords;
constexpr int64_t kOffTile = kOffTrace + 8 * 2 * MIS2_TRACE_CAP * 4;
constexpr int64_t kNoAllocBytes = kOffTile + 4 * kNoAllocTiles;

static __device__ __align__(256) unsigned char g_mis2_noalloc_scratch[kNoAllocBytes];

// The array's device address belongs to the CUDA context that loaded the
// library's module: a device's primary context normally lives until the
// process exits, but cudaDeviceReset (or a caller that switches to a context
// of its own) brings a new one, where the array can sit elsewhere.  The
// address is therefore looked up once per context and cached under the
// context's unique id (cuCtxGetId; ids are never reused within a process).
// The two driver calls are reached through the runtime's entry-point lookup,
// so the library still links no driver library.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct ScratchSlot {
  unsigned long long ctx_id;
  unsigned char* addr;
};
constexpr int kNoAllocSlots = 64;
static std::mutex g_noalloc_mu;
static ScratchSlot g_noalloc_slots[kNoAllocSlots] = {};
static int g_noalloc_next = 0;
static CtxGetCurrentFn g_ctx_get_current = nullptr;
static CtxGetIdFn g_ctx_get_id = nullptr;

static int driver_entry(const char* name, void** fn) {
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  const cudaError_t e = cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (q != cudaDriverEntryPointSuccess || *fn == nullptr) {
    set_error_text("mis2_run_noalloc: driver entry point not found");
    return MIS2_ERR_CUDA;
  }
  return MIS2_OK;
}

// Unique id of the calling thread's current context (the runtime's primary
// context of the current device unless the caller made another current).
// Called with g_noalloc_mu held.
static int context_id(unsigned long long* id) {
  if (g_ctx_get_current == nullptr) {
    MIS2_TRY(driver_entry("cuCtxGetCurrent", reinterpret_cast<void**>(&g_ctx_get_current)));
    MIS2_TRY(driver_entry("cuCtxGetId", reinterpret_cast<void**>(&g_ctx_get_id)));
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return MIS2_ERR_CUDA;
  if (ctx == nullptr) {
    // no context current yet in this thread: a runtime call that needs the
    // device binds the current device's primary context
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_mis2_noalloc_scratch);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return MIS2_ERR_CUDA;
  }
  if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return MIS2_ERR_CUDA;
  return MIS2_OK;
}

// Device address of the scratch array in the current context (the
// host-side symbol is only a stand-in, never a device address): looked up
// with cudaGetSymbolAddress once per context, with that context current.
static int noalloc_scratch(unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  unsigned long long id = 0;
  MIS2_TRY(context_id(&id));
  for (const ScratchSlot& sl : g_noalloc_slots)
    if (sl.addr != nullptr && sl.ctx_id == id) {
      *out = sl.addr;
      return MIS2_OK;
    }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_mis2_noalloc_scratch);
  if (e != cudaSuccess) return set_cuda_error(e);
  g_noalloc_slots[g_noalloc_next] = ScratchSlot{id, static_cast<unsigned char*>(p)};
  g_noalloc_next = (g_noalloc_next + 1) % kNoAllocSlots;
  *out = static_cast<unsigned char*>(p);
  return MIS2_OK;
}

}  // namespace mis2

using namespace mis2;

extern "C" int mis2_run_noalloc(const mis2_csr* g, uint64_t seed, uint8_t* in_set, int32_t* roots,
                                int64_t* n_roots, int32_t* n_rounds, void* stream) {
  if (g == nullptr || n_roots == nullptr) return MIS2_ERR_INVALID_ARG;
  if (g->n > kNoAllocMaxN) {
    set_error_text("mis2_run_noalloc: graph has more vertices than MIS2_NOALLOC_MAX_N");
    return MIS2_ERR_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  unsigned char* base = nullptr;
  MIS2_TRY(noalloc_scratch(&base));

  // A context on the stack whose scratch pointers all point into the array.
  mis2_ctx c;
  c.device = dev;
  e = cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  mis2_config_default(&c.cfg);
  c.cfg.loop = MIS2_LOOP_DEVICE;
  c.max_n = kNoAllocMaxN;
  c.max_nnz = ((int64_t)1 << 31) - 1;  // colind is caller memory, never copied
  c.s.T = reinterpret_cast<uint32_t*>(base + kOffT);
  c.s.M = reinterpret_cast<uint32_t*>(base + kOffM);
  int32_t* wl = reinterpret_cast<int32_t*>(base + kOffWl);
  for (int b = 0; b < 2; b++)
    for (int k = 0; k < kClasses; k++) {
      c.s.wl1[b][k] = wl + ((0 * 2 + b) * kClasses + k) * kNoAllocMaxN;
      c.s.wl2[b][k] = wl + ((1 * 2 + b) * kClasses + k) * kNoAllocMaxN;
    }
  c.s.ctr = reinterpret_cast<int32_t*>(base + kOffCtr);
  c.s.dtrace = reinterpret_cast<int64_t*>(base + kOffTrace);
  c.s.tile = reinterpret_cast<int32_t*>(base + kOffTile);
  int32_t host_ctr[kCtrWords];
  int64_t host_trace[2 * MIS2_TRACE_CAP * 4];
  c.h_ctr = host_ctr;
  c.h_trace = host_trace;

  GraphArgs ga;
  if (g->n < 0 || g->nnz < 0 || g->nnz >= ((int64_t)1 << 31) || g->rowptr == nullptr ||
      (g->nnz > 0 && g->colind == nullptr) || (g->rowptr_is_64 != 0 && g->rowptr_is_64 != 1) ||
      (reinterpret_cast<uintptr_t>(g->colind) & 3u) != 0)
    return MIS2_ERR_INVALID_ARG;
  ga.n = g->n;
  ga.nnz = g->nnz;
  ga.rp64 = g->rowptr_is_64 != 0;
  ga.rowptr = g->rowptr;
  ga.colind = g->colind;
  ga.vec = (reinterpret_cast<uintptr_t>(g->colind) & 15u) == 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(c.s.ctr, 0, kCtrWords * sizeof(int32_t), st);
  if (e != cudaSuccess) return set_cuda_error(e);
  const int rc = run_impl(&c, ga, make_prio(&c, ga.n, seed), in_set, roots, n_roots, n_rounds, st);
  c.h_ctr = nullptr;  // stack memory: nothing to free
  c.h_trace = nullptr;
  return rc;
}
