// internal.h -- host-side context and the launchers shared by the
// translation units of the library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <mutex>
#include <utility>
#include <string>
#include <vector>

#include "common.cuh"

namespace mis2 {

// A named range on a profiler's NVTX timeline (ncu --nvtx filters kernels by
// it): pushed for the scope, popped at its end; without a profiler attached
// the calls do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ------------------------------------------------------------- counter words
// Worklist sizes rotate over three slots per round r: input slot r%3, output
// slot (r+1)%3, and slot (r+2)%3 is cleared during round r for round r+1.
__host__ __device__ inline int ctr_c1(int slot, int cls) { return slot * kClasses + cls; }
__host__ __device__ inline int ctr_c2(int slot, int cls) { return 9 + slot * kClasses + cls; }
enum : int {
  kCtrRoots = 18,    // |MIS-2| from the root compaction
  kCtrM2 = 19,       // phase-2 MIS-2 size
  kCtrQual = 20,     // qualifying phase-2 roots
  kCtrHeavy = 21,    // deferred heavy rows
  kCtrLeft = 22,     // phase-3 leftovers (group rows)
  kCtrLeftHeavy = 23,
  kCtrLarge = 24,    // coarse rows needing the block path
  kCtrCnnz = 25,     // coarse nnz
  kCtrErr = 26,      // device error flags (bit 0: barrier timeout)
  kCtrRounds = 27,   // rounds of the device loop
  kCtrBarrier = 28,  // grid barrier: monotonic arrival count (28) and its value at the launch's start (29)
  kCtrLeftMid = 30,  // phase-3 leftovers of medium degree
  kCtrHeavy2 = 31,   // deferred heavy rows of the phase-2 claims (async level path)
  kCtrRounds2 = 32,  // rounds of the phase-2 device loop
  kCtrLargeKb = 33,  // large aggregates handled in the first bitmap batch
  kCtrGiant = 34,    // giant member rows of the current bitmap batch
  kCtrLeftLong = 35,  // phase-3 medium leftovers too long for a warp
  kCtrCheckSums = 36,  // debug checks: two 64-bit entry-hash sums (words 36-39)
  kCtrInitSizes = 40,  // no-worklist mode of the host loop: round-0 list sizes (words 40-45)
  kCtrColorLeft = 48,  // colouring: uncoloured count after each round of a batch (words 48-55)
  kCtrCoarseRest = 56,  // coarse graph: aggregates left to the hash-set kernel
  kCtrWords = 64
};
constexpr int kReadbackWords = 40;
// Member rows of large aggregates longer than this are split into pieces of
// this many entries, spread over the grid (coarse graph).
constexpr int kGiantRow = 4096;
// device error flags (ctr[kCtrErr])
// kErrLargeOverflow: more large aggregates than one bitmap batch holds, seen
// by the single-batch coarse path (the caller finishes the other batches).
enum : int {
  kErrTimeout = 1,
  kErrNoAggregatedNeighbour = 2,
  kErrNoProgress = 4,
  kErrCapacity = 8,
  kErrLargeOverflow = 16,
  kErrBadGraph = 32  // debug checks: malformed or asymmetric CSR, roots not distance-2 independent
};
constexpr int kLoopTsWords = MIS2_LOOP_TS_WORDS;

enum KernelClass : int {
  kKcInit = 0,
  kKcColumn = 1,
  kKcDecide = 2,
  kKcCompact = 3,
  kKcAggregate = 4,
  kKcCoarse = 5,
  kKcDeviceLoop = 6,
  kKcOther = 7
};

struct Scratch {
  uint32_t* T = nullptr;
  uint32_t* M = nullptr;
  int32_t* wl1[2][kClasses] = {};
  int32_t* wl2[2][kClasses] = {};
  int32_t* ctr = nullptr;
  int64_t* dtrace = nullptr;  // [2][MIS2_TRACE_CAP][4]
  int64_t* loop_ts = nullptr;  // [2][kLoopTsWords] device-loop barrier timestamps
  int32_t* tile = nullptr;
  int32_t* roots2 = nullptr;
  int32_t* qlist = nullptr;
  uint8_t* qflag = nullptr;
  int32_t* tent = nullptr;
  int32_t* aggsize = nullptr;
  int32_t* left = nullptr;
  int32_t* left_heavy = nullptr;
  int32_t* left_mid = nullptr;
  int32_t* roots_tmp = nullptr;  // root list when the caller passes none
  int32_t* agg_cnt = nullptr;
  int32_t* agg_ptr = nullptr;
  int32_t* ub = nullptr;
  int32_t* ub_ptr = nullptr;
  int32_t* cursor = nullptr;
  int32_t* members = nullptr;
  int32_t* c_cnt = nullptr;
  int32_t* large = nullptr;
  int32_t* tmp = nullptr;        // coarse rows before packing (max_nnz)
  uint32_t* bitmaps = nullptr;   // coarse graph: bitmaps over aggregate ids for large aggregates
  int64_t* chunk_off = nullptr;  // coarse graph: member-chunk offsets of a batch of large aggregates
  int32_t* giant_v = nullptr;     // coarse graph: member rows longer than kGiantRow of a bitmap batch,
  int32_t* giant_slot = nullptr;  //   their bitmap slot,
  int64_t* giant_off = nullptr;   //   and their piece offsets (capacity nnz / kGiantRow + 1)
  int32_t* labels_tmp = nullptr; // labels when the caller passes none
  int32_t* radix = nullptr;       // stable grouping: per-tile digit counts (group_scratch_words)
  int4* cand = nullptr;           // coarse graph: up to twelve neighbour labels per vertex (3n)
};

struct HostStage {  // device copies for the host-buffer entry point
  void* rowptr = nullptr;
  int32_t* colind = nullptr;
  uint8_t* in_set = nullptr;
  int32_t* roots = nullptr;
  int32_t* labels = nullptr;
  int32_t* c_rowptr = nullptr;
  int32_t* c_colind = nullptr;
  int64_t cap_n = 0, cap_nnz = 0;
};

struct Timer {
  std::vector<cudaEvent_t> ev;
  std::vector<int> cls;
  size_t used = 0;
};

}  // namespace mis2

struct mis2_ctx {
  int device = 0;
  int sm_count = 0;
  int64_t max_n = 0, max_nnz = 0;
  mis2_config cfg{};
  mis2_stats stats{};
  mis2::Scratch s;
  mis2::HostStage stage;
  int32_t* h_ctr = nullptr;  // pinned readback of counter words
  int64_t* h_trace = nullptr;  // pinned readback of the traces
  mis2::Timer timer;
  std::vector<void*> allocations;
  int device_loop_blocks = 0;  // co-resident blocks of the device-loop kernel
  int64_t launches = 0;        // kernels launched by the current call
  // Contexts whose streams run concurrently (server slots) share this lock:
  // a device-loop launch holds it until the kernel has finished, so at most
  // one grid-synchronised kernel of theirs is resident at a time.
  std::mutex* coop_lock = nullptr;
  cudaEvent_t coop_done = nullptr;
  cudaEvent_t ev_counts = nullptr;  // a level's counter readback, waited on while later work runs
  // mis2_run_snapshots: per-round copies of T and M (device; null otherwise)
  uint32_t* snaps = nullptr;
  int32_t snap_rounds = 0;
};

namespace mis2 {

// Graph as the launchers see it.
struct GraphArgs {
  int64_t n, nnz;
  bool rp64;
  const void* rowptr;
  const int32_t* colind;
  bool vec;
};

int set_cuda_error(cudaError_t e);
void set_error_text(const char* msg);
#define MIS2_CUDA(call)                                     \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return ::mis2::set_cuda_error(_e); \
  } while (0)
#define MIS2_TRY(call)               \
  do {                               \
    int _rc = (call);                \
    if (_rc != MIS2_OK) return _rc;  \
  } while (0)

// timing helpers: bracket a launch with events when cfg.timing is set
void timer_begin(mis2_ctx* c, int cls, cudaStream_t st);
void timer_end(mis2_ctx* c, cudaStream_t st);
void timer_reset(mis2_ctx* c);
int timer_collect(mis2_ctx* c);

// Row mapping of the MIS-2 loops: lanes per low-degree row and the degree
// from which a row gets a warp (cfg values when set, else from the average
// degree).
int pick_group_lanes(const mis2_ctx* c, const GraphArgs& g);
int pick_warp_degree(const mis2_ctx* c, const GraphArgs& g);
int grid_for(const mis2_ctx* c, int64_t items, int items_per_block, int blocks_per_sm = 8);
// Launch of the short kernels around the MIS-2 loops: with programmatic
// stream serialisation (unless the configuration asks for serial launches or
// per-kernel timing) a kernel may be scheduled while the one before it in
// the stream finishes, which hides most of the gap between dependent
// launches; each kernel started here begins with pdl_enter().  Errors
// surface through cudaGetLastError, as with <<< >>>.
template <typename... P, typename... A>
inline void launch_k(const mis2_ctx* c, void (*k)(P...), int grid, int block, cudaStream_t st, A&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)grid);
  lc.blockDim = dim3((unsigned)block);
  lc.dynamicSmemBytes = 0;
  lc.stream = st;
  lc.attrs = at;
  lc.numAttrs = (c->cfg.serial_launches == 0 && c->cfg.timing != MIS2_TIMING_ALL) ? 1 : 0;
  (void)cudaLaunchKernelEx(&lc, k, std::forward<A>(args)...);
}
// Resident blocks per SM of a kernel at `block` threads and `smem` bytes of
// dynamic shared memory on the context's device
// (cudaOccupancyMaxActiveBlocksPerMultiprocessor), asked once per (kernel,
// device, block, smem) and remembered, so a persistent launch pays no
// host-side query.  Raises the kernel's dynamic shared memory limit to
// `smem` first when it exceeds the default 48 KB.
int resident_blocks_per_sm(const mis2_ctx* c, const void* kernel, int block, int* per_sm, int smem = 0);

// MIS-2 of g (labels == null) or of {v : labels[v] == -1}; leaves T with
// IN/OUT.  trace_phase 0/1 selects the trace slot.  Host-driven loop.
int mis2_rounds_host(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const PrioCfg& p,
                     int trace_phase, cudaStream_t st, int32_t* rounds);
// Same through the persistent device-loop kernel.
int mis2_rounds_device(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const PrioCfg& p,
                       int trace_phase, cudaStream_t st, int32_t* rounds);
// Device loop without host synchronisation: rounds go to ctr[rounds_slot],
// errors accumulate in ctr[kCtrErr] (cleared by the caller).
int mis2_rounds_device_async(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const PrioCfg& p,
                             int trace_phase, int rounds_slot, cudaStream_t st);
// Per-aggregate member counts and summed member row lengths of the coarse
// graph (its histogram), accumulated by the level path's aggregation
// kernels when not null.
struct AggCounts {
  int32_t* cnt = nullptr;
  int32_t* deg = nullptr;
};
// Arrays of n words the root compaction also initialises (null: none):
// minus1[v] = -1, zero[k][v] = 0 (the level path's frozen labels and
// per-aggregate counters, set in the pass that visits every vertex anyway).
struct LevelFill {
  int32_t* minus1 = nullptr;
  int32_t* zero[3] = {nullptr, nullptr, nullptr};
};
// Ordered compaction of {v : T_v = IN}: ascending roots, flags, count on
// device at *count_dev; fills `fill`.
int extract_in_set(mis2_ctx* c, int64_t n, uint8_t* flags, int32_t* roots, int32_t* count_dev,
                   cudaStream_t st, const LevelFill& fill = LevelFill{});
// Exclusive scan of vals[0, n) into out[0, n], out[n] = total; total also
// stored at *total_dev, and out[0, n) copied to out2, when not null.
int exclusive_scan_i32(mis2_ctx* c, const int32_t* vals, int64_t n, int32_t* out, int32_t* total_dev,
                       cudaStream_t st, int32_t* out2 = nullptr);
// Ordered compaction of indices j < n with flags[j] != 0 mapped through
// map[j] (map null: j itself) into out; count to *count_dev.
int compact_flags(mis2_ctx* c, const uint8_t* flags, const int32_t* map, int64_t n, int32_t* out,
                  int32_t* count_dev, cudaStream_t st);

// Aggregation phases (Algorithm 3), exposed for the batched engine.
int agg_phase1(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, int64_t n_roots, int32_t* labels,
               cudaStream_t st);
int agg_phase2(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, int32_t* labels, int32_t label_base,
               int32_t* rounds2, int64_t* nq, cudaStream_t st);
int agg_phase3(mis2_ctx* c, const GraphArgs& g, int32_t* labels, int64_t total, cudaStream_t st);
// Sync-free variants: counts stay on the device (roots count at
// ctr[kCtrRoots], qualifying phase-2 roots at ctr[kCtrQual]); errors in
// ctr[kCtrErr].
int agg_level_async(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, const PrioCfg& p, int mode, int32_t* labels,
                    cudaStream_t st);
// Coarse graph without host synchronisation; the caller synchronises, reads
// the counters into c->h_ctr and checks coarsen_fast_needs_retry (more large
// aggregates than one batch of bitmaps: coarsen_fast_finish completes the
// result) and kErrCapacity (c_colind too small) before trusting the result.
// ctr_fresh: the coarse graph's counter words are still zero from the
// level's start (not cleared again here).
int coarsen_fast(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                 int32_t* c_colind, int64_t c_colind_cap, cudaStream_t st, bool prelude_done = false,
                 bool cand_ready = false, bool ctr_fresh = false);
// The labels-only first steps of coarsen_fast, queued before n_aggs is known
// on the host (then pass prelude_done = true and the returned cand_ready).
// hist_done: the aggregation already left the histogram (s.agg_cnt, s.ub).
int coarsen_prelude(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, bool* cand_ready, cudaStream_t st,
                    bool hist_done = false);
bool coarsen_fast_needs_retry(const mis2_ctx* c);
// Debug-mode validation (synchronises): MIS2_ERR_BAD_GRAPH for a malformed or
// asymmetric CSR, or for roots that are not ascending and pairwise more than
// two hops apart.
int check_graph(mis2_ctx* c, const GraphArgs& g, cudaStream_t st);
int check_roots(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, int64_t n_roots, cudaStream_t st);
int check_labels(mis2_ctx* c, const int32_t* labels, int64_t n, int64_t n_aggs, cudaStream_t st);
int coarse_weights_impl(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const int32_t* c_rowptr,
                        const int32_t* c_colind, int64_t c_nnz, int32_t* c_weights, cudaStream_t st);
int misk_impl(mis2_ctx* c, const GraphArgs& g, int k, const PrioCfg& p, uint8_t* in_set, int32_t* roots,
              int64_t* n_roots, int32_t* n_rounds, cudaStream_t st);
// Rows by length: light (<= light_max entries) for the G-lanes-per-row
// kernels, medium (up to heavy_min) for a warp each, heavy (longer) for a
// block each.  The lists are ascending; counts on the host and the device.
// Uses the scratch arrays qflag, aggsize, left_mid, large.  Synchronises.
struct LenLists {
  const int32_t* medium = nullptr;
  const int32_t* heavy = nullptr;
  const int32_t* n_medium_dev = nullptr;
  const int32_t* n_heavy_dev = nullptr;
  int32_t n_medium = 0, n_heavy = 0;
};
int classify_rows(mis2_ctx* c, const GraphArgs& g, int64_t light_max, int64_t heavy_min, LenLists* rl,
                  cudaStream_t st);
// Stable grouping of 0..n-1 by keys[i] in [0, n_keys): ptr[n_keys + 1],
// list[n] (each key's indices ascending).  Keys outside the range set
// kErrBadGraph in ctr[kCtrErr] (read by the caller).  Asynchronous; uses the
// scratch arrays M, roots2, tent, qlist, radix.
int64_t group_scratch_words(int64_t n);
int group_by_key(mis2_ctx* c, const int32_t* keys, int64_t n, int64_t n_keys, int32_t* ptr, int32_t* list,
                 cudaStream_t st);
// Algorithm 1 through the plain tuple engine (the packed-tuple ablation):
// packed (Eq. 1, the same MIS-2 as mis2_run) or unpacked (status, priority,
// id) tuples.  Fills in_set / roots like mis2_run; synchronises.
int tuple_engine_impl(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, bool unpacked, uint8_t* in_set,
                      int32_t* roots, int64_t* n_roots, int32_t* n_rounds, cudaStream_t st);
int color_impl(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, int32_t* colors, int32_t* color_ptr,
               int32_t* color_list, int32_t* n_colors, int32_t* n_rounds, cudaStream_t st);
int prolongator_impl(mis2_ctx* c, const int32_t* labels, int64_t n, int64_t n_aggs, int normalize,
                     int32_t* p_rowptr, int32_t* p_colind, double* p_values, cudaStream_t st);
int coarsen_fast_finish(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                        int32_t* c_colind, int64_t c_colind_cap, int64_t* c_nnz, cudaStream_t st);
int aggregate_impl(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, int64_t n_roots, uint64_t seed,
                   int mode, int32_t* labels, int64_t* n_aggs, cudaStream_t st);
int coarsen_impl(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                 int32_t* c_colind, int64_t c_colind_cap, int64_t* c_nnz, cudaStream_t st);
int run_impl(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, uint8_t* in_set, int32_t* roots,
             int64_t* n_roots, int32_t* n_rounds, cudaStream_t st);

PrioCfg make_prio(const mis2_ctx* c, int64_t n, uint64_t seed);

// Batched engine internals for the server's merged launches.  After a
// one-level mis2_batch_coarsen: graph `graph`'s roots (ascending), labels,
// coarse rowptr and colind, renumbered to the graph's own ids, copied into
// the given device arrays on `st` (asynchronously), with their counts.
// MIS2_ERR_INVALID_ARG for a graph that was not coarsened (n below min_n).
mis2_ctx* batch_context(mis2_batch* b);
int batch_level0_result(const mis2_batch* b, int32_t graph, int32_t* roots, int32_t* labels, int32_t* c_rowptr,
                        int32_t* c_colind, int64_t* n_roots, int64_t* n_aggs, int64_t* c_nnz, cudaStream_t st);
int coarse_bitmap_blocks(const mis2_ctx* c);

}  // namespace mis2
