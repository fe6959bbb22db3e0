// api.cu -- the extern "C" entry points declared in include/mis2.h: context
// and scratch management, argument validation, dispatch to the phase
// launchers, statistics and timing.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.h"

namespace mis2 {

static thread_local char g_last_error[256] = "";

int set_cuda_error(cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return MIS2_ERR_CUDA;
}

void set_error_text(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

void timer_begin(mis2_ctx* c, int cls, cudaStream_t st) {
  if (!c->cfg.timing) return;
  if (c->cfg.timing == MIS2_TIMING_LOOP && cls != kKcDeviceLoop) return;  // its timer_end sees no open interval
  Timer& t = c->timer;
  if (t.used + 2 > t.ev.size()) {
    for (int k = 0; k < 64; k++) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      t.ev.push_back(e);
    }
  }
  cudaEventRecord(t.ev[t.used], st);
  t.cls.push_back(cls);
  t.used += 1;
}

void timer_end(mis2_ctx* c, cudaStream_t st) {
  if (!c->cfg.timing) return;
  Timer& t = c->timer;
  if (t.used == 0 || t.used >= t.ev.size() || (t.used & 1) == 0) return;
  cudaEventRecord(t.ev[t.used], st);
  t.used += 1;
}

void timer_reset(mis2_ctx* c) {
  c->timer.used = 0;
  c->timer.cls.clear();
}

int timer_collect(mis2_ctx* c) {
  if (!c->cfg.timing) return MIS2_OK;
  Timer& t = c->timer;
  for (size_t i = 0; i + 1 < t.used; i += 2) {
    float ms = 0.f;
    MIS2_CUDA(cudaEventSynchronize(t.ev[i + 1]));
    MIS2_CUDA(cudaEventElapsedTime(&ms, t.ev[i], t.ev[i + 1]));
    const int k = t.cls[i / 2];
    c->stats.kernel_ms[k] += ms;
    c->stats.kernel_launches[k] += 1;
  }
  timer_reset(c);
  return MIS2_OK;
}

int resident_blocks_per_sm(const mis2_ctx* c, const void* kernel, int block, int* per_sm, int smem) {
  struct Entry {
    const void* kernel;
    int device, block, smem, per_sm;
  };
  static std::mutex mu;
  static std::vector<Entry> known;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& e : known)
      if (e.kernel == kernel && e.device == c->device && e.block == block && e.smem == smem) {
        *per_sm = e.per_sm;
        return MIS2_OK;
      }
  }
  if (smem > 48 * 1024) MIS2_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int n = 0;
  MIS2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem));
  std::lock_guard<std::mutex> lk(mu);
  known.push_back(Entry{kernel, c->device, block, smem, n});
  *per_sm = n;
  return MIS2_OK;
}

PrioCfg make_prio(const mis2_ctx* c, int64_t n, uint64_t seed) {
  PrioCfg p;
  p.seed = seed;
  p.table = nullptr;
  p.table_n = n;
  p.table_rounds = 0;
  p.gid = nullptr;
  p.voff = nullptr;
  p.gbits = nullptr;
  p.b = id_bits(n);
  p.variant = c->cfg.hash_variant;
  p.pad = 0;
  return p;
}

static int validate_cfg(const mis2_config* cfg) {
  if (cfg->hash_variant < 0 || cfg->hash_variant > 2) return MIS2_ERR_INVALID_ARG;
  if (cfg->agg_mode < 0 || cfg->agg_mode > 1) return MIS2_ERR_INVALID_ARG;
  const int gl = cfg->group_lanes;
  if (gl != 0 && gl != 1 && gl != 2 && gl != 4 && gl != 8 && gl != 16 && gl != 32) return MIS2_ERR_INVALID_ARG;
  if (cfg->warp_degree < 0 || cfg->block_degree < 1 || cfg->block_degree < cfg->warp_degree)
    return MIS2_ERR_INVALID_ARG;
  if (cfg->block_size != kBlock) return MIS2_ERR_INVALID_ARG;
  if (cfg->loop != MIS2_LOOP_HOST && cfg->loop != MIS2_LOOP_DEVICE) return MIS2_ERR_INVALID_ARG;
  if (cfg->spin_limit < 1 || cfg->loop_blocks_per_sm < 0) return MIS2_ERR_INVALID_ARG;
  if (cfg->timing < 0 || cfg->timing > MIS2_TIMING_LOOP) return MIS2_ERR_INVALID_ARG;
  if ((cfg->ablation & ~(MIS2_ABLATE_NO_WORKLISTS | MIS2_ABLATE_TUPLE_ENGINE | MIS2_ABLATE_UNPACKED_TUPLES)) != 0 ||
      (cfg->serial_launches != 0 && cfg->serial_launches != 1))
    return MIS2_ERR_INVALID_ARG;
  return MIS2_OK;
}

static int validate_graph(const mis2_ctx* c, const mis2_csr* g, GraphArgs* out, bool device_ptrs = true) {
  if (g == nullptr) return MIS2_ERR_INVALID_ARG;
  if (g->n < 0 || g->nnz < 0 || g->n >= ((int64_t)1 << 31) || g->nnz >= ((int64_t)1 << 31))
    return MIS2_ERR_INVALID_ARG;
  if (g->n > c->max_n || g->nnz > c->max_nnz) return MIS2_ERR_OUT_OF_MEMORY;
  if (g->rowptr == nullptr) return MIS2_ERR_INVALID_ARG;
  if (g->nnz > 0 && g->colind == nullptr) return MIS2_ERR_INVALID_ARG;
  if (g->rowptr_is_64 != 0 && g->rowptr_is_64 != 1) return MIS2_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(g->colind) & 3u) != 0) return MIS2_ERR_INVALID_ARG;
  out->n = g->n;
  out->nnz = g->nnz;
  out->rp64 = g->rowptr_is_64 != 0;
  out->rowptr = g->rowptr;
  out->colind = g->colind;
  out->vec = (reinterpret_cast<uintptr_t>(g->colind) & 15u) == 0;
  (void)device_ptrs;
  return MIS2_OK;
}

template <typename T>
static int dev_alloc(mis2_ctx* c, T** p, int64_t count) {
  void* q = nullptr;
  const size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(T);
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return MIS2_ERR_OUT_OF_MEMORY;
  }
  c->allocations.push_back(q);
  *p = static_cast<T*>(q);
  return MIS2_OK;
}

static void free_all(mis2_ctx* c) {
  for (void* p : c->allocations) cudaFree(p);
  c->allocations.clear();
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  if (c->h_trace) cudaFreeHost(c->h_trace);
  c->h_ctr = nullptr;
  c->h_trace = nullptr;
  for (cudaEvent_t e : c->timer.ev) cudaEventDestroy(e);
  c->timer.ev.clear();
  if (c->ev_counts) cudaEventDestroy(c->ev_counts);
  c->ev_counts = nullptr;
}

static int alloc_scratch(mis2_ctx* c) {
  Scratch& s = c->s;
  const int64_t n = std::max<int64_t>(c->max_n, 1), nnz = std::max<int64_t>(c->max_nnz, 1);
  MIS2_TRY(dev_alloc(c, &s.T, n));
  MIS2_TRY(dev_alloc(c, &s.M, n));
  for (int b = 0; b < 2; b++)
    for (int k = 0; k < kClasses; k++) {
      MIS2_TRY(dev_alloc(c, &s.wl1[b][k], n));
      MIS2_TRY(dev_alloc(c, &s.wl2[b][k], n));
    }
  MIS2_TRY(dev_alloc(c, &s.ctr, kCtrWords));
  MIS2_TRY(dev_alloc(c, &s.dtrace, 2 * MIS2_TRACE_CAP * 4));
  MIS2_TRY(dev_alloc(c, &s.loop_ts, 2 * kLoopTsWords));
  MIS2_TRY(dev_alloc(c, &s.tile, n / 2048 + 4));
  MIS2_TRY(dev_alloc(c, &s.roots2, n));
  MIS2_TRY(dev_alloc(c, &s.qlist, n));
  MIS2_TRY(dev_alloc(c, &s.qflag, n));
  MIS2_TRY(dev_alloc(c, &s.tent, n));
  MIS2_TRY(dev_alloc(c, &s.aggsize, n));
  MIS2_TRY(dev_alloc(c, &s.left, n));
  MIS2_TRY(dev_alloc(c, &s.left_heavy, n));
  MIS2_TRY(dev_alloc(c, &s.left_mid, n));
  MIS2_TRY(dev_alloc(c, &s.roots_tmp, n));
  MIS2_TRY(dev_alloc(c, &s.agg_cnt, n + 1));
  MIS2_TRY(dev_alloc(c, &s.agg_ptr, n + 1));
  MIS2_TRY(dev_alloc(c, &s.ub, n + 1));
  MIS2_TRY(dev_alloc(c, &s.ub_ptr, n + 1));
  MIS2_TRY(dev_alloc(c, &s.cursor, n + 1));
  MIS2_TRY(dev_alloc(c, &s.members, n));
  MIS2_TRY(dev_alloc(c, &s.c_cnt, n + 1));
  MIS2_TRY(dev_alloc(c, &s.large, n));
  MIS2_TRY(dev_alloc(c, &s.tmp, nnz + 4));
  MIS2_TRY(dev_alloc(c, &s.labels_tmp, n));
  MIS2_TRY(dev_alloc(c, &s.radix, group_scratch_words(n)));
  MIS2_TRY(dev_alloc(c, &s.cand, 3 * n));
  MIS2_TRY(dev_alloc(c, &s.bitmaps, (int64_t)coarse_bitmap_blocks(c) * ((n + 31) / 32)));
  MIS2_TRY(dev_alloc(c, &s.chunk_off, n + 1));
  const int64_t giant_cap = nnz / kGiantRow + 1;
  MIS2_TRY(dev_alloc(c, &s.giant_v, giant_cap));
  MIS2_TRY(dev_alloc(c, &s.giant_slot, giant_cap));
  MIS2_TRY(dev_alloc(c, &s.giant_off, giant_cap + 1));
  if (cudaMallocHost(&c->h_ctr, kCtrWords * sizeof(int32_t)) != cudaSuccess) return MIS2_ERR_OUT_OF_MEMORY;
  if (cudaMallocHost(&c->h_trace, 2 * MIS2_TRACE_CAP * 4 * sizeof(int64_t)) != cudaSuccess)
    return MIS2_ERR_OUT_OF_MEMORY;
  MIS2_CUDA(cudaMemset(s.ctr, 0, kCtrWords * sizeof(int32_t)));
  return MIS2_OK;
}

// Debug-mode validation of a graph argument (MIS2_DEBUG_VALIDATE).
static int debug_graph(mis2_ctx* c, const GraphArgs& ga, cudaStream_t st) {
  if (!(c->cfg.debug_checks & MIS2_DEBUG_VALIDATE)) return MIS2_OK;
  return check_graph(c, ga, st);
}

static void begin_call(mis2_ctx* c) {
  c->launches = 0;
  memset(c->stats.loop_ns, 0, sizeof(c->stats.loop_ns));
  timer_reset(c);
  memset(c->stats.kernel_ms, 0, sizeof(c->stats.kernel_ms));
  memset(c->stats.kernel_launches, 0, sizeof(c->stats.kernel_launches));
}

// Copy the device trace of `phase` into the stats after a synchronised call.
static int fetch_trace(mis2_ctx* c, int phase, int32_t rounds, cudaStream_t st) {
  int64_t(*dst)[4] = phase == 0 ? c->stats.trace : c->stats.trace2;
  memset(dst, 0, sizeof(c->stats.trace));
  const int r = std::min<int32_t>(rounds, MIS2_TRACE_CAP);
  if (r <= 0) return MIS2_OK;
  MIS2_CUDA(cudaMemcpyAsync(c->h_trace, c->s.dtrace + (int64_t)phase * MIS2_TRACE_CAP * 4,
                            (size_t)r * 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  memcpy(dst, c->h_trace, (size_t)r * 4 * sizeof(int64_t));
  return MIS2_OK;
}

// The tuple-engine ablation bits apply to mis2_run alone; the other calls
// that run MIS-2 refuse a context with them set.
static bool tuple_ablation(const mis2_ctx* c) {
  return (c->cfg.ablation & (MIS2_ABLATE_TUPLE_ENGINE | MIS2_ABLATE_UNPACKED_TUPLES)) != 0;
}

int run_impl(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, uint8_t* in_set, int32_t* roots, int64_t* n_roots,
             int32_t* n_rounds, cudaStream_t st) {
  int32_t r = 0;
  if (g.n > 0) {
    if (c->cfg.loop == MIS2_LOOP_DEVICE)
      MIS2_TRY(mis2_rounds_device(c, g, nullptr, p, 0, st, &r));
    else
      MIS2_TRY(mis2_rounds_host(c, g, nullptr, p, 0, st, &r));
  }
  MIS2_TRY(extract_in_set(c, g.n, in_set, roots, c->s.ctr + kCtrRoots, st));
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, c->s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  *n_roots = c->h_ctr[kCtrRoots];
  if (n_rounds) *n_rounds = r;
  c->stats.rounds = r;
  c->stats.n_roots = *n_roots;
  return fetch_trace(c, 0, r, st);
}

}  // namespace mis2

using namespace mis2;

extern "C" {

void mis2_config_default(mis2_config* cfg) {
  if (cfg == nullptr) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->hash_variant = MIS2_HASH_XORSHIFT_STAR;
  cfg->agg_mode = MIS2_AGG_ALG3;
  cfg->group_lanes = 0;
  cfg->warp_degree = 0;
  cfg->block_degree = 2048;
  cfg->block_size = kBlock;
  cfg->loop = MIS2_LOOP_HOST;
  cfg->debug_checks = 0;
  cfg->timing = 0;
  cfg->spin_limit = (int64_t)1 << 23;
}

int mis2_ctx_create(mis2_ctx** out, int64_t max_n, int64_t max_nnz, const mis2_config* cfg) {
  if (out == nullptr) return MIS2_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_n < 0 || max_nnz < 0 || max_n >= ((int64_t)1 << 31) || max_nnz >= ((int64_t)1 << 31))
    return MIS2_ERR_INVALID_ARG;
  mis2_ctx* c = new mis2_ctx();
  mis2_config_default(&c->cfg);
  if (cfg != nullptr) {
    int rc = validate_cfg(cfg);
    if (rc != MIS2_OK) {
      delete c;
      return rc;
    }
    c->cfg = *cfg;
  }
  c->max_n = max_n;
  c->max_nnz = max_nnz;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return set_cuda_error(e);
  }
  int rc = alloc_scratch(c);
  if (rc != MIS2_OK) {
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return MIS2_OK;
}

int mis2_ctx_destroy(mis2_ctx* c) {
  if (c == nullptr) return MIS2_OK;
  cudaDeviceSynchronize();
  free_all(c);
  delete c;
  return MIS2_OK;
}

int mis2_ctx_set_config(mis2_ctx* c, const mis2_config* cfg) {
  if (c == nullptr || cfg == nullptr) return MIS2_ERR_INVALID_ARG;
  MIS2_TRY(validate_cfg(cfg));
  c->cfg = *cfg;
  return MIS2_OK;
}

int mis2_get_stats(const mis2_ctx* c, mis2_stats* out) {
  if (c == nullptr || out == nullptr) return MIS2_ERR_INVALID_ARG;
  *out = c->stats;
  out->launches = c->launches;
  return MIS2_OK;
}

int mis2_run(mis2_ctx* c, const mis2_csr* g, uint64_t seed, uint8_t* in_set, int32_t* roots, int64_t* n_roots,
             int32_t* n_rounds, void* stream) {
  NvtxRange nvtx_call("mis2_run");
  if (c == nullptr || n_roots == nullptr) return MIS2_ERR_INVALID_ARG;
  GraphArgs ga;
  MIS2_TRY(validate_graph(c, g, &ga));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  MIS2_TRY(debug_graph(c, ga, st));
  int rc;
  if (tuple_ablation(c))
    rc = tuple_engine_impl(c, ga, make_prio(c, ga.n, seed), (c->cfg.ablation & MIS2_ABLATE_UNPACKED_TUPLES) != 0,
                           in_set, roots, n_roots, n_rounds, st);
  else
    rc = run_impl(c, ga, make_prio(c, ga.n, seed), in_set, roots, n_roots, n_rounds, st);
  if (rc == MIS2_OK) rc = timer_collect(c);
  return rc;
}

static int run_priorities_impl(mis2_ctx* c, const mis2_csr* g, const uint32_t* prio_table, int32_t table_rounds,
                               uint32_t* snaps, int32_t snap_rounds, uint8_t* in_set, int32_t* roots,
                               int64_t* n_roots, int32_t* n_rounds, void* stream) {
  if (c == nullptr || n_roots == nullptr || table_rounds < 0 || (table_rounds > 0 && prio_table == nullptr) ||
      snap_rounds < 0 || (snap_rounds > 0 && snaps == nullptr) || tuple_ablation(c))
    return MIS2_ERR_INVALID_ARG;
  GraphArgs ga;
  MIS2_TRY(validate_graph(c, g, &ga));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  MIS2_TRY(debug_graph(c, ga, st));
  PrioCfg p = make_prio(c, ga.n, 0);
  uint32_t* dtab = nullptr;
  const size_t bytes = (size_t)table_rounds * (size_t)ga.n * sizeof(uint32_t);
  if (bytes > 0) {
    MIS2_CUDA(cudaMalloc(&dtab, bytes));
    cudaError_t e = cudaMemcpyAsync(dtab, prio_table, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaFree(dtab);
      return set_cuda_error(e);
    }
    p.table = dtab;
    p.table_rounds = table_rounds;
  }
  int rc = MIS2_OK;
  if (snap_rounds > 0 && ga.n > 0) {
    const cudaError_t e = cudaMemsetAsync(snaps, 0xFF, (size_t)snap_rounds * 3 * (size_t)ga.n * sizeof(uint32_t), st);
    if (e != cudaSuccess) rc = set_cuda_error(e);
    c->snaps = snaps;
    c->snap_rounds = snap_rounds;
  }
  if (rc == MIS2_OK) rc = run_impl(c, ga, p, in_set, roots, n_roots, n_rounds, st);
  c->snaps = nullptr;
  c->snap_rounds = 0;
  if (dtab) {
    cudaStreamSynchronize(st);
    cudaFree(dtab);
  }
  if (rc == MIS2_OK) rc = timer_collect(c);
  return rc;
}

int mis2_run_with_priorities(mis2_ctx* c, const mis2_csr* g, const uint32_t* prio_table, int32_t table_rounds,
                             uint8_t* in_set, int32_t* roots, int64_t* n_roots, int32_t* n_rounds, void* stream) {
  NvtxRange nvtx_call("mis2_run_with_priorities");
  return run_priorities_impl(c, g, prio_table, table_rounds, nullptr, 0, in_set, roots, n_roots, n_rounds, stream);
}

int mis2_run_snapshots(mis2_ctx* c, const mis2_csr* g, const uint32_t* prio_table, int32_t table_rounds,
                       uint32_t* snaps, int32_t snap_rounds, uint8_t* in_set, int32_t* roots, int64_t* n_roots,
                       int32_t* n_rounds, void* stream) {
  NvtxRange nvtx_call("mis2_run_snapshots");
  return run_priorities_impl(c, g, prio_table, table_rounds, snaps, snap_rounds, in_set, roots, n_roots, n_rounds,
                             stream);
}

int mis2_aggregate(mis2_ctx* c, const mis2_csr* g, const int32_t* roots, int64_t n_roots, uint64_t seed,
                   int32_t mode, int32_t* labels, int64_t* n_aggs, void* stream) {
  NvtxRange nvtx_call("mis2_aggregate");
  if (c == nullptr || n_aggs == nullptr || (mode != MIS2_AGG_ALG3 && mode != MIS2_AGG_BASIC) || tuple_ablation(c))
    return MIS2_ERR_INVALID_ARG;
  GraphArgs ga;
  MIS2_TRY(validate_graph(c, g, &ga));
  if (n_roots < 0 || n_roots > ga.n || (n_roots > 0 && roots == nullptr) || (ga.n > 0 && labels == nullptr))
    return MIS2_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  MIS2_TRY(debug_graph(c, ga, st));
  if (c->cfg.debug_checks & MIS2_DEBUG_VALIDATE) MIS2_TRY(check_roots(c, ga, roots, n_roots, st));
  int rc = aggregate_impl(c, ga, roots, n_roots, seed, mode, labels, n_aggs, st);
  if (rc == MIS2_OK) rc = fetch_trace(c, 1, c->stats.rounds2, st);
  if (rc == MIS2_OK) {
    c->stats.n_phase1 = n_roots;
    c->stats.n_aggs = *n_aggs;
    rc = timer_collect(c);
  }
  return rc;
}

int mis2_coarsen(mis2_ctx* c, const mis2_csr* g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                 int32_t* c_colind, int64_t c_colind_cap, int64_t* c_nnz, void* stream) {
  NvtxRange nvtx_call("mis2_coarsen");
  if (c == nullptr || c_nnz == nullptr || c_rowptr == nullptr) return MIS2_ERR_INVALID_ARG;
  GraphArgs ga;
  MIS2_TRY(validate_graph(c, g, &ga));
  if (n_aggs < 0 || n_aggs > ga.n || (ga.n > 0 && labels == nullptr) || (n_aggs == 0 && ga.n > 0) ||
      c_colind_cap < 0 || (c_colind_cap > 0 && c_colind == nullptr))
    return MIS2_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  MIS2_TRY(debug_graph(c, ga, st));
  if (c->cfg.debug_checks & MIS2_DEBUG_VALIDATE) MIS2_TRY(check_labels(c, labels, ga.n, n_aggs, st));
  int rc = coarsen_impl(c, ga, labels, n_aggs, c_rowptr, c_colind, c_colind_cap, c_nnz, st);
  if (rc == MIS2_OK) {
    c->stats.c_nnz = *c_nnz;
    rc = timer_collect(c);
  }
  return rc;
}

static int device_error(int32_t err) {
  if (err & kErrTimeout) return MIS2_ERR_TIMEOUT;
  if (err & kErrNoProgress) return MIS2_ERR_NO_PROGRESS;
  if (err & kErrNoAggregatedNeighbour) return MIS2_ERR_BAD_GRAPH;
  return MIS2_OK;
}

// One level with the persistent round loop and two host round trips: the
// counts that size later steps (roots, phase-2 roots, large aggregates) stay
// on the device and are read by the kernels that need them; the host waits
// once for n_aggs (which sizes the coarse graph's launches) and once at the
// end.  Results are those of the step-by-step path.
static int level_fast(mis2_ctx* c, const GraphArgs& ga, uint64_t seed, uint8_t* in_set, int32_t* rl, int32_t* lab,
                      int32_t* c_rowptr, int32_t* c_colind, int64_t c_colind_cap, int64_t* n_roots, int64_t* n_aggs,
                      int64_t* c_nnz, cudaStream_t st) {
  Scratch& s = c->s;
  const PrioCfg p = make_prio(c, ga.n, seed);
  MIS2_CUDA(cudaMemsetAsync(s.ctr, 0, kCtrWords * sizeof(int32_t), st));
  {
    NvtxRange r("MIS-2 (Algorithm 1)");
    MIS2_TRY(mis2_rounds_device_async(c, ga, nullptr, p, 0, kCtrRounds, st));
    // the same pass initialises the aggregation's frozen labels and sizes
    // and the coarse graph's histogram
    LevelFill fill;
    fill.minus1 = s.tent;
    fill.zero[0] = s.aggsize;
    fill.zero[1] = s.agg_cnt;
    fill.zero[2] = s.ub;
    MIS2_TRY(extract_in_set(c, ga.n, in_set, rl, s.ctr + kCtrRoots, st, fill));
  }
  {
    NvtxRange r("aggregation (Algorithm 3)");
    MIS2_TRY(agg_level_async(c, ga, rl, p, c->cfg.agg_mode, lab, st));
  }
  MIS2_CUDA(cudaMemcpyAsync(c->h_trace, s.dtrace, 2 * MIS2_TRACE_CAP * 4 * sizeof(int64_t), cudaMemcpyDeviceToHost,
                            st));
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (c->ev_counts == nullptr) MIS2_CUDA(cudaEventCreateWithFlags(&c->ev_counts, cudaEventDisableTiming));
  MIS2_CUDA(cudaEventRecord(c->ev_counts, st));
  // the coarse graph's labels-only steps run while the host waits for the
  // counts (n_aggs sizes the rest)
  bool cand_ready = false;
  if (c_rowptr != nullptr) {
    NvtxRange r("coarse graph");
    MIS2_TRY(coarsen_prelude(c, ga, lab, &cand_ready, st, true));
  }
  MIS2_CUDA(cudaEventSynchronize(c->ev_counts));
  MIS2_TRY(device_error(c->h_ctr[kCtrErr]));
  const int64_t nr = c->h_ctr[kCtrRoots];
  const int64_t na = nr + c->h_ctr[kCtrQual];
  c->stats.rounds = c->h_ctr[kCtrRounds];
  c->stats.rounds2 = c->cfg.agg_mode == MIS2_AGG_ALG3 ? c->h_ctr[kCtrRounds2] : 0;
  c->stats.n_roots = nr;
  c->stats.n_phase1 = nr;
  c->stats.n_aggs = na;
  memcpy(c->stats.trace, c->h_trace, sizeof(c->stats.trace));
  memset(c->stats.trace2, 0, sizeof(c->stats.trace2));
  if (c->cfg.agg_mode == MIS2_AGG_ALG3)
    memcpy(c->stats.trace2, c->h_trace + MIS2_TRACE_CAP * 4, sizeof(c->stats.trace2));
  int64_t cn = 0;
  if (c_rowptr != nullptr) {
    NvtxRange r("coarse graph");
    MIS2_TRY(coarsen_fast(c, ga, lab, na, c_rowptr, c_colind, c_colind_cap, st, true, cand_ready, true));
    MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    if (coarsen_fast_needs_retry(c)) {
      MIS2_TRY(coarsen_fast_finish(c, ga, lab, na, c_rowptr, c_colind, c_colind_cap, &cn, st));
    } else {
      if (c->h_ctr[kCtrErr] & kErrCapacity) return MIS2_ERR_INVALID_ARG;
      cn = c->h_ctr[kCtrCnnz];
    }
    c->stats.c_nnz = cn;
  }
  if (n_roots) *n_roots = nr;
  if (n_aggs) *n_aggs = na;
  if (c_nnz) *c_nnz = cn;
  return MIS2_OK;
}

static int level_impl(mis2_ctx* c, const GraphArgs& ga, uint64_t seed, uint8_t* in_set, int32_t* roots,
                      int32_t* labels, int32_t* c_rowptr, int32_t* c_colind, int64_t c_colind_cap, int64_t* n_roots,
                      int64_t* n_aggs, int64_t* c_nnz, cudaStream_t st) {
  int32_t* rl = roots != nullptr ? roots : c->s.roots_tmp;
  int32_t* lab = labels != nullptr ? labels : c->s.labels_tmp;
  if (c->cfg.loop == MIS2_LOOP_DEVICE && ga.n > 0)
    return level_fast(c, ga, seed, in_set, rl, lab, c_rowptr, c_colind, c_colind_cap, n_roots, n_aggs, c_nnz, st);
  int64_t nr = 0, na = 0, cn = 0;
  MIS2_TRY(run_impl(c, ga, make_prio(c, ga.n, seed), in_set, rl, &nr, nullptr, st));
  MIS2_TRY(aggregate_impl(c, ga, rl, nr, seed, c->cfg.agg_mode, lab, &na, st));
  MIS2_TRY(fetch_trace(c, 1, c->stats.rounds2, st));
  c->stats.n_phase1 = nr;
  c->stats.n_aggs = na;
  if (c_rowptr != nullptr) {
    MIS2_TRY(coarsen_impl(c, ga, lab, na, c_rowptr, c_colind, c_colind_cap, &cn, st));
    c->stats.c_nnz = cn;
  }
  if (n_roots) *n_roots = nr;
  if (n_aggs) *n_aggs = na;
  if (c_nnz) *c_nnz = cn;
  return MIS2_OK;
}

int mis2_coarsen_level(mis2_ctx* c, const mis2_csr* g, uint64_t seed, uint8_t* in_set, int32_t* roots,
                       int32_t* labels, int32_t* c_rowptr, int32_t* c_colind, int64_t c_colind_cap, int64_t* n_roots,
                       int64_t* n_aggs, int64_t* c_nnz, void* stream) {
  NvtxRange nvtx_call("mis2_coarsen_level");
  if (c == nullptr || tuple_ablation(c)) return MIS2_ERR_INVALID_ARG;
  GraphArgs ga;
  MIS2_TRY(validate_graph(c, g, &ga));
  if (c_colind_cap < 0 || (c_rowptr != nullptr && c_colind_cap > 0 && c_colind == nullptr))
    return MIS2_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  MIS2_TRY(debug_graph(c, ga, st));
  int rc = level_impl(c, ga, seed, in_set, roots, labels, c_rowptr, c_colind, c_colind_cap, n_roots, n_aggs, c_nnz,
                      st);
  if (rc == MIS2_OK) rc = timer_collect(c);
  return rc;
}

static int ensure_stage(mis2_ctx* c, int64_t n, int64_t nnz) {
  HostStage& h = c->stage;
  if (h.cap_n >= n && h.cap_nnz >= nnz && h.rowptr != nullptr) return MIS2_OK;
  if (h.rowptr != nullptr) return MIS2_ERR_OUT_OF_MEMORY;  // staged once at the context's maximum
  n = c->max_n;
  nnz = c->max_nnz;
  MIS2_TRY(dev_alloc(c, reinterpret_cast<int64_t**>(&h.rowptr), n + 1));
  MIS2_TRY(dev_alloc(c, &h.colind, nnz + 4));
  MIS2_TRY(dev_alloc(c, &h.in_set, n));
  MIS2_TRY(dev_alloc(c, &h.roots, n));
  MIS2_TRY(dev_alloc(c, &h.labels, n));
  MIS2_TRY(dev_alloc(c, &h.c_rowptr, n + 1));
  MIS2_TRY(dev_alloc(c, &h.c_colind, nnz + 4));
  h.cap_n = n;
  h.cap_nnz = nnz;
  return MIS2_OK;
}

int mis2_coarsen_level_host(mis2_ctx* c, const mis2_csr* gh, uint64_t seed, uint8_t* in_set, int32_t* roots,
                            int32_t* labels, int32_t* c_rowptr, int32_t* c_colind, int64_t c_colind_cap,
                            int64_t* n_roots, int64_t* n_aggs, int64_t* c_nnz, void* stream) {
  NvtxRange nvtx_call("mis2_coarsen_level_host");
  if (c == nullptr || gh == nullptr || tuple_ablation(c)) return MIS2_ERR_INVALID_ARG;
  if (gh->n < 0 || gh->nnz < 0 || gh->rowptr == nullptr || (gh->nnz > 0 && gh->colind == nullptr))
    return MIS2_ERR_INVALID_ARG;
  if (gh->n > c->max_n || gh->nnz > c->max_nnz) return MIS2_ERR_OUT_OF_MEMORY;
  MIS2_TRY(ensure_stage(c, gh->n, gh->nnz));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HostStage& h = c->stage;
  const size_t rp_bytes = (size_t)(gh->n + 1) * (gh->rowptr_is_64 ? 8 : 4);
  begin_call(c);
  MIS2_CUDA(cudaMemcpyAsync(h.rowptr, gh->rowptr, rp_bytes, cudaMemcpyHostToDevice, st));
  if (gh->nnz > 0)
    MIS2_CUDA(cudaMemcpyAsync(h.colind, gh->colind, (size_t)gh->nnz * 4, cudaMemcpyHostToDevice, st));
  mis2_csr gd = *gh;
  gd.rowptr = h.rowptr;
  gd.colind = h.colind;
  GraphArgs ga;
  MIS2_TRY(validate_graph(c, &gd, &ga));
  MIS2_TRY(debug_graph(c, ga, st));
  int64_t nr = 0, na = 0, cn = 0;
  MIS2_TRY(level_impl(c, ga, seed, h.in_set, h.roots, h.labels, c_rowptr ? h.c_rowptr : nullptr, h.c_colind,
                      c->max_nnz, &nr, &na, &cn, st));
  const int64_t n = ga.n;
  if (in_set && n > 0) MIS2_CUDA(cudaMemcpyAsync(in_set, h.in_set, (size_t)n, cudaMemcpyDeviceToHost, st));
  if (roots && nr > 0) MIS2_CUDA(cudaMemcpyAsync(roots, h.roots, (size_t)nr * 4, cudaMemcpyDeviceToHost, st));
  if (labels && n > 0) MIS2_CUDA(cudaMemcpyAsync(labels, h.labels, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
  if (c_rowptr) {
    if (cn > c_colind_cap) return MIS2_ERR_INVALID_ARG;
    MIS2_CUDA(cudaMemcpyAsync(c_rowptr, h.c_rowptr, (size_t)(na + 1) * 4, cudaMemcpyDeviceToHost, st));
    if (cn > 0) MIS2_CUDA(cudaMemcpyAsync(c_colind, h.c_colind, (size_t)cn * 4, cudaMemcpyDeviceToHost, st));
  }
  MIS2_CUDA(cudaStreamSynchronize(st));
  if (n_roots) *n_roots = nr;
  if (n_aggs) *n_aggs = na;
  if (c_nnz) *c_nnz = cn;
  return timer_collect(c);
}

int mis2_run_k(mis2_ctx* c, const mis2_csr* g, int32_t k, uint64_t seed, uint8_t* in_set, int32_t* roots,
               int64_t* n_roots, int32_t* n_rounds, void* stream) {
  NvtxRange nvtx_call("mis2_run_k");
  if (c == nullptr || n_roots == nullptr || k < 1 || k > 16) return MIS2_ERR_INVALID_ARG;
  GraphArgs ga;
  MIS2_TRY(validate_graph(c, g, &ga));
  if (ga.n > 0 && roots == nullptr) return MIS2_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  MIS2_TRY(debug_graph(c, ga, st));
  int rc = misk_impl(c, ga, k, make_prio(c, ga.n, seed), in_set, roots, n_roots, n_rounds, st);
  return rc == MIS2_OK ? timer_collect(c) : rc;
}

int mis2_color(mis2_ctx* c, const mis2_csr* g, uint64_t seed, int32_t* colors, int32_t* color_ptr,
               int32_t* color_list, int32_t* n_colors, int32_t* n_rounds, void* stream) {
  NvtxRange nvtx_call("mis2_color");
  if (c == nullptr || n_colors == nullptr || color_ptr == nullptr) return MIS2_ERR_INVALID_ARG;
  GraphArgs ga;
  MIS2_TRY(validate_graph(c, g, &ga));
  if (ga.n > 0 && (colors == nullptr || color_list == nullptr)) return MIS2_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  MIS2_TRY(debug_graph(c, ga, st));
  const int rc = color_impl(c, ga, make_prio(c, ga.n, seed), colors, color_ptr, color_list, n_colors, n_rounds, st);
  return rc == MIS2_OK ? timer_collect(c) : rc;
}

int mis2_coarse_weights(mis2_ctx* c, const mis2_csr* g, const int32_t* labels, int64_t n_aggs,
                        const int32_t* c_rowptr, const int32_t* c_colind, int64_t c_nnz, int32_t* c_weights,
                        void* stream) {
  NvtxRange nvtx_call("mis2_coarse_weights");
  if (c == nullptr || c_rowptr == nullptr) return MIS2_ERR_INVALID_ARG;
  GraphArgs ga;
  MIS2_TRY(validate_graph(c, g, &ga));
  if (n_aggs < 0 || n_aggs > ga.n || (ga.n > 0 && labels == nullptr) || c_nnz < 0 ||
      (c_nnz > 0 && (c_colind == nullptr || c_weights == nullptr)))
    return MIS2_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  MIS2_TRY(debug_graph(c, ga, st));
  if (c->cfg.debug_checks & MIS2_DEBUG_VALIDATE) MIS2_TRY(check_labels(c, labels, ga.n, n_aggs, st));
  const int rc = coarse_weights_impl(c, ga, labels, c_rowptr, c_colind, c_nnz, c_weights, st);
  return rc == MIS2_OK ? timer_collect(c) : rc;
}

int mis2_tentative_prolongator(mis2_ctx* c, const int32_t* labels, int64_t n, int64_t n_aggs, int32_t normalize,
                               int32_t* p_rowptr, int32_t* p_colind, double* p_values, void* stream) {
  NvtxRange nvtx_call("mis2_tentative_prolongator");
  if (c == nullptr || n < 0 || n > c->max_n || n_aggs < 0 || n_aggs > n || p_rowptr == nullptr ||
      (n > 0 && (labels == nullptr || p_colind == nullptr || p_values == nullptr)))
    return MIS2_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  if (c->cfg.debug_checks & MIS2_DEBUG_VALIDATE) MIS2_TRY(check_labels(c, labels, n, n_aggs, st));
  return prolongator_impl(c, labels, n, n_aggs, normalize, p_rowptr, p_colind, p_values, st);
}

int mis2_cluster_lists(mis2_ctx* c, const int32_t* labels, int64_t n, int64_t n_aggs, int32_t* c_ptr,
                       int32_t* members, void* stream) {
  NvtxRange nvtx_call("mis2_cluster_lists");
  if (c == nullptr || n < 0 || n > c->max_n || n_aggs < 0 || n_aggs > n || (n > 0 && n_aggs == 0) ||
      c_ptr == nullptr || (n > 0 && (labels == nullptr || members == nullptr)))
    return MIS2_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  begin_call(c);
  MIS2_TRY(group_by_key(c, labels, n, n_aggs, c_ptr, members, st));
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, c->s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  if (c->h_ctr[kCtrErr] & kErrBadGraph) return MIS2_ERR_BAD_GRAPH;
  return timer_collect(c);
}

const char* mis2_status_string(int status) {
  switch (status) {
    case MIS2_OK: return "MIS2_OK";
    case MIS2_ERR_INVALID_ARG: return "MIS2_ERR_INVALID_ARG";
    case MIS2_ERR_OUT_OF_MEMORY: return "MIS2_ERR_OUT_OF_MEMORY";
    case MIS2_ERR_CUDA: return "MIS2_ERR_CUDA";
    case MIS2_ERR_BAD_GRAPH: return "MIS2_ERR_BAD_GRAPH";
    case MIS2_ERR_TIMEOUT: return "MIS2_ERR_TIMEOUT";
    case MIS2_ERR_NO_PROGRESS: return "MIS2_ERR_NO_PROGRESS";
    case MIS2_ERR_CANCELLED: return "MIS2_ERR_CANCELLED";
    default: return "MIS2_ERR_UNKNOWN";
  }
}

const char* mis2_last_error(void) { return g_last_error; }

const char* mis2_version(void) { return "0.1.0"; }

}  // extern "C"
