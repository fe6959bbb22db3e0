// batch.cu -- many graphs of uneven sizes, and every level of their recursive
// coarsening hierarchies (Section I: multilevel methods coarsen recursively
// until the graph is below a threshold), processed together.
//
// All live graphs of a level are stored as one block-diagonal union CSR.  No
// edge crosses two graphs, so MIS-2 (Algorithm 1) on the union is the MIS-2
// of each graph, provided each vertex carries the tuple its graph would give
// it alone: local id, the graph's own id bits, the round counter restarting
// at 0 for every graph together (PrioCfg.gid / voff / gbits).  One persistent
// launch runs the rounds of every graph, with one worklist holding every
// graph's undecided vertices and grid-wide barriers between phases.
//
// Aggregation (Algorithm 3) runs on the union too.  Phase-1 and phase-2
// roots come out in ascending union order, i.e. graph-major; after phase 2
// the temporary ids are renumbered to "graph offset + local id" (phase-1
// roots, then phase-2 roots, per graph), which keeps the phase-3 tie-break
// on minimum id identical to a per-graph run.  The coarse union CSR is then
// block diagonal with each graph's coarse rows at its aggregate offset; the
// graphs that keep coarsening are compacted into the next level's union.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace mis2 {

struct GraphSrc {
  const void* rowptr;
  const int32_t* colind;
  int64_t n, nnz;
  int64_t voff, eoff;
  int32_t rp64;
  int32_t pad;
};

// Copy every input graph into the union: rowptr shifted by the graph's entry
// offset, colind shifted by its vertex offset, gid filled.  blockIdx.y picks
// the graph, blockIdx.x a slice of it.
__global__ void __launch_bounds__(kBlock) k_union_build(const GraphSrc* src, int32_t* u_rowptr, int32_t* u_colind,
                                                        int32_t* gid) {
  const GraphSrc gs = src[blockIdx.y];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = t0; i < gs.n; i += stride) {
    const int64_t r = gs.rp64 ? static_cast<const int64_t*>(gs.rowptr)[i]
                              : (int64_t) static_cast<const int32_t*>(gs.rowptr)[i];
    u_rowptr[gs.voff + i] = (int32_t)(r + gs.eoff);
    gid[gs.voff + i] = (int32_t)blockIdx.y;
  }
  for (int64_t k = t0; k < gs.nnz; k += stride) u_colind[gs.eoff + k] = gs.colind[k] + (int32_t)gs.voff;
}

__global__ void k_union_end(int32_t* u_rowptr, int64_t n, int64_t nnz) { u_rowptr[n] = (int32_t)nnz; }

// out[g] = first index of `list` (ascending, count entries) holding a value
// >= bounds[g], for g < nb.
__global__ void k_lower_bounds(const int32_t* list, const int32_t* count, const int64_t* bounds, int nb,
                               int64_t* out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nb) return;
  int64_t lo = 0, hi = *count;
  const int64_t x = bounds[g];
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (list[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  out[g] = lo;
}

struct RemapTables {
  const int32_t* gid;
  const int64_t* r1off;   // per graph: first phase-1 root rank
  const int64_t* qoff;    // per graph: first phase-2 root rank
  const int64_t* n1;      // per graph: phase-1 aggregates
  const int64_t* aggoff;  // per graph: first union aggregate id
  int64_t R1;             // all phase-1 roots
};

// Temporary ids (phase-1 rank j < R1, or R1 + phase-2 rank) -> graph-major
// final ids: aggoff[g] + local id.
__global__ void __launch_bounds__(kBlock) k_remap_labels(int64_t n, int32_t* labels, RemapTables t) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int32_t l = labels[v];
    if (l < 0) continue;
    const int32_t g = t.gid[v];
    int64_t f;
    if (l < t.R1) f = t.aggoff[g] + (l - t.r1off[g]);
    else f = t.aggoff[g] + t.n1[g] + (l - t.R1 - t.qoff[g]);
    labels[v] = (int32_t)f;
  }
}

struct CompactTables {
  const int32_t* src_graph;  // per new graph: index in the old level
  const int64_t* src_aoff;   // per old graph: aggregate offset (old coarse rows)
  const int64_t* dst_voff;   // per new graph: vertex offset (size ng+1)
  const int64_t* dst_eoff;   // per new graph: entry offset
  int32_t ng;
};

// Next level's union: rows of the continuing graphs, renumbered.
__global__ void __launch_bounds__(kBlock) k_union_compact(const int32_t* c_rowptr, const int32_t* c_colind,
                                                          CompactTables t, int32_t* u_rowptr, int32_t* u_colind,
                                                          int32_t* gid) {
  const int g = blockIdx.y;
  const int32_t og = t.src_graph[g];
  const int64_t aoff = t.src_aoff[og];
  const int64_t n = t.dst_voff[g + 1] - t.dst_voff[g];
  const int64_t ebase = c_rowptr[aoff];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t r0 = c_rowptr[aoff + i], r1 = c_rowptr[aoff + i + 1];
    const int64_t dst = t.dst_eoff[g] + (r0 - ebase);
    u_rowptr[t.dst_voff[g] + i] = (int32_t)dst;
    gid[t.dst_voff[g] + i] = g;
    for (int64_t k = r0; k < r1; k++) u_colind[dst + (k - r0)] = (int32_t)(c_colind[k] - aoff + t.dst_voff[g]);
  }
}

__global__ void __launch_bounds__(kBlock) k_sub_copy(const int32_t* src, int64_t count, int64_t sub, int32_t* dst) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    dst[i] = (int32_t)(src[i] - sub);
}

__global__ void k_gather_i32(const int32_t* src, const int64_t* idx, int count, int64_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = src[idx[i]];
}

}  // namespace mis2

using namespace mis2;

struct BatchLevel {
  int64_t n_union = 0, nnz_union = 0, n_aggs = 0, c_nnz = 0;
  std::vector<int32_t> graph;           // live index -> input graph id
  std::vector<int64_t> voff, aggoff;    // per live graph (+1 entry)
  int32_t* labels = nullptr;
  int32_t* c_rowptr = nullptr;
  int32_t* c_colind = nullptr;
  int64_t cap_labels = 0, cap_crp = 0, cap_cci = 0;
  int32_t rounds = 0, rounds2 = 0;
  std::vector<int64_t> r1off;    // per live graph (+1 entry): first union root of the graph
  std::vector<int64_t> ebounds;  // per live graph: [first, end) coarse entry of its rows
};

struct mis2_batch {
  mis2_ctx* ctx = nullptr;
  int32_t max_graphs = 0;
  int64_t max_total_n = 0, max_total_nnz = 0;
  int32_t* u_rowptr[2] = {nullptr, nullptr};
  int32_t* u_colind[2] = {nullptr, nullptr};
  int32_t* gid = nullptr;
  int64_t* d_tab = nullptr;  // 8 tables of (max_graphs + 1) int64
  int32_t* d_tab32 = nullptr;
  GraphSrc* d_src = nullptr;
  int64_t* h_tab = nullptr;  // pinned mirror of d_tab
  std::vector<BatchLevel> levels;
  int32_t n_levels = 0, n_graphs = 0;
  std::vector<std::vector<int64_t>> lvl_n, lvl_naggs, lvl_cnnz;  // [level][input graph]
  std::vector<void*> allocations;
};

namespace {

template <typename T>
int balloc(mis2_batch* b, T** p, int64_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, (size_t)std::max<int64_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return MIS2_ERR_OUT_OF_MEMORY;
  }
  b->allocations.push_back(q);
  *p = static_cast<T*>(q);
  return MIS2_OK;
}

// Per-level outputs grow on demand; a repeated run with the same sizes
// allocates nothing.
int ensure_level_storage(mis2_batch* b, BatchLevel& L, int64_t n, int64_t nnz) {
  if (L.cap_labels < n) {
    MIS2_TRY(balloc(b, &L.labels, n));
    L.cap_labels = n;
  }
  if (L.cap_crp < n + 1) {
    MIS2_TRY(balloc(b, &L.c_rowptr, n + 1));
    L.cap_crp = n + 1;
  }
  if (L.cap_cci < nnz) {
    MIS2_TRY(balloc(b, &L.c_colind, nnz));
    L.cap_cci = nnz;
  }
  return MIS2_OK;
}

// Per-graph tables, each (max_graphs + 1) int64 in d_tab / h_tab; the last
// two take 2 * (max_graphs + 1) entries.
enum { kTabVoff = 0, kTabR1 = 2, kTabQ = 3, kTabN1 = 4, kTabAgg = 5, kTabEoff = 6, kTabSrcA = 8, kTabCount = 10 };

}  // namespace

extern "C" {

int mis2_batch_create(mis2_batch** out, int32_t max_graphs, int64_t max_total_n, int64_t max_total_nnz,
                      const mis2_config* cfg) {
  if (out == nullptr) return MIS2_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_graphs < 1 || max_total_n < 1 || max_total_nnz < 0 || max_total_n >= ((int64_t)1 << 31) ||
      max_total_nnz >= ((int64_t)1 << 31) ||
      (cfg != nullptr && (cfg->ablation & (MIS2_ABLATE_TUPLE_ENGINE | MIS2_ABLATE_UNPACKED_TUPLES)) != 0))
    return MIS2_ERR_INVALID_ARG;
  mis2_batch* b = new mis2_batch();
  b->max_graphs = max_graphs;
  b->max_total_n = max_total_n;
  b->max_total_nnz = max_total_nnz;
  int rc = mis2_ctx_create(&b->ctx, max_total_n, max_total_nnz, cfg);
  const int64_t tg = (int64_t)max_graphs + 1;
  for (int k = 0; rc == MIS2_OK && k < 2; k++) {
    rc = balloc(b, &b->u_rowptr[k], max_total_n + 1);
    if (rc == MIS2_OK) rc = balloc(b, &b->u_colind[k], max_total_nnz + 4);
  }
  if (rc == MIS2_OK) rc = balloc(b, &b->gid, max_total_n);
  if (rc == MIS2_OK) rc = balloc(b, &b->d_tab, kTabCount * tg);
  if (rc == MIS2_OK) rc = balloc(b, &b->d_tab32, 2 * tg);
  if (rc == MIS2_OK) rc = balloc(b, &b->d_src, tg);
  if (rc == MIS2_OK && cudaMallocHost(&b->h_tab, kTabCount * tg * sizeof(int64_t)) != cudaSuccess)
    rc = MIS2_ERR_OUT_OF_MEMORY;
  if (rc != MIS2_OK) {
    mis2_batch_destroy(b);
    return rc;
  }
  *out = b;
  return MIS2_OK;
}

int mis2_batch_destroy(mis2_batch* b) {
  if (b == nullptr) return MIS2_OK;
  cudaDeviceSynchronize();
  for (void* p : b->allocations) cudaFree(p);
  if (b->h_tab) cudaFreeHost(b->h_tab);
  if (b->ctx) mis2_ctx_destroy(b->ctx);
  delete b;
  return MIS2_OK;
}

int mis2_batch_coarsen(mis2_batch* b, int32_t n_graphs, const mis2_csr* graphs, uint64_t seed, int64_t min_n,
                       int32_t max_levels, int32_t* n_levels_out, void* stream) {
  if (b == nullptr || graphs == nullptr || n_graphs < 1 || n_graphs > b->max_graphs || max_levels < 1 ||
      min_n < 0)
    return MIS2_ERR_INVALID_ARG;
  mis2_ctx* c = b->ctx;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t tg = (int64_t)b->max_graphs + 1;
  int64_t* tab = b->h_tab;
  // ---------------------------------------------------------------- level-0 union
  std::vector<GraphSrc> src(n_graphs);
  int64_t vo = 0, eo = 0, maxn = 0;
  for (int g = 0; g < n_graphs; g++) {
    const mis2_csr& gr = graphs[g];
    if (gr.n < 0 || gr.nnz < 0 || gr.rowptr == nullptr || (gr.nnz > 0 && gr.colind == nullptr))
      return MIS2_ERR_INVALID_ARG;
    src[g] = GraphSrc{gr.rowptr, gr.colind, gr.n, gr.nnz, vo, eo, gr.rowptr_is_64, 0};
    vo += gr.n;
    eo += gr.nnz;
    maxn = std::max(maxn, gr.n);
  }
  if (vo > b->max_total_n || eo > b->max_total_nnz) return MIS2_ERR_OUT_OF_MEMORY;
  b->n_graphs = n_graphs;
  b->lvl_n.clear();
  b->lvl_naggs.clear();
  b->lvl_cnnz.clear();
  c->launches = 0;
  timer_reset(c);
  memset(c->stats.kernel_ms, 0, sizeof(c->stats.kernel_ms));
  memset(c->stats.kernel_launches, 0, sizeof(c->stats.kernel_launches));
  // graphs below the threshold are not coarsened at all; the rest form the
  // level-0 union
  int cur = 0;
  std::vector<int32_t> live(n_graphs);
  std::vector<int64_t> live_n(n_graphs), live_nnz(n_graphs);
  std::vector<GraphSrc> keep;
  int nl = 0;
  int64_t un = 0, unnz = 0;
  for (int g = 0; g < n_graphs; g++) {
    if (src[g].n < min_n || src[g].n == 0) continue;
    live[nl] = g;
    live_n[nl] = src[g].n;
    live_nnz[nl] = src[g].nnz;
    keep.push_back(src[g]);
    keep.back().voff = un;
    keep.back().eoff = unnz;
    un += src[g].n;
    unnz += src[g].nnz;
    nl++;
  }
  if (nl > 0) {
    MIS2_CUDA(cudaMemcpyAsync(b->d_src, keep.data(), nl * sizeof(GraphSrc), cudaMemcpyHostToDevice, st));
    dim3 grid((unsigned)std::min<int64_t>(64, std::max<int64_t>(1, (maxn + kBlock - 1) / kBlock)), (unsigned)nl);
    k_union_build<<<grid, kBlock, 0, st>>>(b->d_src, b->u_rowptr[cur], b->u_colind[cur], b->gid);
    k_union_end<<<1, 1, 0, st>>>(b->u_rowptr[cur], un, unnz);
    c->launches += 2;
    MIS2_CUDA(cudaGetLastError());
  }
  // per-level loop
  int level = 0;
  std::vector<int64_t> voff(nl + 1);
  voff[0] = 0;
  for (int i = 0; i < nl; i++) voff[i + 1] = voff[i] + live_n[i];
  while (nl > 0 && level < max_levels) {
    if ((int)b->levels.size() <= level) b->levels.emplace_back();
    BatchLevel& L = b->levels[level];
    MIS2_TRY(ensure_level_storage(b, L, un, unnz));
    MIS2_CUDA(cudaStreamSynchronize(st));  // h_tab uploads of the previous level are done
    L.n_union = un;
    L.nnz_union = unnz;
    L.graph.assign(live.begin(), live.begin() + nl);
    L.voff.assign(voff.begin(), voff.begin() + nl + 1);
    // tables: voff, gbits
    for (int i = 0; i <= nl; i++) tab[kTabVoff * tg + i] = voff[i];
    std::vector<int32_t> bits(nl);
    for (int i = 0; i < nl; i++) bits[i] = id_bits(live_n[i]);
    MIS2_CUDA(cudaMemcpyAsync(b->d_tab + kTabVoff * tg, tab + kTabVoff * tg, (nl + 1) * sizeof(int64_t),
                              cudaMemcpyHostToDevice, st));
    MIS2_CUDA(cudaMemcpyAsync(b->d_tab32, bits.data(), nl * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    GraphArgs ga{un, unnz, false, b->u_rowptr[cur], b->u_colind[cur], true};
    PrioCfg p = make_prio(c, un, seed);
    p.gid = b->gid;
    p.voff = b->d_tab + kTabVoff * tg;
    p.gbits = b->d_tab32;
    // MIS-2 of every graph at once
    int64_t R1 = 0;
    int32_t r1 = 0;
    MIS2_TRY(run_impl(c, ga, p, nullptr, c->s.roots_tmp, &R1, &r1, st));
    L.rounds = r1;
    k_lower_bounds<<<(nl + 1 + 127) / 128, 128, 0, st>>>(c->s.roots_tmp, c->s.ctr + kCtrRoots,
                                                         b->d_tab + kTabVoff * tg, nl + 1, b->d_tab + kTabR1 * tg);
    c->launches++;
    // phase 1 with temporary ids = global root rank
    MIS2_TRY(agg_phase1(c, ga, c->s.roots_tmp, R1, L.labels, st));
    int64_t NQ = 0;
    int32_t r2 = 0;
    if (c->cfg.agg_mode == MIS2_AGG_ALG3) {
      MIS2_TRY(agg_phase2(c, ga, p, L.labels, (int32_t)R1, &r2, &NQ, st));
      k_lower_bounds<<<(nl + 1 + 127) / 128, 128, 0, st>>>(c->s.qlist, c->s.ctr + kCtrQual,
                                                           b->d_tab + kTabVoff * tg, nl + 1, b->d_tab + kTabQ * tg);
      c->launches++;
    } else {
      MIS2_CUDA(cudaMemsetAsync(b->d_tab + kTabQ * tg, 0, (nl + 1) * sizeof(int64_t), st));
    }
    L.rounds2 = r2;
    MIS2_CUDA(cudaMemcpyAsync(tab + kTabR1 * tg, b->d_tab + kTabR1 * tg, 2 * tg * sizeof(int64_t),
                              cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    // per graph: phase-1 and phase-2 aggregates, aggregate offsets
    std::vector<int64_t> n1(nl), nq(nl), naggs(nl);
    L.r1off.assign(tab + kTabR1 * tg, tab + kTabR1 * tg + nl + 1);
    L.aggoff.assign(nl + 1, 0);
    for (int i = 0; i < nl; i++) {
      n1[i] = tab[kTabR1 * tg + i + 1] - tab[kTabR1 * tg + i];
      nq[i] = tab[kTabQ * tg + i + 1] - tab[kTabQ * tg + i];
      naggs[i] = n1[i] + nq[i];
      L.aggoff[i + 1] = L.aggoff[i] + naggs[i];
      tab[kTabN1 * tg + i] = n1[i];
      tab[kTabAgg * tg + i] = L.aggoff[i];
    }
    tab[kTabAgg * tg + nl] = L.aggoff[nl];
    MIS2_CUDA(cudaMemcpyAsync(b->d_tab + kTabN1 * tg, tab + kTabN1 * tg, 2 * tg * sizeof(int64_t),
                              cudaMemcpyHostToDevice, st));
    RemapTables rt{b->gid, b->d_tab + kTabR1 * tg, b->d_tab + kTabQ * tg, b->d_tab + kTabN1 * tg,
                   b->d_tab + kTabAgg * tg, R1};
    k_remap_labels<<<grid_for(c, un, kBlock), kBlock, 0, st>>>(un, L.labels, rt);
    c->launches++;
    MIS2_CUDA(cudaGetLastError());
    const int64_t total = R1 + NQ;
    MIS2_TRY(agg_phase3(c, ga, L.labels, total, st));
    // coarse union graph
    int64_t cn = 0;
    MIS2_TRY(coarsen_impl(c, ga, L.labels, total, L.c_rowptr, L.c_colind, L.cap_cci, &cn, st));
    L.n_aggs = total;
    L.c_nnz = cn;
    // coarse entry range of every live graph inside the coarse union
    for (int i = 0; i < nl; i++) {
      tab[kTabEoff * tg + 2 * i] = L.aggoff[i];
      tab[kTabEoff * tg + 2 * i + 1] = L.aggoff[i + 1];
    }
    MIS2_CUDA(cudaMemcpyAsync(b->d_tab + kTabEoff * tg, tab + kTabEoff * tg, 2 * nl * sizeof(int64_t),
                              cudaMemcpyHostToDevice, st));
    int64_t* d_ebounds = b->d_tab + kTabSrcA * tg;
    k_gather_i32<<<(2 * nl + 127) / 128, 128, 0, st>>>(L.c_rowptr, b->d_tab + kTabEoff * tg, 2 * nl, d_ebounds);
    c->launches++;
    MIS2_CUDA(cudaMemcpyAsync(tab + kTabSrcA * tg, d_ebounds, 2 * nl * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    std::vector<int64_t> ebl(2 * nl);
    for (int j = 0; j < 2 * nl; j++) ebl[j] = tab[kTabSrcA * tg + j];
    L.ebounds = ebl;
    // record sizes per input graph
    b->lvl_n.emplace_back(n_graphs, 0);
    b->lvl_naggs.emplace_back(n_graphs, 0);
    b->lvl_cnnz.emplace_back(n_graphs, 0);
    for (int i = 0; i < nl; i++) {
      b->lvl_n[level][live[i]] = live_n[i];
      b->lvl_naggs[level][live[i]] = naggs[i];
      b->lvl_cnnz[level][live[i]] = ebl[2 * i + 1] - ebl[2 * i];
    }
    level++;
    // graphs that keep coarsening: still >= min_n and shrinking
    std::vector<int32_t> nxt;
    for (int i = 0; i < nl; i++)
      if (naggs[i] >= min_n && naggs[i] < live_n[i] && naggs[i] > 0) nxt.push_back(i);
    if (nxt.empty() || level >= max_levels) break;
    const int nn = (int)nxt.size();
    std::vector<int64_t> eb(2 * nn);
    for (int j = 0; j < nn; j++) {
      eb[2 * j] = ebl[2 * nxt[j]];
      eb[2 * j + 1] = ebl[2 * nxt[j] + 1];
    }
    std::vector<int64_t> dvoff(nn + 1, 0), deoff(nn + 1, 0);
    std::vector<int32_t> srcg(nn);
    std::vector<int64_t> srcaoff(nl + 1);
    int64_t maxrows = 0;
    for (int j = 0; j < nn; j++) {
      const int i = nxt[j];
      srcg[j] = i;
      dvoff[j + 1] = dvoff[j] + naggs[i];
      deoff[j + 1] = deoff[j] + (eb[2 * j + 1] - eb[2 * j]);
      maxrows = std::max(maxrows, naggs[i]);
    }
    for (int i = 0; i <= nl; i++) srcaoff[i] = L.aggoff[i];
    // tables for the compaction: src graph (int32), src aggoff, dst voff, dst eoff
    for (int i = 0; i <= nl; i++) tab[kTabAgg * tg + i] = srcaoff[i];
    for (int j = 0; j <= nn; j++) {
      tab[kTabVoff * tg + j] = dvoff[j];
      tab[kTabEoff * tg + j] = deoff[j];
    }
    MIS2_CUDA(cudaMemcpyAsync(b->d_tab + kTabAgg * tg, tab + kTabAgg * tg, (nl + 1) * sizeof(int64_t),
                              cudaMemcpyHostToDevice, st));
    MIS2_CUDA(cudaMemcpyAsync(b->d_tab + kTabVoff * tg, tab + kTabVoff * tg, (nn + 1) * sizeof(int64_t),
                              cudaMemcpyHostToDevice, st));
    MIS2_CUDA(cudaMemcpyAsync(b->d_tab + kTabEoff * tg, tab + kTabEoff * tg, (nn + 1) * sizeof(int64_t),
                              cudaMemcpyHostToDevice, st));
    MIS2_CUDA(cudaMemcpyAsync(b->d_tab32 + tg, srcg.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const int nxt_buf = cur ^ 1;
    CompactTables ct{b->d_tab32 + tg, b->d_tab + kTabAgg * tg, b->d_tab + kTabVoff * tg, b->d_tab + kTabEoff * tg,
                     nn};
    dim3 grid((unsigned)std::min<int64_t>(64, std::max<int64_t>(1, (maxrows + kBlock - 1) / kBlock)), (unsigned)nn);
    k_union_compact<<<grid, kBlock, 0, st>>>(L.c_rowptr, L.c_colind, ct, b->u_rowptr[nxt_buf], b->u_colind[nxt_buf],
                                            b->gid);
    k_union_end<<<1, 1, 0, st>>>(b->u_rowptr[nxt_buf], dvoff[nn], deoff[nn]);
    c->launches += 2;
    MIS2_CUDA(cudaGetLastError());
    // the next level's live set
    std::vector<int32_t> live2(nn);
    std::vector<int64_t> n2(nn), nnz2(nn);
    for (int j = 0; j < nn; j++) {
      live2[j] = live[nxt[j]];
      n2[j] = naggs[nxt[j]];
      nnz2[j] = deoff[j + 1] - deoff[j];
    }
    for (int j = 0; j < nn; j++) {
      live[j] = live2[j];
      live_n[j] = n2[j];
      live_nnz[j] = nnz2[j];
    }
    nl = nn;
    voff.assign(dvoff.begin(), dvoff.end());
    un = dvoff[nn];
    unnz = deoff[nn];
    cur = nxt_buf;
  }
  MIS2_CUDA(cudaStreamSynchronize(st));
  b->n_levels = level;
  if (n_levels_out) *n_levels_out = level;
  return timer_collect(c);
}

int mis2_batch_level_sizes(const mis2_batch* b, int32_t level, int64_t* n, int64_t* n_aggs, int64_t* c_nnz) {
  if (b == nullptr || level < 0 || level >= b->n_levels) return MIS2_ERR_INVALID_ARG;
  for (int g = 0; g < b->n_graphs; g++) {
    if (n) n[g] = b->lvl_n[level][g];
    if (n_aggs) n_aggs[g] = b->lvl_naggs[level][g];
    if (c_nnz) c_nnz[g] = b->lvl_cnnz[level][g];
  }
  return MIS2_OK;
}

static int find_live(const mis2_batch* b, int32_t level, int32_t graph, int* li) {
  if (b == nullptr || level < 0 || level >= b->n_levels || graph < 0 || graph >= b->n_graphs)
    return MIS2_ERR_INVALID_ARG;
  const BatchLevel& L = b->levels[level];
  for (int i = 0; i < (int)L.graph.size(); i++)
    if (L.graph[i] == graph) {
      *li = i;
      return MIS2_OK;
    }
  return MIS2_ERR_INVALID_ARG;  // the graph was not coarsened at this level
}

int mis2_batch_labels(const mis2_batch* b, int32_t level, int32_t graph, int32_t* labels, void* stream) {
  int li = 0;
  MIS2_TRY(find_live(b, level, graph, &li));
  if (labels == nullptr) return MIS2_ERR_INVALID_ARG;
  const BatchLevel& L = b->levels[level];
  const int64_t n = L.voff[li + 1] - L.voff[li];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_sub_copy<<<grid_for(b->ctx, n, kBlock), kBlock, 0, st>>>(L.labels + L.voff[li], n, L.aggoff[li], labels);
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

int mis2_batch_coarse(const mis2_batch* b, int32_t level, int32_t graph, int32_t* c_rowptr, int32_t* c_colind,
                      int64_t c_colind_cap, void* stream) {
  int li = 0;
  MIS2_TRY(find_live(b, level, graph, &li));
  if (c_rowptr == nullptr) return MIS2_ERR_INVALID_ARG;
  const BatchLevel& L = b->levels[level];
  const int64_t a0 = L.aggoff[li], na = L.aggoff[li + 1] - a0;
  if (b->lvl_cnnz[level][graph] > c_colind_cap) return MIS2_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t base = 0, end = 0;
  MIS2_CUDA(cudaMemcpyAsync(&base, L.c_rowptr + a0, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaMemcpyAsync(&end, L.c_rowptr + a0 + na, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  k_sub_copy<<<grid_for(b->ctx, na + 1, kBlock), kBlock, 0, st>>>(L.c_rowptr + a0, na + 1, base, c_rowptr);
  if (end > base) {
    if (c_colind == nullptr) return MIS2_ERR_INVALID_ARG;
    k_sub_copy<<<grid_for(b->ctx, end - base, kBlock), kBlock, 0, st>>>(L.c_colind + base, end - base, a0, c_colind);
  }
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

int mis2_batch_stats(const mis2_batch* b, mis2_stats* out) {
  if (b == nullptr || out == nullptr) return MIS2_ERR_INVALID_ARG;
  return mis2_get_stats(b->ctx, out);
}

}  // extern "C"

namespace mis2 {

mis2_ctx* batch_context(mis2_batch* b) { return b->ctx; }

int batch_level0_result(const mis2_batch* b, int32_t graph, int32_t* roots, int32_t* labels, int32_t* c_rowptr,
                        int32_t* c_colind, int64_t* n_roots, int64_t* n_aggs, int64_t* c_nnz, cudaStream_t st) {
  int li = 0;
  MIS2_TRY(find_live(b, 0, graph, &li));
  const BatchLevel& L = b->levels[0];
  const int64_t v0 = L.voff[li], n = L.voff[li + 1] - v0;
  const int64_t a0 = L.aggoff[li], na = L.aggoff[li + 1] - a0;
  const int64_t r0 = L.r1off[li], nr = L.r1off[li + 1] - r0;
  const int64_t e0 = L.ebounds[2 * li], ne = L.ebounds[2 * li + 1] - e0;
  if (nr > 0)
    k_sub_copy<<<grid_for(b->ctx, nr, kBlock), kBlock, 0, st>>>(b->ctx->s.roots_tmp + r0, nr, v0, roots);
  if (n > 0) k_sub_copy<<<grid_for(b->ctx, n, kBlock), kBlock, 0, st>>>(L.labels + v0, n, a0, labels);
  k_sub_copy<<<grid_for(b->ctx, na + 1, kBlock), kBlock, 0, st>>>(L.c_rowptr + a0, na + 1, e0, c_rowptr);
  if (ne > 0) k_sub_copy<<<grid_for(b->ctx, ne, kBlock), kBlock, 0, st>>>(L.c_colind + e0, ne, a0, c_colind);
  MIS2_CUDA(cudaGetLastError());
  *n_roots = nr;
  *n_aggs = na;
  *c_nnz = ne;
  return MIS2_OK;
}

}  // namespace mis2
