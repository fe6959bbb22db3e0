// agg.cu -- MIS-2 aggregation, Algorithm 3 (Section III-B), with Algorithm 2
// as the BASIC mode:
//   phase 1  every MIS-2 root and its neighbours form an aggregate;
//   phase 2  (Alg. 3 only) MIS-2 of the subgraph of unaggregated vertices;
//            a root with >= 2 unaggregated neighbours claims them;
//   phase 3  each leftover joins the adjacent aggregate of maximum coupling
//            (ties: minimum tentative size, then minimum id), coupling and
//            sizes read from the frozen "tentative" labels.
// Aggregate ids: phase-1 roots in ascending order, then qualifying phase-2
// roots in ascending order.
#include <algorithm>

#include "internal.h"
#include "mis_rows.cuh"

namespace mis2 {

constexpr int kErrNoAggregatedNeighbour = 2;
constexpr int kPhase3Window = 8192;

// Root list entry j claims itself and every neighbour still labelled -1 for
// aggregate base + j.  Roots are more than two hops apart (in the graph, or
// in the phase-2 subgraph), so no two claims touch the same vertex.  Rows of
// degree >= block_degree are deferred to the block kernel.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_agg_claim(GraphView<I> g, const int32_t* list, int64_t n_host,
                                                      const int32_t* n_dev, int32_t* labels, int32_t base,
                                                      int32_t* heavy, int32_t* heavy_cnt, int32_t block_degree) {
  const int64_t cnt = n_dev != nullptr ? *n_dev : n_host;
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt; j += nw) {
    const int32_t v = list[j];
    int64_t s, e;
    row_range(g, v, s, e);
    if (e - s >= block_degree) {
      if (lane == 0) heavy[atomicAdd(heavy_cnt, 1)] = (int32_t)j;
      continue;
    }
    const int32_t id = base + (int32_t)j;
    if (lane == 0) labels[v] = id;
    visit_row<32>(g.colind, g.nnz, s, e, lane, g.vec, [&](int32_t w) {
      if (w != v && labels[w] == -1) labels[w] = id;
    });
  }
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_agg_claim_block(GraphView<I> g, const int32_t* list,
                                                            const int32_t* heavy, const int32_t* heavy_cnt,
                                                            int32_t* labels, int32_t base) {
  const int64_t cnt = *heavy_cnt;
  for (int64_t h = blockIdx.x; h < cnt; h += gridDim.x) {
    const int32_t j = heavy[h];
    const int32_t v = list[j];
    int64_t s, e;
    row_range(g, v, s, e);
    const int32_t id = base + j;
    if (threadIdx.x == 0) labels[v] = id;
    visit_row<kBlock>(g.colind, g.nnz, s, e, threadIdx.x, g.vec, [&](int32_t w) {
      if (w != v && labels[w] == -1) labels[w] = id;
    });
  }
}

// Phase 2 test: qflag[v] = 1 for a phase-2 root v with >= 2 unaggregated
// neighbours u != v (labels at the end of phase 1).  Warp per root.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_qualify(GraphView<I> g, const int32_t* list, const int32_t* n_dev,
                                                    const int32_t* labels, uint8_t* qflag) {
  const int64_t cnt = *n_dev;
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt; j += nw) {
    const int32_t v = list[j];
    int64_t s, e;
    row_range(g, v, s, e);
    int c = 0;
    visit_row<32>(g.colind, g.nnz, s, e, lane, g.vec, [&](int32_t w) { c += (w != v && labels[w] == -1); });
    c = group_sum<32>(c);
    if (lane == 0) qflag[v] = c >= 2 ? 1 : 0;
  }
}

// aggsize(a) = |{v : tent_v = a}|, one atomic per distinct label per warp.
__global__ void __launch_bounds__(kBlock) k_aggsize(int64_t n, const int32_t* tent, int32_t* aggsize) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = lane_id();
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += stride) {
    const int64_t v = base + lane;
    const int32_t a = v < n ? tent[v] : -1;
    const unsigned peers = __match_any_sync(kFull, a);
    if (a >= 0 && lane == __ffs(peers) - 1) atomicAdd(aggsize + a, __popc(peers));
  }
}

// Leftovers of phases 1-2, split by degree (block rows go to `heavy`).
template <typename I>
__global__ void __launch_bounds__(kBlock) k_leftovers(GraphView<I> g, const int32_t* tent, int32_t* left,
                                                      int32_t* left_cnt, int32_t* heavy, int32_t* heavy_cnt,
                                                      int32_t block_degree) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = lane_id();
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < g.n; base += stride) {
    const int64_t v = base + lane;
    bool lo = false, hi = false;
    if (v < g.n && tent[v] == -1) {
      int64_t s, e;
      row_range(g, v, s, e);
      (e - s >= block_degree ? hi : lo) = true;
    }
    warp_append(lo, (int32_t)v, left, left_cnt);
    warp_append(hi, (int32_t)v, heavy, heavy_cnt);
  }
}

__device__ __forceinline__ bool better(int c, int sz, int a, int bc, int bs, int ba) {
  return ba < 0 || c > bc || (c == bc && (sz < bs || (sz == bs && a < ba)));
}

// Phase 3, group of G lanes per leftover: visit the adjacent aggregates in
// increasing id order (one min-reduction per distinct id), count coupling
// for each, keep the best by (max coupling, min size, min id).
template <int G, typename I>
__global__ void __launch_bounds__(kBlock) k_phase3(GraphView<I> g, const int32_t* tent, const int32_t* aggsize,
                                                   const int32_t* left, const int32_t* left_cnt, int32_t* labels,
                                                   int32_t* err) {
  constexpr int RPW = 32 / G;
  const int64_t cnt = *left_cnt;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * RPW; base < cnt; base += nw * RPW) {
    const int64_t i = base + sub;
    const bool active = i < cnt;
    int32_t v = 0;
    int64_t s = 0, e = 0;
    if (active) {
      v = left[i];
      row_range(g, v, s, e);
    }
    bool done = !active;
    int32_t last = -1, best = -1;
    int bc = 0, bs = 0;
    while (__any_sync(kFull, !done)) {
      uint32_t a = 0xFFFFFFFFu;
      if (!done)
        visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) {
          const int32_t t = tent[w];
          if (w != v && t > last && (uint32_t)t < a) a = (uint32_t)t;
        });
      a = group_min<G>(a);
      int c = 0;
      if (!done && a != 0xFFFFFFFFu)
        visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) { c += (w != v && tent[w] == (int32_t)a); });
      c = group_sum<G>(c);
      if (!done) {
        if (a == 0xFFFFFFFFu) {
          done = true;
        } else {
          const int sz = aggsize[a];
          if (better(c, sz, (int32_t)a, bc, bs, best)) {
            best = (int32_t)a;
            bc = c;
            bs = sz;
          }
          last = (int32_t)a;
        }
      }
    }
    if (active && lg == 0) {
      labels[v] = best;
      if (best < 0) atomicOr(err, kErrNoAggregatedNeighbour);
    }
  }
}

// Phase 3 for leftovers of degree >= block_degree: count coupling in
// shared-memory windows of kPhase3Window aggregate ids.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_phase3_block(GraphView<I> g, const int32_t* tent,
                                                         const int32_t* aggsize, const int32_t* list,
                                                         const int32_t* list_cnt, int32_t* labels, int32_t* err) {
  __shared__ int cnt[kPhase3Window];
  __shared__ uint32_t sh[40];
  const int64_t n_items = *list_cnt;
  for (int64_t i = blockIdx.x; i < n_items; i += gridDim.x) {
    const int32_t v = list[i];
    int64_t s, e;
    row_range(g, v, s, e);
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    visit_row<kBlock>(g.colind, g.nnz, s, e, threadIdx.x, g.vec, [&](int32_t w) {
      const int32_t t = tent[w];
      if (w != v && t >= 0) {
        lo = min(lo, (uint32_t)t);
        hi = max(hi, (uint32_t)t);
      }
    });
    lo = block_min_u32(lo, sh);
    hi = block_max_u32(hi, sh);
    int32_t best = -1;
    int bc = 0, bs = 0;
    if (lo != 0xFFFFFFFFu) {
      for (int64_t wb = lo; wb <= (int64_t)hi; wb += kPhase3Window) {
        for (int j = threadIdx.x; j < kPhase3Window; j += blockDim.x) cnt[j] = 0;
        __syncthreads();
        visit_row<kBlock>(g.colind, g.nnz, s, e, threadIdx.x, g.vec, [&](int32_t w) {
          const int32_t t = tent[w];
          if (w != v && t >= wb && t < wb + kPhase3Window) atomicAdd(&cnt[t - wb], 1);
        });
        __syncthreads();
        int lc = 0, ls = 0;
        int32_t la = -1;
        for (int j = threadIdx.x; j < kPhase3Window; j += blockDim.x) {
          const int c = cnt[j];
          if (c > 0) {
            const int32_t a = (int32_t)(wb + j);
            const int sz = aggsize[a];
            if (better(c, sz, a, lc, ls, la)) {
              la = a;
              lc = c;
              ls = sz;
            }
          }
        }
        // block argmax by (max c, min size, min id) as three reductions
        const uint32_t mc = block_max_u32(la >= 0 ? (uint32_t)lc : 0u, sh);
        const uint32_t ms = block_min_u32(la >= 0 && (uint32_t)lc == mc ? (uint32_t)ls : 0xFFFFFFFFu, sh);
        const uint32_t ma = block_min_u32(la >= 0 && (uint32_t)lc == mc && (uint32_t)ls == ms ? (uint32_t)la
                                                                                                  : 0xFFFFFFFFu,
                                          sh);
        if (mc > 0 && better((int)mc, (int)ms, (int32_t)ma, bc, bs, best)) {
          best = (int32_t)ma;
          bc = (int)mc;
          bs = (int)ms;
        }
      }
    }
    if (threadIdx.x == 0) {
      labels[v] = best;
      if (best < 0) atomicOr(err, kErrNoAggregatedNeighbour);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host side
template <typename I>
static GraphView<I> gview(const GraphArgs& g) {
  GraphView<I> v;
  v.rowptr = static_cast<const I*>(g.rowptr);
  v.colind = g.colind;
  v.n = g.n;
  v.nnz = g.nnz;
  v.vec = g.vec ? 1 : 0;
  v.pad = 0;
  return v;
}

template <typename I>
static void launch_claim(mis2_ctx* c, const GraphView<I>& gv, const int32_t* list, int64_t n_host,
                         const int32_t* n_dev, int32_t* labels, int32_t base, cudaStream_t st) {
  Scratch& s = c->s;
  const int64_t items = n_dev != nullptr ? gv.n : n_host;
  cudaMemsetAsync(s.ctr + kCtrHeavy, 0, sizeof(int32_t), st);
  k_agg_claim<I><<<grid_for(c, items, kBlock / 32), kBlock, 0, st>>>(gv, list, n_host, n_dev, labels, base,
                                                                      s.left_heavy, s.ctr + kCtrHeavy,
                                                                      c->cfg.block_degree);
  k_agg_claim_block<I><<<c->sm_count * 2, kBlock, 0, st>>>(gv, list, s.left_heavy, s.ctr + kCtrHeavy, labels,
                                                           base);
  c->launches += 2;
}

template <typename I>
static void launch_phase3(mis2_ctx* c, const GraphView<I>& gv, int G, int32_t* labels, cudaStream_t st) {
  Scratch& s = c->s;
  const int blocks = grid_for(c, gv.n, kBlock, 8);
#define MIS2_P3(GG)                                                                                   \
  k_phase3<GG, I><<<blocks, kBlock, 0, st>>>(gv, s.tent, s.aggsize, s.left, s.ctr + kCtrLeft, labels, \
                                             s.ctr + kCtrErr)
  switch (G) {
    case 1: MIS2_P3(1); break;
    case 2: MIS2_P3(2); break;
    case 4: MIS2_P3(4); break;
    case 8: MIS2_P3(8); break;
    case 16: MIS2_P3(16); break;
    default: MIS2_P3(32); break;
  }
#undef MIS2_P3
  k_phase3_block<I><<<c->sm_count * 2, kBlock, 0, st>>>(gv, s.tent, s.aggsize, s.left_heavy,
                                                        s.ctr + kCtrLeftHeavy, labels, s.ctr + kCtrErr);
  c->launches += 2;
}

template <typename I>
static int aggregate_t(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, int64_t n_roots, uint64_t seed,
                       int mode, int32_t* labels, int64_t* n_aggs, cudaStream_t st) {
  Scratch& s = c->s;
  const GraphView<I> gv = gview<I>(g);
  const int64_t n = g.n;
  c->stats.rounds2 = 0;
  memset(c->stats.trace2, 0, sizeof(c->stats.trace2));
  if (n == 0) {
    *n_aggs = 0;
    return MIS2_OK;
  }
  MIS2_CUDA(cudaMemsetAsync(labels, 0xFF, n * sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrM2, 0, (kCtrErr - kCtrM2 + 1) * sizeof(int32_t), st));
  // phase 1
  timer_begin(c, kKcAggregate, st);
  launch_claim<I>(c, gv, roots, n_roots, nullptr, labels, 0, st);
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  int64_t nq = 0;
  if (mode == MIS2_AGG_ALG3) {
    // phase 2: MIS-2 of G minus the aggregated vertices
    const PrioCfg p = make_prio(c, n, seed);
    int32_t r2 = 0;
    if (c->cfg.loop == MIS2_LOOP_DEVICE)
      MIS2_TRY(mis2_rounds_device(c, g, labels, p, 1, st, &r2));
    else
      MIS2_TRY(mis2_rounds_host(c, g, labels, p, 1, st, &r2));
    c->stats.rounds2 = r2;
    MIS2_TRY(extract_in_set(c, n, nullptr, s.roots2, s.ctr + kCtrM2, st));
    MIS2_CUDA(cudaMemsetAsync(s.qflag, 0, n, st));
    timer_begin(c, kKcAggregate, st);
    k_qualify<I><<<grid_for(c, n, kBlock / 32), kBlock, 0, st>>>(gv, s.roots2, s.ctr + kCtrM2, labels, s.qflag);
    c->launches++;
    timer_end(c, st);
    MIS2_CUDA(cudaGetLastError());
    MIS2_TRY(compact_flags(c, s.qflag, nullptr, n, s.qlist, s.ctr + kCtrQual, st));
    timer_begin(c, kKcAggregate, st);
    launch_claim<I>(c, gv, s.qlist, 0, s.ctr + kCtrQual, labels, (int32_t)n_roots, st);
    timer_end(c, st);
    MIS2_CUDA(cudaGetLastError());
    MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    nq = c->h_ctr[kCtrQual];
  }
  const int64_t total = n_roots + nq;
  // phase 3: leftovers join by coupling, read from the frozen labels
  timer_begin(c, kKcAggregate, st);
  MIS2_CUDA(cudaMemcpyAsync(s.tent, labels, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  MIS2_CUDA(cudaMemsetAsync(s.aggsize, 0, std::max<int64_t>(total, 1) * sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrLeft, 0, 2 * sizeof(int32_t), st));
  k_aggsize<<<grid_for(c, n, kBlock), kBlock, 0, st>>>(n, s.tent, s.aggsize);
  k_leftovers<I><<<grid_for(c, n, kBlock), kBlock, 0, st>>>(gv, s.tent, s.left, s.ctr + kCtrLeft, s.left_heavy,
                                                             s.ctr + kCtrLeftHeavy, c->cfg.block_degree);
  c->launches += 2;
  launch_phase3<I>(c, gv, pick_group_lanes(c, g), labels, st);
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  if (c->h_ctr[kCtrErr] & kErrNoAggregatedNeighbour) return MIS2_ERR_BAD_GRAPH;
  *n_aggs = total;
  return MIS2_OK;
}

int aggregate_impl(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, int64_t n_roots, uint64_t seed, int mode,
                   int32_t* labels, int64_t* n_aggs, cudaStream_t st) {
  return g.rp64 ? aggregate_t<int64_t>(c, g, roots, n_roots, seed, mode, labels, n_aggs, st)
                : aggregate_t<int32_t>(c, g, roots, n_roots, seed, mode, labels, n_aggs, st);
}

}  // namespace mis2
