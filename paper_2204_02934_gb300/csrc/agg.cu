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
#include <cstring>

#include "internal.h"
#include "mis_rows.cuh"

namespace mis2 {

constexpr int kPhase3Window = 8192;   // aggregate ids counted per pass for the heaviest rows
constexpr int kPhase3SortCap = 8192;  // rows up to this length are sorted in shared memory

// Claim the entries of row [s, e) still labelled -1 (other than v itself)
// for aggregate id, lane lg of a group of G lanes taking 16-byte pieces.
// The labels of a piece are all read before any is written: the vertices one
// claim touches are distinct, and no other root's claim touches them, so the
// reads need not wait for one another.
template <int G>
__device__ __forceinline__ void claim_row(const int32_t* __restrict__ colind, int64_t nnz, int64_t s, int64_t e,
                                          int lg, bool vec, int32_t v, int32_t id, int32_t* labels) {
  if (vec) {
    for (int64_t p = (s & ~int64_t(3)) + 4 * lg; p < e; p += 4 * G) {
      int32_t w[4];
      if (p + 4 <= nnz) {
        const int4 q = __ldg(reinterpret_cast<const int4*>(colind + p));
        w[0] = q.x;
        w[1] = q.y;
        w[2] = q.z;
        w[3] = q.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; k++) w[k] = p + k < e ? __ldg(colind + p + k) : v;
      }
      bool in[4];
      int32_t l[4];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        in[k] = p + k >= s && p + k < e && w[k] != v;
        l[k] = in[k] ? labels[w[k]] : 0;
      }
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (in[k] && l[k] == -1) labels[w[k]] = id;
    }
  } else {
    for (int64_t p = s + lg; p < e; p += G) {
      const int32_t w = __ldg(colind + p);
      if (w != v && labels[w] == -1) labels[w] = id;
    }
  }
}

// Root list entry j claims itself and every neighbour still labelled -1 for
// aggregate base + j, a group of G lanes per root (32 / G roots in flight
// per warp).  Roots are more than two hops apart (in the graph, or in the
// phase-2 subgraph), so no two claims touch the same vertex.  Rows of
// degree >= block_degree are deferred to the block kernel.
template <int G, typename I>
__global__ void __launch_bounds__(kBlock) k_agg_claim(GraphView<I> g, const int32_t* list, int64_t n_host,
                                                      const int32_t* n_dev, int32_t* labels, int32_t base_host,
                                                      const int32_t* base_dev, int32_t* heavy, int32_t* heavy_cnt,
                                                      int32_t block_degree) {
  pdl_enter();
  constexpr int RPW = 32 / G;
  const int64_t cnt = n_dev != nullptr ? block_load(n_dev) : n_host;
  const int32_t base = base_dev != nullptr ? block_load(base_dev) : base_host;
  const int lane = lane_id(), lg = lane & (G - 1);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = warp * RPW + lane / G; j < cnt; j += nw * RPW) {
    const int32_t v = list[j];
    int64_t s, e;
    row_range(g, v, s, e);
    if (e - s >= block_degree) {
      if (lg == 0) heavy[atomicAdd(heavy_cnt, 1)] = (int32_t)j;
      continue;
    }
    const int32_t id = base + (int32_t)j;
    if (lg == 0) labels[v] = id;
    claim_row<G>(g.colind, g.nnz, s, e, lg, g.vec, v, id, labels);
  }
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_agg_claim_block(GraphView<I> g, const int32_t* list,
                                                            const int32_t* heavy, const int32_t* heavy_cnt,
                                                            int32_t* labels, int32_t base_host,
                                                            const int32_t* base_dev) {
  pdl_enter();
  const int64_t cnt = block_load(heavy_cnt);
  const int32_t base = base_dev != nullptr ? *base_dev : base_host;
  for (int64_t h = blockIdx.x; h < cnt; h += gridDim.x) {
    const int32_t j = heavy[h];
    const int32_t v = list[j];
    int64_t s, e;
    row_range(g, v, s, e);
    const int32_t id = base + j;
    if (threadIdx.x == 0) labels[v] = id;
    claim_row<kBlock>(g.colind, g.nnz, s, e, threadIdx.x, g.vec, v, id, labels);
  }
}

// Phase 2 test: qflag[v] = 1 for a phase-2 root v with >= 2 unaggregated
// neighbours u != v (labels at the end of phase 1).  A group of G lanes per
// root.
template <int G, typename I>
__global__ void __launch_bounds__(kBlock) k_qualify(GraphView<I> g, const int32_t* list, const int32_t* n_dev,
                                                    const int32_t* labels, uint8_t* qflag) {
  pdl_enter();
  constexpr int RPW = 32 / G;
  const int64_t cnt = block_load(n_dev);
  const int lane = lane_id(), lg = lane & (G - 1);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // every lane runs the same trip count: group_sum spans the warp
  for (int64_t jb = warp * RPW; jb < cnt; jb += nw * RPW) {
    const int64_t j = jb + lane / G;
    int c = 0;
    int32_t v = -1;
    if (j < cnt) {
      v = list[j];
      int64_t s, e;
      row_range(g, v, s, e);
      visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) { c += (w != v && labels[w] == -1); });
    }
    c = group_sum<G>(c);
    if (j < cnt && lg == 0) qflag[v] = c >= 2 ? 1 : 0;
  }
}

// aggsize(a) = |{v : tent_v = a}| (one atomic per distinct label per warp),
// and the leftovers of phases 1-2 split by degree: short rows (<=
// kLaneRowMax entries) to `left`, medium rows to `mid`, rows above
// kPhase3SortCap to `heavy`.  The appends of a block's 256 vertices take one
// reservation per list (one scan of the three counts packed in one word).
// labels_out (or null): receives tent_v for every aggregated v.
// fin (or null): the coarse graph's per-aggregate member counts and summed
// row lengths, started here from the aggregated vertices (phase 3 adds the
// leftovers), so that the coarse step needs no histogram pass of its own.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_aggsize_leftovers(GraphView<I> g, const int32_t* tent, int32_t* aggsize,
                                                              int32_t* labels_out, AggCounts fin, int32_t* left,
                                                              int32_t* left_cnt, int32_t* mid, int32_t* mid_cnt,
                                                              int32_t* heavy, int32_t* heavy_cnt) {
  pdl_enter();
  __shared__ int sh_scan[40];
  __shared__ int32_t sh_base[3];
  const int lane = lane_id();
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    const int32_t a = v < g.n ? tent[v] : -2;
    const unsigned peers = __match_any_sync(kFull, a);
    int deg = 0;
    if (v < g.n && (a == -1 || fin.cnt != nullptr)) {
      int64_t s, e;
      row_range(g, v, s, e);
      deg = (int)(e - s);
    }
    const bool leader = a >= 0 && lane == __ffs(peers) - 1;
    if (leader) atomicAdd(aggsize + a, __popc(peers));
    if (fin.cnt != nullptr) {
      // summed row lengths of the lanes holding the same label
      int sum = 0;
#pragma unroll
      for (int src = 0; src < 32; src++) {
        const int x = __shfl_sync(kFull, deg, src);
        if ((peers >> src) & 1u) sum += x;
      }
      if (leader) {
        atomicAdd(fin.cnt + a, __popc(peers));
        if (sum > 0) atomicAdd(fin.deg + a, sum);
      }
    }
    if (a >= 0 && labels_out != nullptr) labels_out[v] = a;
    int cls = -1;
    if (a == -1) cls = deg <= kLaneRowMax ? 0 : (deg <= kPhase3SortCap ? 1 : 2);
    // 10 bits per list: at most 256 entries of each per block
    const int x = cls < 0 ? 0 : 1 << (10 * cls);
    int total;
    const int pos = block_exclusive_scan(x, sh_scan, &total);
    if (threadIdx.x < 3) {
      const int k = threadIdx.x, nk = (total >> (10 * k)) & 1023;
      int32_t* ck = k == 0 ? left_cnt : (k == 1 ? mid_cnt : heavy_cnt);
      sh_base[k] = nk > 0 ? atomicAdd(ck, nk) : 0;
    }
    __syncthreads();
    if (cls >= 0) {
      int32_t* lk = cls == 0 ? left : (cls == 1 ? mid : heavy);
      lk[sh_base[cls] + ((pos >> (10 * cls)) & 1023)] = (int32_t)v;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ bool better(int c, int sz, int a, int bc, int bs, int ba) {
  return ba < 0 || c > bc || (c == bc && (sz < bs || (sz == bs && a < ba)));
}

// The best adjacent aggregate of one leftover from the tentative labels of
// its W row entries (lab[k] < 0: no aggregate, or not an entry): sort them
// in registers (a bitonic network with fixed indices), the coupling of an
// aggregate being the length of its run; then, over the runs of maximum
// length, the minimum size and, the runs lying in ascending label order, the
// first of those.  The sizes of those runs only are read, and all at once.
// Returns -1 when no entry has an aggregate.
template <int W>
__device__ __forceinline__ int32_t phase3_pick(int32_t (&lab)[kLaneRowMax], const int32_t* aggsize) {
  constexpr int32_t kNone = 0x7FFFFFFF;  // sorts after every label
#pragma unroll
  for (int k = 0; k < W; k++) lab[k] = lab[k] < 0 ? kNone : lab[k];
#pragma unroll
  for (int k = 2; k <= W; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i = 0; i < W; i++) {
        const int l = i ^ j;
        if (l > i) {
          const int32_t x = lab[i], y = lab[l];
          const bool up = (i & k) == 0;
          lab[i] = up ? min(x, y) : max(x, y);
          lab[l] = up ? max(x, y) : min(x, y);
        }
      }
    }
  }
  int cmax = 0, run = 0;
#pragma unroll
  for (int k = 0; k < W; k++) {
    run = (k > 0 && lab[k] == lab[k - 1]) ? run + 1 : 1;
    if (lab[k] != kNone) cmax = max(cmax, run);
  }
  if (cmax == 0) return -1;
  int32_t sz[W];
  run = 0;
#pragma unroll
  for (int k = 0; k < W; k++) {  // a run of length cmax ends at k: read its size
    run = (k > 0 && lab[k] == lab[k - 1]) ? run + 1 : 1;
    const bool end = lab[k] != kNone && run == cmax && (k == W - 1 || lab[k + 1] != lab[k]);
    sz[k] = end ? __ldg(aggsize + lab[k]) : 0x7FFFFFFF;
  }
  int32_t best = -1, bs = 0x7FFFFFFF;
#pragma unroll
  for (int k = 0; k < W; k++) {
    if (sz[k] < bs) {  // strict: equal sizes keep the smaller label, met first
      bs = sz[k];
      best = lab[k];
    }
  }
  return best;
}

// Phase 3, one lane per short leftover row: stage the row, gather its
// neighbours' tentative labels into registers, and pick the best adjacent
// aggregate by (max coupling, min size, min id).
// A leftover of row length deg joins aggregate a: count it into fin.
__device__ __forceinline__ void fin_add(const AggCounts& fin, int32_t a, int64_t deg) {
  if (fin.cnt == nullptr || a < 0) return;
  atomicAdd(fin.cnt + a, 1);
  if (deg > 0) atomicAdd(fin.deg + a, (int32_t)deg);
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_phase3_lane(GraphView<I> g, const int32_t* tent, const int32_t* aggsize,
                                                        const int32_t* left, const int32_t* left_cnt, int32_t* labels,
                                                        int32_t* err, AggCounts fin) {
  pdl_enter();
  __shared__ __align__(16) int32_t stage[kBlock / 32][kStageWarpWords];
  const int lane = lane_id();
  int32_t* area = stage[threadIdx.x >> 5];
  const int64_t cnt = block_load(left_cnt);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < cnt; base += nw * 32) {
    const int64_t i = base + lane;
    const bool active = i < cnt;
    int32_t v = 0;
    int64_t s = 0, e = 0;
    if (active) {
      v = left[i];
      row_range(g, v, s, e);
    }
    const int len = active ? (int)(e - s < kLaneRowMax ? e - s : kLaneRowMax) : -1;  // leftovers here have <= 32 entries
    int wd;
    const int32_t* myw = stage_rows_warp(g.colind, g.nnz, g.vec, s, len, area, &wd);
    int32_t lab[kLaneRowMax];
#pragma unroll
    for (int j = 0; j < kLaneRowMax; j++) {
      int32_t t = -1;
      if (j < len) {
        const int32_t w = myw[j];
        t = w != v ? tent[w] : -1;
      }
      lab[j] = t;
    }
    int32_t best = -1;
    if (wd == 8) best = phase3_pick<8>(lab, aggsize);
    else if (wd == 16) best = phase3_pick<16>(lab, aggsize);
    else best = phase3_pick<32>(lab, aggsize);
    if (active) {
      labels[v] = best;
      if (best < 0) atomicOr(err, kErrNoAggregatedNeighbour);
    }
    if (fin.cnt != nullptr) {
      // one pair of atomics per aggregate and warp: hub aggregates take
      // many leftovers
      const int32_t key = active ? best : -1;
      const unsigned peers = __match_any_sync(kFull, key);
      const int deg = active ? (int)(e - s) : 0;
      int sum = 0;
#pragma unroll
      for (int src = 0; src < 32; src++) {
        const int x = __shfl_sync(kFull, deg, src);
        if ((peers >> src) & 1u) sum += x;
      }
      if (key >= 0 && lane == __ffs(peers) - 1) {
        atomicAdd(fin.cnt + key, __popc(peers));
        if (sum > 0) atomicAdd(fin.deg + key, sum);
      }
    }
    __syncwarp();
  }
}

// Phase 3, one warp per medium leftover row of up to kP3WarpMax entries:
// count its neighbours' tentative labels in a shared-memory hash table of
// the warp (one insertion per distinct label per step, the count added
// with it), then reduce the best entry by (max coupling, min size, min id).
// Longer rows are passed on to `longer` for the block kernel.
constexpr int kP3WarpMax = 256;
constexpr int kP3WarpSlots = 512;  // at most half full

template <typename I>
__global__ void __launch_bounds__(kBlock) k_phase3_warp(GraphView<I> g, const int32_t* tent, const int32_t* aggsize,
                                                        const int32_t* list, const int32_t* list_cnt, int32_t* labels,
                                                        int32_t* err, AggCounts fin, int32_t* longer,
                                                        int32_t* longer_cnt) {
  pdl_enter();
  __shared__ int32_t keys[kBlock / 32][kP3WarpSlots];
  __shared__ int32_t cnts[kBlock / 32][kP3WarpSlots];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  int32_t* K = keys[wib];
  int32_t* C = cnts[wib];
  const int64_t n_items = block_load(list_cnt);
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_items; it += nw) {
    const int32_t v = list[it];
    int64_t s, e;
    row_range(g, v, s, e);
    if (e - s > kP3WarpMax) {  // warp-uniform
      if (lane == 0) longer[atomicAdd(longer_cnt, 1)] = v;
      continue;
    }
#pragma unroll
    for (int j = lane; j < kP3WarpSlots; j += 32) {
      K[j] = -1;
      C[j] = 0;
    }
    __syncwarp();
    for (int64_t pb = s; pb < e; pb += 32) {  // warp-uniform
      int32_t t = -1;
      if (pb + lane < e) {
        const int32_t w = g.colind[pb + lane];
        t = w != v ? tent[w] : -1;
      }
      const unsigned peers = __match_any_sync(kFull, t);
      if (t >= 0 && lane == __ffs(peers) - 1) {
        uint32_t h = ((uint32_t)t * 2654435761u) >> 23;  // 9 bits
        for (int probe = 0; probe < kP3WarpSlots; probe++) {
          const int32_t old = atomicCAS(K + h, -1, t);
          if (old == -1 || old == t) {
            atomicAdd(C + h, __popc(peers));
            break;
          }
          h = (h + 1) & (kP3WarpSlots - 1);
        }
      }
    }
    __syncwarp();
    int32_t ka[kP3WarpSlots / 32], sz[kP3WarpSlots / 32];
#pragma unroll
    for (int r = 0; r < kP3WarpSlots / 32; r++) {
      ka[r] = K[lane + 32 * r];
      sz[r] = ka[r] >= 0 ? __ldg(aggsize + ka[r]) : 0;
    }
    int32_t la = -1;
    int lc = 0, ls = 0;
#pragma unroll
    for (int r = 0; r < kP3WarpSlots / 32; r++)
      if (ka[r] >= 0 && better(C[lane + 32 * r], sz[r], ka[r], lc, ls, la)) {
        la = ka[r];
        lc = C[lane + 32 * r];
        ls = sz[r];
      }
    const uint32_t mc = __reduce_max_sync(kFull, la >= 0 ? (uint32_t)lc : 0u);
    const uint32_t ms = __reduce_min_sync(kFull, la >= 0 && (uint32_t)lc == mc ? (uint32_t)ls : 0xFFFFFFFFu);
    const uint32_t ma =
        __reduce_min_sync(kFull, la >= 0 && (uint32_t)lc == mc && (uint32_t)ls == ms ? (uint32_t)la : 0xFFFFFFFFu);
    if (lane == 0) {
      const int32_t best = mc > 0 ? (int32_t)ma : -1;
      labels[v] = best;
      fin_add(fin, best, e - s);
      if (best < 0) atomicOr(err, kErrNoAggregatedNeighbour);
    }
    __syncwarp();  // the table is cleared for the next row
  }
}

// Phase 3, one block per medium leftover row: sort its neighbours'
// tentative labels in shared memory, count each run, reduce the best run.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_phase3_sort(GraphView<I> g, const int32_t* tent, const int32_t* aggsize,
                                                        const int32_t* list, const int32_t* list_cnt, int32_t* labels,
                                                        int32_t* err, AggCounts fin) {
  pdl_enter();
  __shared__ int32_t buf[kPhase3SortCap];
  __shared__ uint32_t sh[40];
  __shared__ int fill;
  const int64_t n_items = block_load(list_cnt);
  for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
    const int32_t v = list[it];
    int64_t s, e;
    row_range(g, v, s, e);
    if (threadIdx.x == 0) fill = 0;
    __syncthreads();
    visit_row<kBlock>(g.colind, g.nnz, s, e, threadIdx.x, g.vec, [&](int32_t w) {
      const int32_t t = w != v ? tent[w] : -1;
      if (t >= 0) buf[atomicAdd(&fill, 1)] = t;
    });
    __syncthreads();
    const int cnt = fill;
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int i = cnt + threadIdx.x; i < P; i += blockDim.x) buf[i] = 0x7FFFFFFF;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const int32_t x = buf[i], y = buf[ixj];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              buf[i] = y;
              buf[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    // each run start counts its run; best by (max count, min size, min id)
    int lc = 0, ls = 0;
    int32_t la = -1;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      if (i > 0 && buf[i - 1] == buf[i]) continue;
      const int32_t a = buf[i];
      int lo = i + 1, hi = cnt;  // first index past the run
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (buf[mid] == a) lo = mid + 1;
        else hi = mid;
      }
      const int c = lo - i, sz = aggsize[a];
      if (better(c, sz, a, lc, ls, la)) {
        la = a;
        lc = c;
        ls = sz;
      }
    }
    const uint32_t mc = block_max_u32(la >= 0 ? (uint32_t)lc : 0u, sh);
    const uint32_t ms = block_min_u32(la >= 0 && (uint32_t)lc == mc ? (uint32_t)ls : 0xFFFFFFFFu, sh);
    const uint32_t ma =
        block_min_u32(la >= 0 && (uint32_t)lc == mc && (uint32_t)ls == ms ? (uint32_t)la : 0xFFFFFFFFu, sh);
    if (threadIdx.x == 0) {
      const int32_t best = mc > 0 ? (int32_t)ma : -1;
      labels[v] = best;
      fin_add(fin, best, e - s);
      if (best < 0) atomicOr(err, kErrNoAggregatedNeighbour);
    }
    __syncthreads();
  }
}

// Phase 3 for leftovers of degree > kPhase3SortCap: count coupling in
// shared-memory windows of kPhase3Window aggregate ids.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_phase3_block(GraphView<I> g, const int32_t* tent,
                                                         const int32_t* aggsize, const int32_t* list,
                                                         const int32_t* list_cnt, int32_t* labels, int32_t* err,
                                                         AggCounts fin) {
  pdl_enter();
  __shared__ int cnt[kPhase3Window];
  __shared__ uint32_t sh[40];
  const int64_t n_items = block_load(list_cnt);
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
      fin_add(fin, best, e - s);
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

// Lanes per root row for the claim and qualify kernels: 4 entries per lane
// and pass, so that a row of average length takes one pass.
static int root_lanes(int64_t n, int64_t nnz) {
  const int64_t avg = nnz / std::max<int64_t>(n, 1) + 3;
  return avg <= 16 ? 4 : (avg <= 32 ? 8 : (avg <= 64 ? 16 : 32));
}

template <int G, typename I>
static void launch_claim_g(mis2_ctx* c, const GraphView<I>& gv, const int32_t* list, int64_t n_host,
                           const int32_t* n_dev, int32_t* labels, int32_t base, cudaStream_t st,
                           const int32_t* base_dev, int32_t* heavy_cnt) {
  Scratch& s = c->s;
  const int64_t items = n_dev != nullptr ? gv.n : n_host;
  launch_k(c, k_agg_claim<G, I>, grid_for(c, items, kBlock / G), kBlock, st, gv, list, n_host, n_dev, labels, base,
                                                                        base_dev, s.left_heavy, heavy_cnt,
                                                                        c->cfg.block_degree);
  launch_k(c, k_agg_claim_block<I>, c->sm_count * 2, kBlock, st, gv, list, s.left_heavy, heavy_cnt, labels, base,
                                                           base_dev);
  c->launches += 2;
}

// heavy_cnt: the deferred-row counter, zero on entry (null: the context's,
// cleared here)
template <typename I>
static void launch_claim(mis2_ctx* c, const GraphView<I>& gv, const int32_t* list, int64_t n_host,
                         const int32_t* n_dev, int32_t* labels, int32_t base, cudaStream_t st,
                         const int32_t* base_dev = nullptr, int32_t* heavy_cnt = nullptr) {
  if (heavy_cnt == nullptr) {
    heavy_cnt = c->s.ctr + kCtrHeavy;
    cudaMemsetAsync(heavy_cnt, 0, sizeof(int32_t), st);
  }
  switch (root_lanes(gv.n, gv.nnz)) {
    case 4: launch_claim_g<4, I>(c, gv, list, n_host, n_dev, labels, base, st, base_dev, heavy_cnt); break;
    case 8: launch_claim_g<8, I>(c, gv, list, n_host, n_dev, labels, base, st, base_dev, heavy_cnt); break;
    case 16: launch_claim_g<16, I>(c, gv, list, n_host, n_dev, labels, base, st, base_dev, heavy_cnt); break;
    default: launch_claim_g<32, I>(c, gv, list, n_host, n_dev, labels, base, st, base_dev, heavy_cnt); break;
  }
}

template <typename I>
static void launch_qualify(mis2_ctx* c, const GraphView<I>& gv, const int32_t* list, const int32_t* n_dev,
                           const int32_t* labels, uint8_t* qflag, cudaStream_t st) {
  const int G = root_lanes(gv.n, gv.nnz);
  const int grid = grid_for(c, gv.n, kBlock / G);
  switch (G) {
    case 4: launch_k(c, k_qualify<4, I>, grid, kBlock, st, gv, list, n_dev, labels, qflag); break;
    case 8: launch_k(c, k_qualify<8, I>, grid, kBlock, st, gv, list, n_dev, labels, qflag); break;
    case 16: launch_k(c, k_qualify<16, I>, grid, kBlock, st, gv, list, n_dev, labels, qflag); break;
    default: launch_k(c, k_qualify<32, I>, grid, kBlock, st, gv, list, n_dev, labels, qflag); break;
  }
  c->launches++;
}

// labels_out: where the aggregated vertices' labels are copied (null: they
// are there already); fin: the coarse histogram to start (null: none)
template <typename I>
static void launch_leftovers(mis2_ctx* c, const GraphView<I>& gv, cudaStream_t st, int32_t* labels_out = nullptr,
                             AggCounts fin = AggCounts{}) {
  Scratch& s = c->s;
  launch_k(c, k_aggsize_leftovers<I>, grid_for(c, gv.n, kBlock), kBlock, st, gv, s.tent, s.aggsize, labels_out, fin,
           s.left, s.ctr + kCtrLeft, s.left_mid, s.ctr + kCtrLeftMid, s.left_heavy, s.ctr + kCtrLeftHeavy);
  c->launches++;
}

template <typename I>
static void launch_phase3(mis2_ctx* c, const GraphView<I>& gv, int32_t* labels, cudaStream_t st,
                          AggCounts fin = AggCounts{}) {
  Scratch& s = c->s;
  launch_k(c, k_phase3_lane<I>, grid_for(c, gv.n, kBlock, 8), kBlock, st, gv, s.tent, s.aggsize, s.left,
           s.ctr + kCtrLeft, labels, s.ctr + kCtrErr, fin);
  // medium rows: a warp each up to kP3WarpMax entries, the longer ones
  // (passed on through s.roots2, free by now) a block each
  launch_k(c, k_phase3_warp<I>, grid_for(c, gv.n, kBlock / 32, 4), kBlock, st, gv, s.tent, s.aggsize, s.left_mid,
           s.ctr + kCtrLeftMid, labels, s.ctr + kCtrErr, fin, s.roots2, s.ctr + kCtrLeftLong);
  launch_k(c, k_phase3_sort<I>, c->sm_count * 4, kBlock, st, gv, s.tent, s.aggsize, s.roots2, s.ctr + kCtrLeftLong,
           labels, s.ctr + kCtrErr, fin);
  launch_k(c, k_phase3_block<I>, c->sm_count * 2, kBlock, st, gv, s.tent, s.aggsize, s.left_heavy,
           s.ctr + kCtrLeftHeavy, labels, s.ctr + kCtrErr, fin);
  c->launches += 4;
}

template <typename I>
static int phase1_t(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, int64_t n_roots, int32_t* labels,
                    cudaStream_t st) {
  Scratch& s = c->s;
  const GraphView<I> gv = gview<I>(g);
  MIS2_CUDA(cudaMemsetAsync(labels, 0xFF, g.n * sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrM2, 0, (kCtrErr - kCtrM2 + 1) * sizeof(int32_t), st));
  timer_begin(c, kKcAggregate, st);
  launch_claim<I>(c, gv, roots, n_roots, nullptr, labels, 0, st);
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

// Phase 2 leaves the qualifying phase-2 roots, ascending, in s.qlist.
template <typename I>
static int phase2_t(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, int32_t* labels, int32_t label_base,
                    int32_t* rounds2, int64_t* nq, cudaStream_t st) {
  Scratch& s = c->s;
  const GraphView<I> gv = gview<I>(g);
  const int64_t n = g.n;
  if (c->cfg.loop == MIS2_LOOP_DEVICE)
    MIS2_TRY(mis2_rounds_device(c, g, labels, p, 1, st, rounds2));
  else
    MIS2_TRY(mis2_rounds_host(c, g, labels, p, 1, st, rounds2));
  MIS2_TRY(extract_in_set(c, n, nullptr, s.roots2, s.ctr + kCtrM2, st));
  MIS2_CUDA(cudaMemsetAsync(s.qflag, 0, n, st));
  timer_begin(c, kKcAggregate, st);
  launch_qualify<I>(c, gv, s.roots2, s.ctr + kCtrM2, labels, s.qflag, st);
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  MIS2_TRY(compact_flags(c, s.qflag, nullptr, n, s.qlist, s.ctr + kCtrQual, st));
  timer_begin(c, kKcAggregate, st);
  launch_claim<I>(c, gv, s.qlist, 0, s.ctr + kCtrQual, labels, label_base, st);
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  *nq = c->h_ctr[kCtrQual];
  return MIS2_OK;
}

template <typename I>
static int phase3_t(mis2_ctx* c, const GraphArgs& g, int32_t* labels, int64_t total, cudaStream_t st) {
  Scratch& s = c->s;
  const GraphView<I> gv = gview<I>(g);
  const int64_t n = g.n;
  timer_begin(c, kKcAggregate, st);
  MIS2_CUDA(cudaMemcpyAsync(s.tent, labels, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  MIS2_CUDA(cudaMemsetAsync(s.aggsize, 0, std::max<int64_t>(total, 1) * sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrLeft, 0, 2 * sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrLeftMid, 0, sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrLeftLong, 0, sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrErr, 0, sizeof(int32_t), st));
  launch_leftovers<I>(c, gv, st);
  launch_phase3<I>(c, gv, labels, st);
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  if (c->h_ctr[kCtrErr] & kErrNoAggregatedNeighbour) return MIS2_ERR_BAD_GRAPH;
  return MIS2_OK;
}

int agg_phase1(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, int64_t n_roots, int32_t* labels,
               cudaStream_t st) {
  return g.rp64 ? phase1_t<int64_t>(c, g, roots, n_roots, labels, st)
                : phase1_t<int32_t>(c, g, roots, n_roots, labels, st);
}

int agg_phase2(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, int32_t* labels, int32_t label_base,
               int32_t* rounds2, int64_t* nq, cudaStream_t st) {
  return g.rp64 ? phase2_t<int64_t>(c, g, p, labels, label_base, rounds2, nq, st)
                : phase2_t<int32_t>(c, g, p, labels, label_base, rounds2, nq, st);
}

int agg_phase3(mis2_ctx* c, const GraphArgs& g, int32_t* labels, int64_t total, cudaStream_t st) {
  return g.rp64 ? phase3_t<int64_t>(c, g, labels, total, st) : phase3_t<int32_t>(c, g, labels, total, st);
}

// The level's aggregation without host synchronisation.  The counter words
// it uses were cleared at the level's start, and the level's root
// compaction has set s.tent to -1 and s.aggsize, s.agg_cnt and s.ub to 0.
// Phases 1 and 2 label into s.tent, the frozen labels phase 3 reads; the
// fused sizes / leftovers pass copies every aggregated vertex's label to
// `labels`, and phase 3 adds the leftovers' (no device-to-device copy of the
// labels).  The coarse graph's histogram (s.agg_cnt, s.ub) is accumulated on
// the way.
template <typename I>
static int agg_async_t(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, const PrioCfg& p, int mode,
                       int32_t* labels, cudaStream_t st) {
  Scratch& s = c->s;
  const GraphView<I> gv = gview<I>(g);
  const int64_t n = g.n;
  int32_t* tent = s.tent;
  timer_begin(c, kKcAggregate, st);
  launch_claim<I>(c, gv, roots, 0, s.ctr + kCtrRoots, tent, 0, st, nullptr, s.ctr + kCtrHeavy);
  timer_end(c, st);
  if (mode == MIS2_AGG_ALG3) {
    MIS2_TRY(mis2_rounds_device_async(c, g, tent, p, 1, kCtrRounds2, st));
    // qflag = 1 at the phase-2 roots, 0 elsewhere; k_qualify clears the
    // roots that do not qualify
    MIS2_TRY(extract_in_set(c, n, s.qflag, s.roots2, s.ctr + kCtrM2, st));
    timer_begin(c, kKcAggregate, st);
    launch_qualify<I>(c, gv, s.roots2, s.ctr + kCtrM2, tent, s.qflag, st);
    timer_end(c, st);
    MIS2_TRY(compact_flags(c, s.qflag, nullptr, n, s.qlist, s.ctr + kCtrQual, st));
    timer_begin(c, kKcAggregate, st);
    launch_claim<I>(c, gv, s.qlist, 0, s.ctr + kCtrQual, tent, 0, st, s.ctr + kCtrRoots, s.ctr + kCtrHeavy2);
    timer_end(c, st);
  }
  timer_begin(c, kKcAggregate, st);
  const AggCounts fin{s.agg_cnt, s.ub};
  launch_leftovers<I>(c, gv, st, labels, fin);
  launch_phase3<I>(c, gv, labels, st, fin);
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

int agg_level_async(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, const PrioCfg& p, int mode, int32_t* labels,
                    cudaStream_t st) {
  return g.rp64 ? agg_async_t<int64_t>(c, g, roots, p, mode, labels, st)
                : agg_async_t<int32_t>(c, g, roots, p, mode, labels, st);
}

int aggregate_impl(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, int64_t n_roots, uint64_t seed, int mode,
                   int32_t* labels, int64_t* n_aggs, cudaStream_t st) {
  c->stats.rounds2 = 0;
  memset(c->stats.trace2, 0, sizeof(c->stats.trace2));
  if (g.n == 0) {
    *n_aggs = 0;
    return MIS2_OK;
  }
  MIS2_TRY(agg_phase1(c, g, roots, n_roots, labels, st));
  int64_t nq = 0;
  if (mode == MIS2_AGG_ALG3) {
    int32_t r2 = 0;
    MIS2_TRY(agg_phase2(c, g, make_prio(c, g.n, seed), labels, (int32_t)n_roots, &r2, &nq, st));
    c->stats.rounds2 = r2;
  }
  MIS2_TRY(agg_phase3(c, g, labels, n_roots + nq, st));
  *n_aggs = n_roots + nq;
  return MIS2_OK;
}

}  // namespace mis2
