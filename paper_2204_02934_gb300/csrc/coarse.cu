// coarse.cu -- coarse graph A_c of an aggregation (Section III-C, setup of
// Algorithm 4: one coarse vertex per aggregate, coarse edge A-B whenever a
// fine edge joins a member of A to a member of B, A != B).
//
// No global sort: vertices are bucketed by aggregate (counting sort), then
// each aggregate's neighbour labels are de-duplicated on chip.
//   - Aggregates whose members hold <= kWarpEntries entries and have at
//     most kDistinctCap coarse neighbours: one warp with a shared-memory hash
//     set; the distinct labels are sorted on chip.
//   - Everything else: a global bitmap over all aggregate ids per aggregate,
//     filled by the whole grid 32 members at a time, then read out in order
//     by one block (k_large_or / k_large_emit).
// Member rows of <= 32 entries are staged in shared memory by the warp (one
// coalesced copy per row) and read lane-per-row; longer rows are walked by
// the whole warp.
// Rows land in a scratch buffer at the aggregate's degree-sum offset, then
// are packed behind the prefix sum of the row lengths.
#include <algorithm>

#include "internal.h"
#include "mis_rows.cuh"
#include "scan.cuh"

namespace mis2 {

constexpr int kCoarseWarps = 4;        // warps per block of the warp-per-aggregate kernel
constexpr int kSortCap = 1024;         // entries per warp
constexpr int kWarpEntries = 8192;     // larger aggregates go to the block kernel

template <typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_hist(GraphView<I> g, const int32_t* labels, int32_t* agg_cnt,
                                                        int32_t* ub) {
  pdl_enter();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = lane_id();
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < g.n; base += stride) {
    const int64_t v = base + lane;
    const int32_t a = v < g.n ? labels[v] : -1;
    const unsigned peers = __match_any_sync(kFull, a);
    int deg = 0;
    if (a >= 0) {
      int64_t s, e;
      row_range(g, v, s, e);
      deg = (int)(e - s);
    }
    // sum of the degrees of the lanes holding the same label (one atomic per
    // label per warp: an aggregate can hold millions of vertices)
    int sum = 0;
#pragma unroll
    for (int src = 0; src < 32; src++) {
      const int x = __shfl_sync(kFull, deg, src);
      if ((peers >> src) & 1u) sum += x;
    }
    if (a >= 0 && lane == __ffs(peers) - 1) {
      atomicAdd(agg_cnt + a, __popc(peers));
      if (sum > 0) atomicAdd(ub + a, sum);
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_coarse_scatter(int64_t n, const int32_t* labels, int32_t* cursor,
                                                           int32_t* members) {
  pdl_enter();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = lane_id();
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < n; base += stride) {
    const int64_t v = base + lane;
    const int32_t a = v < n ? labels[v] : -1;
    const unsigned peers = __match_any_sync(kFull, a);
    const int leader = __ffs(peers) - 1;
    int pos = 0;
    if (a >= 0 && lane == leader) pos = atomicAdd(cursor + a, __popc(peers));
    pos = __shfl_sync(peers, pos, leader);
    if (a >= 0) members[pos + __popc(peers & ((1u << lane) - 1u))] = (int32_t)v;
  }
}

// Labels of a staged row (W unrolled gathers, len <= W): -1 where absent or
// equal to a.
template <int W, typename FB>
__device__ __forceinline__ void staged_labels(const int32_t* labels, const int32_t* row, int len, int32_t a,
                                              FB&& fb) {
  int32_t lab[W];
#pragma unroll
  for (int j = 0; j < W; j++) {
    const int32_t l = j < len ? labels[row[j]] : a;
    lab[j] = l != a ? l : -1;
  }
  fb(lab);
}

// Walk every fine entry of aggregate a (members [mb, me)) with one warp.
// fb(lab) receives a register array of neighbour labels, -1 where the entry
// is absent or belongs to a itself; every lane calls it with its own array
// (32 entries for a staged member row, 4 per step of a long row), so a
// callback can issue all its memory operations before waiting on any.
// Member rows longer than kGiantRow found while walking a large aggregate
// are handed to this list instead (vertex, bitmap slot) and walked later in
// pieces by the whole grid.
struct GiantList {
  int32_t* v;
  int32_t* slot;
  int32_t* cnt;
  int32_t cur_slot;
};

// CONVERGED: every lane calls fb for every batch of 32 members, with one
// 32-entry array (lanes without a staged row get all -1), so fb may use
// warp-wide primitives; otherwise only lanes with a staged row call it, with
// the narrowest of 8, 16 or 32 entries that bounds the batch's rows.
template <typename I, bool CONVERGED = false, typename FB>
__device__ __forceinline__ void walk_aggregate(const GraphView<I>& g, const int32_t* labels, const int32_t* members,
                                               int64_t mb, int64_t me, int32_t a, int32_t* stage_warp, FB&& fb,
                                               const GiantList* giant = nullptr) {
  const int lane = lane_id();
  for (int64_t kb = mb; kb < me; kb += 32) {
    const int64_t k = kb + lane;
    int64_t s = 0, e = 0;
    const bool has = k < me;
    if (has) row_range(g, members[k], s, e);
    const int len = has && e - s <= kLaneRowMax ? (int)(e - s) : -1;
    int wd;
    const int32_t* mine = stage_rows_warp(g.colind, g.nnz, g.vec, s, len, stage_warp, &wd);
    if constexpr (CONVERGED) {
      staged_labels<32>(labels, mine, len, a, fb);
    } else if (len > 0) {
      if (wd == 8) staged_labels<8>(labels, mine, len, a, fb);
      else if (wd == 16) staged_labels<16>(labels, mine, len, a, fb);
      else staged_labels<32>(labels, mine, len, a, fb);
    }
    __syncwarp();
    if (giant != nullptr) {
      const bool gi = has && e - s > kGiantRow;
      const unsigned gm = __ballot_sync(kFull, gi);
      if (gm) {
        int base = 0;
        if (lane == __ffs(gm) - 1) base = atomicAdd(giant->cnt, __popc(gm));
        base = __shfl_sync(kFull, base, __ffs(gm) - 1);
        if (gi) {
          const int idx = base + __popc(gm & ((1u << lane) - 1u));
          giant->v[idx] = members[k];
          giant->slot[idx] = giant->cur_slot;
        }
      }
    }
    unsigned longm = __ballot_sync(kFull, has && len < 0 && (giant == nullptr || e - s <= kGiantRow));
    while (longm) {
      const int j = __ffs(longm) - 1;
      longm &= longm - 1;
      const int64_t sj = __shfl_sync(kFull, s, j), ej = __shfl_sync(kFull, e, j);
      // warp-uniform trip count (every lane calls fb the same number of
      // times); lanes past the row's end see only -1 labels
      for (int64_t pb = sj & ~int64_t(3); pb < ej; pb += 128) {
        const int64_t p = pb + 4 * lane;
        int32_t w4[4];
        if (p < ej && g.vec && p + 4 <= g.nnz) {
          const int4 q = __ldg(reinterpret_cast<const int4*>(g.colind + p));
          w4[0] = q.x, w4[1] = q.y, w4[2] = q.z, w4[3] = q.w;
        } else {
#pragma unroll
          for (int t = 0; t < 4; t++) w4[t] = (p + t >= sj && p + t < ej) ? g.colind[p + t] : 0;
        }
        int32_t lab[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const int32_t l = (p + t >= sj && p + t < ej) ? labels[w4[t]] : a;
          lab[t] = l != a ? l : -1;
        }
        fb(lab);
      }
    }
  }
}

// Small aggregates (at most kSmallMembers members and kSmallEntries fine
// entries) are handled several at a time by one warp, without a hash set:
// a warp takes kSmallWindow consecutive aggregate ids, groups its small
// aggregates into
// sub-batches of at most 32 members and 256 entries, loads every entry of a
// sub-batch at once (8 per lane), forms keys (local aggregate << 27 | label)
// for labels of other aggregates, sorts the 256 keys in registers (bitonic),
// and writes each aggregate's distinct labels in ascending order.  The keys
// need n_aggs < 2^27; larger aggregations take the hash path throughout.
constexpr int kSmallMembers = 32;
constexpr int kSmallK = 8;  // keys per lane
constexpr int kSmallEntries = 32 * kSmallK;
constexpr int kSmallLabelBits = 27;
constexpr int kSmallWindow = 8;  // aggregate ids per warp task

__device__ __forceinline__ bool small_aggregate(int32_t members, int32_t ub, bool enabled) {
  return enabled && members <= kSmallMembers && ub <= kSmallEntries;
}

__device__ __forceinline__ int warp_inclusive_sum(int x) {
  const int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Ascending bitonic sort of 32 * K keys held lane-major (key index =
// lane * K + r), in registers and shuffles.
template <int K>
__device__ __forceinline__ void warp_sort_keys(uint32_t (&k)[K]) {
  const int lane = lane_id();
#pragma unroll
  for (int size = 2; size <= 32 * K; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride < K) {
#pragma unroll
        for (int r = 0; r < K; r++) {
          const int q = r ^ stride;
          if (q > r) {
            const bool up = (((lane * K + r) & size) == 0);
            const uint32_t x = k[r], y = k[q];
            const bool sw = (x > y) == up;
            k[r] = sw ? y : x;
            k[q] = sw ? x : y;
          }
        }
      } else {
        const int lx = stride / K;
        const bool lower = (lane & lx) == 0;
#pragma unroll
        for (int r = 0; r < K; r++) {
          const uint32_t o = __shfl_xor_sync(kFull, k[r], lx);
          const bool up = (((lane * K + r) & size) == 0);
          k[r] = (lower == up) ? min(k[r], o) : max(k[r], o);
        }
      }
    }
  }
}

// rest / rest_cnt: the aggregates with fine entries that are not small are
// listed there (one reservation per warp and window), so that the kernel
// for the others visits those alone.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_small(GraphView<I> g, const int32_t* labels, int64_t n_aggs,
                                                         const int32_t* agg_ptr, const int32_t* members,
                                                         const int32_t* ub, const int32_t* ub_ptr, int32_t* tmp,
                                                         int32_t* c_cnt, int32_t* rest, int32_t* rest_cnt) {
  pdl_enter();
  __shared__ int32_t sh_cnt[kBlock / 32][32];
  __shared__ int32_t sh_sel[kBlock / 32][32];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  int32_t* cnt = sh_cnt[wib];  // distinct labels per local aggregate
  int32_t* sel = sh_sel[wib];  // local aggregate -> lane of its id in the window
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t A = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kSmallWindow; A < n_aggs;
       A += nw * kSmallWindow) {
    const int64_t a = A + lane;
    const bool in = lane < kSmallWindow && a < n_aggs;
    const int32_t p0 = in ? agg_ptr[a] : 0;
    const int32_t p1 = in ? agg_ptr[a + 1] : 0;
    const int32_t u = in ? ub[a] : 0;
    // an aggregate without fine entries (an isolated vertex) has an empty row
    if (in && u == 0) c_cnt[a] = 0;
    const bool sm = in && u > 0 && small_aggregate(p1 - p0, u, true);
    warp_append(in && u > 0 && !sm, (int32_t)a, rest, rest_cnt);
    const int32_t outb = sm ? ub_ptr[a] : 0;
    const int m = sm ? p1 - p0 : 0;
    const int um = sm ? u : 0;
    const int cm = warp_inclusive_sum(m);
    const int cu = warp_inclusive_sum(um);
    unsigned smask = __ballot_sync(kFull, sm);
    while (smask) {
      // sub-batch: the remaining small lanes in order while the members stay
      // <= 32 and the entries <= 256 (the first one always fits)
      const int i0 = __ffs(smask) - 1;
      const int bm0 = __shfl_sync(kFull, cm - m, i0);
      const int bu0 = __shfl_sync(kFull, cu - um, i0);
      const unsigned bm = __ballot_sync(kFull, ((smask >> lane) & 1u) && cm - bm0 <= kSmallMembers &&
                                                   cu - bu0 <= kSmallEntries);
      smask &= ~bm;
      const bool mine = (bm >> lane) & 1u;
      const int slot0 = cm - m - bm0;  // first member slot of this lane's aggregate
      if (mine) {
        const int li = __popc(bm & ((1u << lane) - 1u));
        sel[li] = lane;
        cnt[li] = 0;
      }
      const unsigned starts = __reduce_or_sync(kFull, mine ? 1u << slot0 : 0u);
      const int M = __shfl_sync(kFull, cm, 31 - __clz(bm)) - bm0;
      __syncwarp();
      // member slot `lane`: its local aggregate, owner lane, vertex, row
      const int loc = lane < M ? __popc(starts & ((2u << lane) - 1u)) - 1 : 0;
      const int owner = sel[loc];
      const int32_t own_p0 = __shfl_sync(kFull, p0, owner);
      const int own_slot0 = __shfl_sync(kFull, slot0, owner);
      int64_t s = 0, e = 0;
      if (lane < M) row_range(g, members[own_p0 + (lane - own_slot0)], s, e);
      const int d = (int)(e - s);
      const int offi = warp_inclusive_sum(d);
      const int E = __shfl_sync(kFull, offi, 31);
      const int offx = offi - d;
      // entry t = r * 32 + lane: its member (last slot with offx <= t), column, label
      int32_t w[kSmallK];
      int lj[kSmallK];
#pragma unroll
      for (int r = 0; r < kSmallK; r++) {
        const int t = r * 32 + lane;
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int c = lo + step;
          const int oc = __shfl_sync(kFull, offx, c & 31);
          if (c < M && oc <= t) lo = c;
        }
        const int64_t sj = __shfl_sync(kFull, s, lo);
        const int oj = __shfl_sync(kFull, offx, lo);
        lj[r] = __shfl_sync(kFull, loc, lo);
        w[r] = t < E ? g.colind[sj + (t - oj)] : -1;
      }
      uint32_t key[kSmallK];
#pragma unroll
      for (int r = 0; r < kSmallK; r++) {
        const int32_t l = w[r] >= 0 ? labels[w[r]] : -1;
        const int32_t own = (int32_t)A + sel[lj[r]];
        key[r] = (l >= 0 && l != own) ? ((uint32_t)lj[r] << kSmallLabelBits) | (uint32_t)l : 0xFFFFFFFFu;
      }
      warp_sort_keys<kSmallK>(key);
      // distinct keys in order: their index among all distinct keys
      uint32_t prev = __shfl_up_sync(kFull, key[kSmallK - 1], 1);
      if (lane == 0) prev = 0xFFFFFFFFu;
      bool uq[kSmallK];
      int nu = 0;
#pragma unroll
      for (int r = 0; r < kSmallK; r++) {
        uq[r] = key[r] != 0xFFFFFFFFu && key[r] != (r == 0 ? prev : key[r - 1]);
        nu += uq[r] ? 1 : 0;
        if (uq[r]) atomicAdd(cnt + (key[r] >> kSmallLabelBits), 1);
      }
      const int ubase = warp_inclusive_sum(nu) - nu;
      __syncwarp();
      const int nb = __popc(bm);
      const int cl = lane < nb ? cnt[lane] : 0;
      const int first_u = warp_inclusive_sum(cl) - cl;  // first distinct index of local aggregate `lane`
      const int out_l = __shfl_sync(kFull, outb, lane < nb ? sel[lane] : 0);  // ub_ptr of local aggregate `lane`
      if (lane < nb) c_cnt[A + sel[lane]] = cl;
      int ui = ubase;
#pragma unroll
      for (int r = 0; r < kSmallK; r++) {
        const int l = uq[r] ? (int)(key[r] >> kSmallLabelBits) : 0;
        const int fu = __shfl_sync(kFull, first_u, l);
        const int ob = __shfl_sync(kFull, out_l, l);
        if (uq[r]) tmp[ob + (ui - fu)] = (int32_t)(key[r] & ((1u << kSmallLabelBits) - 1u));
        ui += uq[r] ? 1 : 0;
      }
      __syncwarp();
    }
  }
}

// Aggregates of mesh-like graphs (tens of members, each row touching a
// handful of other aggregates) in two steps.  k_coarse_cand: for every
// vertex in index order (a lane per vertex, 32 consecutive rows staged by the
// warp), the labels among its neighbours other than its own, at most
// kCand of them (-1 = unused slot), each label written unless it equals one
// of the last four written (a row meets its few neighbour aggregates in
// runs, so the list stays short; a repeat that slips through is harmless,
// the merge removes it).  A vertex needing more slots, or with a row longer
// than 32 entries, gets slot 0 = -2.
constexpr int kCand = 12;  // candidate slots per vertex: three int4
constexpr int kMergeRowCap = 1024;  // overflowing member rows the merge walks itself

template <typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_cand(GraphView<I> g, const int32_t* labels, int4* cand) {
  pdl_enter();
  __shared__ __align__(16) int32_t stage[kBlock / 32][kStageWarpWords];
  __shared__ int32_t outs[kBlock / 32][32 * (kCand + 1)];
  const int lane = lane_id();
  int32_t* area = stage[threadIdx.x >> 5];
  int32_t* my = outs[threadIdx.x >> 5] + lane * (kCand + 1);
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < g.n; base += nw * 32) {
    const int64_t v = base + lane;
    const bool has = v < g.n;
    int64_t s = 0, e = 0;
    int32_t a = -1;
    if (has) {
      row_range(g, v, s, e);
      a = labels[v];
    }
    const int len = has && e - s <= kLaneRowMax ? (int)(e - s) : -1;
    const int32_t* mine = stage_rows_warp(g.colind, g.nnz, g.vec, s, len, area);
    int32_t lab[kLaneRowMax];
#pragma unroll
    for (int k = 0; k < kLaneRowMax; k++) lab[k] = k < len ? labels[mine[k]] : a;
    int32_t w0 = -1, w1 = -1, w2 = -1, w3 = -1;  // the last four labels written
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kLaneRowMax; k++) {
      const int32_t l = lab[k];
      if (l != a && l != w0 && l != w1 && l != w2 && l != w3) {
        if (cnt < kCand) my[cnt] = l;
        cnt++;
        w3 = w2;
        w2 = w1;
        w1 = w0;
        w0 = l;
      }
    }
    if (has) {
      int32_t o[kCand];
#pragma unroll
      for (int k = 0; k < kCand; k++) o[k] = k < cnt ? my[k] : -1;
      if (cnt > kCand || len < 0) o[0] = -2;
#pragma unroll
      for (int q = 0; q < kCand / 4; q++)
        cand[(kCand / 4) * v + q] = make_int4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
    __syncwarp();  // the staged rows are rewritten by the next batch
  }
}

// k_coarse_merge: a warp per aggregate, a member per lane (two passes for up
// to 64 members).  The members' labels from k_coarse_cand go into a
// shared-memory hash set, one insertion per distinct label per step (lanes
// holding equal labels are matched first); the set, at most 32 labels, is
// then sorted across the lanes and written in ascending order.  A member
// flagged by k_coarse_cand (more labels than its slots, or a row longer than
// 32) has its row walked by the warp instead, a lane per entry.  Aggregates
// with more members, a flagged member row longer than kMergeRowCap or more
// than 32 distinct labels go to `rest` (the general hash-set kernel); small
// aggregates are k_coarse_small's.
constexpr int kMergeSlots = 128;
constexpr int kMergeMembers = 64;

// One insertion per distinct label l >= 0 among the lanes into the warp's
// set tab (kMergeSlots slots, linear probing), counting new labels in *cnt.
// Every lane of the warp calls it.
__device__ __forceinline__ void merge_insert(int32_t l, int32_t* tab, int32_t* cnt, int lane) {
  const unsigned peers = __match_any_sync(kFull, l);
  if (l >= 0 && lane == __ffs(peers) - 1) {
    uint32_t h = ((uint32_t)l * 2654435761u) >> 25;
    for (int probe = 0; probe < kMergeSlots; probe++) {
      const int32_t old = atomicCAS(tab + h, -1, l);
      if (old == -1) {
        atomicAdd(cnt, 1);
        break;
      }
      if (old == l) break;
      h = (h + 1) & (kMergeSlots - 1);
    }
  }
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_merge(GraphView<I> g, const int32_t* labels, int64_t n_aggs,
                                                         const int32_t* agg_ptr, const int32_t* members,
                                                         const int32_t* ub, const int32_t* ub_ptr, const int4* cand,
                                                         int32_t* tmp, int32_t* c_cnt, int32_t* rest,
                                                         int32_t* rest_cnt, bool small_on) {
  pdl_enter();
  __shared__ int32_t tabs[kBlock / 32][kMergeSlots];
  __shared__ int32_t dcnt[kBlock / 32];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  int32_t* tab = tabs[wib];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n_aggs; a += nw) {
    const int32_t p0 = agg_ptr[a], M = agg_ptr[a + 1] - p0;
    const int32_t ua = ub[a];
    if (small_aggregate(M, ua, small_on)) continue;  // k_coarse_small's
    if (ua == 0) {  // no fine entries: an empty row
      if (lane == 0) c_cnt[a] = 0;
      continue;
    }
    if (M > kMergeMembers) {
      if (lane == 0) rest[atomicAdd(rest_cnt, 1)] = (int32_t)a;
      continue;
    }
#pragma unroll
    for (int j = lane; j < kMergeSlots; j += 32) tab[j] = -1;
    if (lane == 0) dcnt[wib] = 0;
    __syncwarp();
    bool bad = false;
    for (int m0 = 0; m0 < M; m0 += 32) {  // warp-uniform
      int32_t cs[kCand];
#pragma unroll
      for (int t = 0; t < kCand; t++) cs[t] = -1;
      if (m0 + lane < M) {
        const int64_t u = members[p0 + m0 + lane];
#pragma unroll
        for (int q = 0; q < kCand / 4; q++) {
          const int4 c = cand[(kCand / 4) * u + q];
          cs[4 * q] = c.x;
          cs[4 * q + 1] = c.y;
          cs[4 * q + 2] = c.z;
          cs[4 * q + 3] = c.w;
        }
      }
      // as many steps as the longest list of the warp (lists fill from slot 0)
      int mine = 0;
#pragma unroll
      for (int t = 0; t < kCand; t++) mine += cs[t] >= 0 ? 1 : 0;
      const int steps = (int)__reduce_max_sync(kFull, (unsigned)mine);
#pragma unroll
      for (int t = 0; t < kCand; t++) {
        if (t >= steps) break;  // warp-uniform
        merge_insert(cs[t] >= 0 ? cs[t] : -1, tab, dcnt + wib, lane);
      }
      // members whose list overflowed (or whose row is longer than 32):
      // their rows are walked here, one member at a time, a lane per entry
      unsigned over = __ballot_sync(kFull, cs[0] == -2);
      while (over != 0u) {  // warp-uniform
        const int src = __ffs(over) - 1;
        over &= over - 1u;
        const int64_t u = members[p0 + m0 + src];
        int64_t rs, re;
        row_range(g, u, rs, re);
        if (re - rs > kMergeRowCap) {
          bad = true;
          continue;
        }
        for (int64_t pb = rs; pb < re; pb += 32) {  // warp-uniform
          int32_t l = -1;
          if (pb + lane < re) {
            l = labels[g.colind[pb + lane]];
            if (l == (int32_t)a) l = -1;
          }
          merge_insert(l, tab, dcnt + wib, lane);
        }
      }
    }
    __syncwarp();
    const int nd = dcnt[wib];
    if (__any_sync(kFull, bad) || nd > 32) {
      if (lane == 0) rest[atomicAdd(rest_cnt, 1)] = (int32_t)a;
      __syncwarp();
      continue;
    }
    // the set's labels, one per lane, then a bitonic sort across the lanes
    int32_t v[kMergeSlots / 32];
    int nv = 0;
#pragma unroll
    for (int r = 0; r < kMergeSlots / 32; r++) {
      v[r] = tab[lane * (kMergeSlots / 32) + r];
      nv += v[r] >= 0 ? 1 : 0;
    }
    int pos = nv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, pos, o);
      if (lane >= o) pos += y;
    }
    pos -= nv;
    __syncwarp();  // every lane has read its slots
#pragma unroll
    for (int r = 0; r < kMergeSlots / 32; r++)
      if (v[r] >= 0) tab[pos++] = v[r];
    __syncwarp();
    int32_t x = lane < nd ? tab[lane] : 0x7FFFFFFF;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const int32_t o = __shfl_xor_sync(kFull, x, stride);
        const bool up = (lane & size) == 0, lower = (lane & stride) == 0;
        x = (lower == up) ? min(x, o) : max(x, o);
      }
    }
    if (lane < nd) tmp[ub_ptr[a] + lane] = x;
    if (lane == 0) c_cnt[a] = nd;
    __syncwarp();
  }
}

// Warp per aggregate: insert every neighbour label into a shared-memory hash
// set (256 slots, linear probing); first insertions form the distinct list,
// which is then sorted (bitonic, a few dozen entries) and written out.  An
// aggregate with more than kDistinctCap distinct labels goes to the large
// path instead.
constexpr int kHashSlots = 256;
constexpr int kDistinctCap = 192;
static_assert(kHashSlots + 256 <= kSortCap, "hash table and distinct list share the warp buffer");

__device__ __forceinline__ uint32_t label_hash(int32_t l) { return ((uint32_t)l * 2654435761u) >> 24; }

// With `list` (the aggregates k_coarse_merge left over, *list_cnt of them)
// only those; otherwise every aggregate that is not k_coarse_small's.
template <typename I>
__global__ void __launch_bounds__(kCoarseWarps * 32) k_coarse_rows(
    GraphView<I> g, const int32_t* labels, int64_t n_aggs, const int32_t* agg_ptr, const int32_t* members,
    const int32_t* ub, const int32_t* ub_ptr, int32_t* tmp, int32_t* c_cnt, int32_t* large, int32_t* large_cnt,
    bool small_on, const int32_t* list, const int32_t* list_cnt) {
  pdl_enter();
  __shared__ int32_t sbuf[kCoarseWarps][kSortCap];
  __shared__ __align__(16) int32_t stage[kCoarseWarps][kStageWarpWords];
  __shared__ int32_t scnt[kCoarseWarps];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  int32_t* tab = sbuf[wib];
  int32_t* dl = sbuf[wib] + kHashSlots;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t items = list != nullptr ? (int64_t)block_load(list_cnt) : n_aggs;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < items; i += nw) {
    const int64_t a = list != nullptr ? (int64_t)list[i] : i;
    const int32_t ua = ub[a];
    if (list == nullptr && small_aggregate(agg_ptr[a + 1] - agg_ptr[a], ua, small_on)) continue;  // k_coarse_small's
    if (ua > kWarpEntries) {
      if (lane == 0) large[atomicAdd(large_cnt, 1)] = (int32_t)a;
      continue;
    }
    for (int j = lane; j < kHashSlots; j += 32) tab[j] = -1;
    if (lane == 0) scnt[wib] = 0;
    __syncwarp();
    const int64_t mb = agg_ptr[a], me = agg_ptr[a + 1];
    bool full = false;
    walk_aggregate<I, true>(g, labels, members, mb, me, (int32_t)a, stage[wib], [&](auto& lab) {
      int32_t prev = -1;
#pragma unroll
      for (int j = 0; j < (int)(sizeof(lab) / sizeof(lab[0])); j++) {
        int32_t l = lab[j];
        // past the distinct cap the aggregate goes to the bitmap path: a lane
        // stops inserting once its own insertion found the cap reached, so
        // the table holds at most kDistinctCap + 32 labels and probing ends
        if (l == prev || full) l = -1;
        else if (l >= 0) prev = l;
        // one insertion per distinct label among the lanes (lanes walking
        // neighbouring members mostly meet the same labels at once, and
        // compare-and-swaps on one slot serialise)
        const unsigned peers = __match_any_sync(kFull, l);
        if (l < 0 || lane != __ffs(peers) - 1) continue;
        uint32_t h = label_hash(l);
        for (int probe = 0; probe < kHashSlots; probe++) {
          const int32_t old = atomicCAS(tab + h, -1, l);
          if (old == -1) {
            const int p = atomicAdd(scnt + wib, 1);
            if (p < kDistinctCap) dl[p] = l;
            else full = true;
            break;
          }
          if (old == l) break;
          h = (h + 1) & (kHashSlots - 1);
        }
      }
    });
    __syncwarp();
    const int D = scnt[wib];
    if (D > kDistinctCap) {
      if (lane == 0) large[atomicAdd(large_cnt, 1)] = (int32_t)a;
      __syncwarp();
      continue;
    }
    int P = 32;
    while (P < D) P <<= 1;
    for (int i = D + lane; i < P; i += 32) dl[i] = 0x7FFFFFFF;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < P; i += 32) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const int32_t x = dl[i], y = dl[ixj];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              dl[i] = y;
              dl[ixj] = x;
            }
          }
        }
        __syncwarp();
      }
    }
    const int64_t out = ub_ptr[a];
    for (int i = lane; i < D; i += 32) tmp[out + i] = dl[i];
    if (lane == 0) c_cnt[a] = D;
    __syncwarp();
  }
}

// Large aggregates go through global bitmaps in batches of up to `slots`
// aggregates: every warp of the grid ORs the labels of 32 members at a time
// into its aggregate's bitmap (fire-and-forget atomics, so an aggregate of a
// million members is spread over the whole GPU), then one block per
// aggregate reads its bitmap out in order and clears it.

// chunk_off[i] = number of 32-member chunks of the batch's aggregates < i.
// With n_large_dev set (single-batch path), the batch is the first
// min(kb, n_large) large aggregates, that count goes to *kb_out, and a larger
// n_large raises kErrLargeOverflow.
// One block (kBlock threads) scans the batch in tiles.  It also clears the
// batch's giant-row list.
__global__ void __launch_bounds__(kBlock) k_large_chunks(const int32_t* large, int32_t k0, int32_t kb,
                                                         const int32_t* agg_ptr, int64_t* chunk_off,
                                                         const int32_t* n_large_dev, int32_t* kb_out, int32_t* err,
                                                         int32_t* giant_cnt) {
  pdl_enter();
  __shared__ int sh[40];
  __shared__ int32_t skb;
  if (threadIdx.x == 0) {
    int32_t b = kb;
    if (n_large_dev != nullptr) {
      const int32_t nl = *n_large_dev;
      if (nl > kb) atomicOr(err, kErrLargeOverflow);
      b = min(kb, nl);
      *kb_out = b;
    }
    skb = b;
    *giant_cnt = 0;
  }
  __syncthreads();
  kb = skb;
  int64_t acc = 0;
  for (int t0 = 0; t0 < kb; t0 += kBlock) {
    const int i = t0 + threadIdx.x;
    int c = 0;
    if (i < kb) {
      const int32_t a = large[k0 + i];
      c = (agg_ptr[a + 1] - agg_ptr[a] + 31) / 32;
    }
    int tile_total;
    const int x = block_exclusive_scan(c, sh, &tile_total);
    if (i < kb) chunk_off[i] = acc + x;
    acc += tile_total;
  }
  if (threadIdx.x == 0) chunk_off[kb] = acc;
}

// Piece offsets of the giant rows (kGiantRow entries per piece), one block.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_giant_pieces(GraphView<I> g, const int32_t* giant_v,
                                                         const int32_t* giant_cnt, int64_t* giant_off) {
  pdl_enter();
  __shared__ int sh[40];
  const int32_t ng = block_load(giant_cnt);
  int64_t acc = 0;
  for (int t0 = 0; t0 < ng; t0 += kBlock) {
    const int i = t0 + threadIdx.x;
    int c = 0;
    if (i < ng) {
      int64_t s, e;
      row_range(g, giant_v[i], s, e);
      c = (int)((e - s + kGiantRow - 1) / kGiantRow);
    }
    int tile_total;
    const int x = block_exclusive_scan(c, sh, &tile_total);
    if (i < ng) giant_off[i] = acc + x;
    acc += tile_total;
  }
  if (threadIdx.x == 0) giant_off[ng] = acc;
}

// Every warp of the grid takes pieces of giant rows and ORs their labels into
// the row's bitmap.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_giant_or(GraphView<I> g, const int32_t* labels, const int32_t* large,
                                                     int32_t k0, const int32_t* giant_v, const int32_t* giant_slot,
                                                     const int32_t* giant_cnt, const int64_t* giant_off,
                                                     uint32_t* bitmaps, int64_t words) {
  pdl_enter();
  const int32_t ng = block_load(giant_cnt);
  const int64_t total = block_load(giant_off + ng);
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t pc = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; pc < total; pc += nw) {
    int lo = 0, hi = ng;  // last i with giant_off[i] <= pc
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (giant_off[mid] <= pc) lo = mid;
      else hi = mid;
    }
    const int32_t slot = giant_slot[lo];
    const int32_t a = large[k0 + slot];
    int64_t s, e;
    row_range(g, giant_v[lo], s, e);
    const int64_t ps = s + (pc - giant_off[lo]) * kGiantRow;
    const int64_t pe = min(e, ps + kGiantRow);
    uint32_t* bm = bitmaps + (int64_t)slot * words;
    for (int64_t p = (ps & ~int64_t(3)) + 4 * lane; p < pe; p += 128) {
      int32_t w4[4];
      if (g.vec && p + 4 <= g.nnz) {
        const int4 q = __ldg(reinterpret_cast<const int4*>(g.colind + p));
        w4[0] = q.x, w4[1] = q.y, w4[2] = q.z, w4[3] = q.w;
      } else {
#pragma unroll
        for (int t = 0; t < 4; t++) w4[t] = (p + t >= ps && p + t < pe) ? g.colind[p + t] : 0;
      }
#pragma unroll
      for (int t = 0; t < 4; t++) {
        const int32_t l = (p + t >= ps && p + t < pe) ? labels[w4[t]] : a;
        if (l != a) atomicOr(bm + (l >> 5), 1u << (l & 31));
      }
    }
  }
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_large_or(GraphView<I> g, const int32_t* labels, const int32_t* agg_ptr,
                                                     const int32_t* members, const int32_t* large, int32_t k0,
                                                     int32_t kb, const int64_t* chunk_off, uint32_t* bitmaps,
                                                     int64_t words, const int32_t* kb_dev, int32_t* giant_v,
                                                     int32_t* giant_slot, int32_t* giant_cnt) {
  pdl_enter();
  __shared__ __align__(16) int32_t stage[kBlock / 32][kStageWarpWords];
  if (kb_dev != nullptr) kb = block_load(kb_dev);
  const int64_t total = block_load(chunk_off + kb);
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < total; ch += nw) {
    int lo = 0, hi = kb;  // last i with chunk_off[i] <= ch
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (chunk_off[mid] <= ch) lo = mid;
      else hi = mid;
    }
    const int32_t a = large[k0 + lo];
    const int64_t mb = agg_ptr[a] + (ch - chunk_off[lo]) * 32;
    const int64_t me = min((int64_t)agg_ptr[a + 1], mb + 32);
    uint32_t* bm = bitmaps + (int64_t)lo * words;
    const GiantList gl{giant_v, giant_slot, giant_cnt, lo};
    walk_aggregate<I>(
        g, labels, members, mb, me, a, stage[threadIdx.x >> 5],
        [&](auto& lab) {
#pragma unroll
          for (int j = 0; j < (int)(sizeof(lab) / sizeof(lab[0])); j++)
            if (lab[j] >= 0) atomicOr(bm + (lab[j] >> 5), 1u << (lab[j] & 31));
        },
        &gl);
  }
}

// The bitmaps are emitted in segments of kEmitSeg words, a block per
// (bitmap, segment) pair, so that the bitmap of a hub aggregate (millions of
// set bits) is spread over the grid.  k_large_count: the set bits of every
// pair, seg_cnt[i * nseg + sg].
constexpr int64_t kEmitSeg = 4096;

__global__ void __launch_bounds__(kBlock) k_large_count(int32_t kb, const uint32_t* bitmaps, int64_t words, int nseg,
                                                        int32_t* seg_cnt, const int32_t* kb_dev) {
  pdl_enter();
  __shared__ int sh[40];
  if (kb_dev != nullptr) kb = block_load(kb_dev);
  for (int64_t pr = blockIdx.x; pr < (int64_t)kb * nseg; pr += gridDim.x) {
    const int64_t i = pr / nseg, sg = pr % nseg;
    const uint32_t* bm = bitmaps + i * words;
    const int64_t j0 = sg * kEmitSeg, j1 = min(words, j0 + kEmitSeg);
    int c = 0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) c += __popc(bm[j]);
    c = block_sum_i32(c, sh);
    if (threadIdx.x == 0) seg_cnt[pr] = c;
  }
}

// A block per (bitmap, segment): each warp owns a contiguous run of the
// segment's words; the warps' counts are exchanged once, then each warp
// writes the labels of its non-zero words in ascending order behind the
// segments and warps before it, and clears those words.  The block of a
// bitmap's first segment writes the row length.
__global__ void __launch_bounds__(kBlock) k_large_emit(const int32_t* large, int32_t k0, int32_t kb,
                                                       const int32_t* ub_ptr, uint32_t* bitmaps, int64_t words,
                                                       int nseg, const int32_t* seg_cnt, int32_t* tmp,
                                                       int32_t* c_cnt, const int32_t* kb_dev) {
  pdl_enter();
  constexpr int kW = kBlock / 32;
  __shared__ int64_t wsum[kW];
  __shared__ int64_t sbase, stotal;
  if (kb_dev != nullptr) kb = block_load(kb_dev);
  const int lane = lane_id(), w = threadIdx.x >> 5;
  for (int64_t pr = blockIdx.x; pr < (int64_t)kb * nseg; pr += gridDim.x) {
    const int64_t i = pr / nseg, sg = pr % nseg;
    const int32_t a = large[k0 + i];
    uint32_t* bm = bitmaps + i * words;
    const int64_t s0 = sg * kEmitSeg, s1 = min(words, s0 + kEmitSeg);
    const int64_t seg = ((s1 - s0 + kW - 1) / kW + 31) / 32 * 32;
    const int64_t w0 = min(s1, s0 + (int64_t)w * seg), w1 = min(s1, w0 + seg);
    if (threadIdx.x == 0) {
      int64_t b = 0, t = 0;
      for (int k = 0; k < nseg; k++) {
        const int64_t x = seg_cnt[i * nseg + k];
        b += k < sg ? x : 0;
        t += x;
      }
      sbase = b;
      stotal = t;
    }
    int64_t cnt = 0;
    for (int64_t j = w0 + lane; j < w1; j += 32) cnt += __popc(bm[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
    if (lane == 0) wsum[w] = cnt;
    __syncthreads();
    const int64_t out = ub_ptr[a] + sbase;
    int64_t run = 0;
#pragma unroll
    for (int k = 0; k < kW; k++) run += k < w ? wsum[k] : 0;
    for (int64_t j0 = w0; j0 < w1; j0 += 32) {
      const int64_t j = j0 + lane;
      uint32_t x = j < w1 ? bm[j] : 0u;
      if (__ballot_sync(kFull, x != 0u) == 0u) continue;
      const int c = __popc(x);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      int pos = incl - c;
      if (x != 0u) bm[j] = 0u;
      while (x) {
        const int bit = __ffs(x) - 1;
        x &= x - 1;
        tmp[out + run + pos++] = (int32_t)(j * 32 + bit);
      }
      run += __shfl_sync(kFull, incl, 31);
    }
    if (sg == 0 && threadIdx.x == 0) c_cnt[a] = (int32_t)stotal;
    __syncthreads();
  }
}

// Clears the bitmaps of a batch whose size is only known on the device.
__global__ void __launch_bounds__(kBlock) k_large_zero(uint32_t* bitmaps, int64_t words, const int32_t* kb_dev) {
  pdl_enter();
  const int64_t total = (int64_t)block_load(kb_dev) * words;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    bitmaps[i] = 0u;
}

// Single-batch path: copies nothing when the large aggregates overflowed the
// batch or the coarse rows exceed the output capacity (and flags the latter).
__device__ __forceinline__ bool pack_refused(const int32_t* err, const int32_t* total, int64_t cap) {
  if (err == nullptr) return false;
  const bool over = block_load(total) > cap;
  const int32_t e = block_load(err);
  if (over && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(const_cast<int32_t*>(err), kErrCapacity);
  return over || (e & kErrLargeOverflow) != 0;
}

constexpr int kPackWarpMax = 4096;  // longer coarse rows are copied by the whole grid

__global__ void __launch_bounds__(kBlock) k_coarse_pack(int64_t n_aggs, const int32_t* ub_ptr, const int32_t* c_cnt,
                                                        const int32_t* c_rowptr, const int32_t* tmp,
                                                        int32_t* c_colind, const int32_t* err, const int32_t* total,
                                                        int64_t cap) {
  pdl_enter();
  if (pack_refused(err, total, cap)) return;
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n_aggs; a += nw) {
    const int len = c_cnt[a];
    if (len > kPackWarpMax) continue;
    const int64_t src = ub_ptr[a], dst = c_rowptr[a];
    for (int i = lane; i < len; i += 32) c_colind[dst + i] = tmp[src + i];
  }
}

// Rows longer than kPackWarpMax (only large aggregates have them) are
// copied in chunks of kPackChunk entries, a block per chunk, so that one hub
// row of millions of entries is spread over the grid.  k_pack_chunks (one
// block) lays the chunks out: chunk_off[i] = chunks of the large rows before
// i, chunk_off[n_large] = all of them.
constexpr int64_t kPackChunk = 16384;

__global__ void __launch_bounds__(kBlock) k_pack_chunks(const int32_t* large, const int32_t* n_large,
                                                        const int32_t* c_cnt, int64_t* chunk_off, const int32_t* err,
                                                        const int32_t* total, int64_t cap) {
  pdl_enter();
  if (pack_refused(err, total, cap)) return;
  __shared__ int sh[40];
  const int32_t nl = block_load(n_large);
  int64_t acc = 0;
  for (int32_t t0 = 0; t0 < nl; t0 += kBlock) {
    const int32_t i = t0 + (int32_t)threadIdx.x;
    int ch = 0;
    if (i < nl) {
      const int64_t len = c_cnt[large[i]];
      ch = len > kPackWarpMax ? (int)((len + kPackChunk - 1) / kPackChunk) : 0;
    }
    int tile_total;
    const int x = block_exclusive_scan(ch, sh, &tile_total);
    if (i < nl) chunk_off[i] = acc + x;
    acc += tile_total;
  }
  if (threadIdx.x == 0) chunk_off[nl] = acc;
}

__global__ void __launch_bounds__(kBlock) k_coarse_pack_long(const int32_t* large, const int32_t* n_large,
                                                             const int64_t* chunk_off, const int32_t* ub_ptr,
                                                             const int32_t* c_cnt, const int32_t* c_rowptr,
                                                             const int32_t* tmp, int32_t* c_colind,
                                                             const int32_t* err, const int32_t* total, int64_t cap) {
  pdl_enter();
  if (pack_refused(err, total, cap)) return;
  const int32_t nl = block_load(n_large);
  const int64_t n_ch = block_load(chunk_off + nl);
  for (int64_t ch = blockIdx.x; ch < n_ch; ch += gridDim.x) {
    int lo = 0, hi = nl;  // the last row i with chunk_off[i] <= ch: the one holding chunk ch
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (chunk_off[mid] <= ch) lo = mid;
      else hi = mid;
    }
    const int32_t a = large[lo];
    const int64_t len = c_cnt[a];
    const int64_t k0 = (ch - chunk_off[lo]) * kPackChunk, k1 = min(len, k0 + kPackChunk);
    const int64_t src = ub_ptr[a], dst = c_rowptr[a];
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) c_colind[dst + k] = tmp[src + k];
  }
}

// ------------------------------------------------------------------ host side
int coarse_bitmap_blocks(const mis2_ctx* c) {
  const int64_t words = (std::max<int64_t>(c->max_n, 1) + 31) / 32;
  const int64_t cap = ((int64_t)256 << 20) / (words * 4);
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->sm_count * 2, cap));
}

template <typename I>
static GraphView<I> gview_of(const GraphArgs& g) {
  GraphView<I> gv;
  gv.rowptr = static_cast<const I*>(g.rowptr);
  gv.colind = g.colind;
  gv.n = g.n;
  gv.nnz = g.nnz;
  gv.vec = g.vec ? 1 : 0;
  gv.pad = 0;
  return gv;
}

// The rows of the aggregates that are neither small nor large.  Without the
// small-aggregate kernel (aggregates of many entries, as in 3D meshes):
// neighbour labels per vertex (k_coarse_cand), then a warp per aggregate
// (k_coarse_merge), and the hash-set kernel for the aggregates it leaves
// over; otherwise the hash-set kernel for every non-small aggregate.  Counts
// its launches.
template <typename I>
static int coarse_rows_launch(mis2_ctx* c, const GraphView<I>& gv, const int32_t* labels, int64_t n_aggs,
                              bool small_on, cudaStream_t st, bool cand_ready = false, bool ctr_fresh = false) {
  Scratch& s = c->s;
  const int rows_blocks = grid_for(c, n_aggs, kCoarseWarps, 16);
  if (small_on) {  // the aggregates k_coarse_small listed in s.left_mid
    launch_k(c, k_coarse_rows<I>, rows_blocks, kCoarseWarps * 32, st, gv, labels, n_aggs, s.agg_ptr, s.members, s.ub,
             s.ub_ptr, s.tmp, s.c_cnt, s.large, s.ctr + kCtrLarge, small_on, s.left_mid, s.ctr + kCtrCoarseRest);
    c->launches++;
    return MIS2_OK;
  }
  if (!ctr_fresh) MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrCoarseRest, 0, sizeof(int32_t), st));
  if (!cand_ready) {
    launch_k(c, k_coarse_cand<I>, grid_for(c, (gv.n + 31) / 32, kBlock / 32, 8), kBlock, st, gv, labels, s.cand);
    c->launches++;
  }
  launch_k(c, k_coarse_merge<I>, grid_for(c, n_aggs, kBlock / 32, 8), kBlock, st, gv, labels, n_aggs, s.agg_ptr,
           s.members, s.ub, s.ub_ptr,
                                                                          s.cand, s.tmp, s.c_cnt, s.left_mid,
                                                                          s.ctr + kCtrCoarseRest, small_on);
  launch_k(c, k_coarse_rows<I>, rows_blocks, kCoarseWarps * 32, st, gv, labels, n_aggs, s.agg_ptr, s.members, s.ub, s.ub_ptr,
                                                              s.tmp, s.c_cnt, s.large, s.ctr + kCtrLarge, small_on,
                                                              s.left_mid, s.ctr + kCtrCoarseRest);
  c->launches += 2;
  return MIS2_OK;
}

// Bitmaps per batch of large aggregates: as many as fit the bitmap scratch
// (sized for the context's largest graph), at most n_aggs.
static int32_t bitmap_slots(const mis2_ctx* c, int64_t n_aggs) {
  const int64_t words = (std::max<int64_t>(n_aggs, 1) + 31) / 32;
  const int64_t words_cap = (std::max<int64_t>(c->max_n, 1) + 31) / 32;
  return (int32_t)std::max<int64_t>(1, std::min<int64_t>((int64_t)coarse_bitmap_blocks(c) * words_cap / words,
                                                          std::max<int64_t>(n_aggs, 1)));
}

// Segments per bitmap of the emit: kEmitSeg words each, unless the
// (bitmap, segment) counts would not fit the n + 1 words of s.cursor (free
// by then), in which case one segment per bitmap.
static int emit_segments(const mis2_ctx* c, int64_t n_aggs) {
  const int64_t words = (std::max<int64_t>(n_aggs, 1) + 31) / 32;
  const int64_t nseg = (words + kEmitSeg - 1) / kEmitSeg;
  return (int64_t)bitmap_slots(c, n_aggs) * nseg <= c->max_n + 1 ? (int)nseg : 1;
}

// Large aggregates k_start..n_large-1 in batches of bitmaps, then the row
// offsets (one host read of the total) and the packed colind.
template <typename I>
static int coarse_tail(mis2_ctx* c, const GraphView<I>& gv, const int32_t* labels, int64_t n_aggs, int32_t n_large,
                       int32_t k_start, int32_t* c_rowptr, int32_t* c_colind, int64_t c_colind_cap, int64_t* c_nnz,
                       cudaStream_t st) {
  Scratch& s = c->s;
  if (n_large > k_start) {
    const int64_t words = (n_aggs + 31) / 32;
    const int32_t slots = bitmap_slots(c, n_aggs);
    timer_begin(c, kKcCoarse, st);
    for (int32_t k0 = k_start; k0 < n_large; k0 += slots) {
      const int32_t kb = std::min(slots, n_large - k0);
      MIS2_CUDA(cudaMemsetAsync(s.bitmaps, 0, (size_t)kb * words * sizeof(uint32_t), st));
      launch_k(c, k_large_chunks, 1, kBlock, st, s.large, k0, kb, s.agg_ptr, s.chunk_off, nullptr, nullptr, nullptr,
                                           s.ctr + kCtrGiant);
      launch_k(c, k_large_or<I>, c->sm_count * 8, kBlock, st, gv, labels, s.agg_ptr, s.members, s.large, k0, kb,
                                                        s.chunk_off, s.bitmaps, words, nullptr, s.giant_v,
                                                        s.giant_slot, s.ctr + kCtrGiant);
      launch_k(c, k_giant_pieces<I>, 1, kBlock, st, gv, s.giant_v, s.ctr + kCtrGiant, s.giant_off);
      launch_k(c, k_giant_or<I>, c->sm_count * 8, kBlock, st, gv, labels, s.large, k0, s.giant_v, s.giant_slot,
                                                        s.ctr + kCtrGiant, s.giant_off, s.bitmaps, words);
      const int nseg = emit_segments(c, n_aggs);
      launch_k(c, k_large_count, c->sm_count * 4, kBlock, st, kb, s.bitmaps, words, nseg, s.cursor, nullptr);
      launch_k(c, k_large_emit, c->sm_count * 4, kBlock, st, s.large, k0, kb, s.ub_ptr, s.bitmaps, words, nseg,
               s.cursor, s.tmp, s.c_cnt, nullptr);
      c->launches += 6;
    }
    timer_end(c, st);
    MIS2_CUDA(cudaGetLastError());
  }
  MIS2_TRY(exclusive_scan_i32(c, s.c_cnt, n_aggs, c_rowptr, s.ctr + kCtrCnnz, st));
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  const int64_t total = c->h_ctr[kCtrCnnz];
  if (total > c_colind_cap) return MIS2_ERR_INVALID_ARG;
  timer_begin(c, kKcCoarse, st);
  launch_k(c, k_coarse_pack, grid_for(c, n_aggs, kBlock / 32, 8), kBlock, st, n_aggs, s.ub_ptr, s.c_cnt, c_rowptr, s.tmp,
                                                                        c_colind, nullptr, nullptr, 0);
  c->launches++;
  if (n_large > 0) {
    launch_k(c, k_pack_chunks, 1, kBlock, st, s.large, s.ctr + kCtrLarge, s.c_cnt, s.chunk_off, nullptr, nullptr, 0);
    launch_k(c, k_coarse_pack_long, c->sm_count * 4, kBlock, st, s.large, s.ctr + kCtrLarge, s.chunk_off, s.ub_ptr,
             s.c_cnt, c_rowptr, s.tmp, c_colind, nullptr, nullptr, 0);
    c->launches += 2;
  }
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  *c_nnz = total;
  return MIS2_OK;
}

template <typename I>
static int coarsen_t(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                     int32_t* c_colind, int64_t c_colind_cap, int64_t* c_nnz, cudaStream_t st) {
  Scratch& s = c->s;
  GraphView<I> gv;
  gv.rowptr = static_cast<const I*>(g.rowptr);
  gv.colind = g.colind;
  gv.n = g.n;
  gv.nnz = g.nnz;
  gv.vec = g.vec ? 1 : 0;
  gv.pad = 0;
  const int64_t n = g.n;
  if (n_aggs == 0) {
    MIS2_CUDA(cudaMemsetAsync(c_rowptr, 0, sizeof(int32_t), st));
    *c_nnz = 0;
    return MIS2_OK;
  }
  timer_begin(c, kKcCoarse, st);
  MIS2_CUDA(cudaMemsetAsync(s.agg_cnt, 0, n_aggs * sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(s.ub, 0, n_aggs * sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrLarge, 0, 2 * sizeof(int32_t), st));
  launch_k(c, k_coarse_hist<I>, grid_for(c, n, kBlock), kBlock, st, gv, labels, s.agg_cnt, s.ub);
  c->launches++;
  timer_end(c, st);
  MIS2_TRY(exclusive_scan_i32(c, s.agg_cnt, n_aggs, s.agg_ptr, nullptr, st, s.cursor));
  MIS2_TRY(exclusive_scan_i32(c, s.ub, n_aggs, s.ub_ptr, nullptr, st));
  timer_begin(c, kKcCoarse, st);
  launch_k(c, k_coarse_scatter, grid_for(c, n, kBlock), kBlock, st, n, labels, s.cursor, s.members);
  // the batched path pays off when small aggregates are common: average
  // entries per aggregate at most half the sub-batch
  const bool small_on = n_aggs < ((int64_t)1 << kSmallLabelBits) && g.nnz <= (int64_t)(kSmallEntries / 2) * n_aggs;
  if (small_on) {
    MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrCoarseRest, 0, sizeof(int32_t), st));
    launch_k(c, k_coarse_small<I>, grid_for(c, (n_aggs + kSmallWindow - 1) / kSmallWindow, kBlock / 32, 8), kBlock,
             st, gv, labels, n_aggs, s.agg_ptr, s.members, s.ub, s.ub_ptr, s.tmp, s.c_cnt, s.left_mid,
             s.ctr + kCtrCoarseRest);
    c->launches++;
  }
  MIS2_TRY(coarse_rows_launch<I>(c, gv, labels, n_aggs, small_on, st));
  c->launches++;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  // large aggregates, in batches of `slots` bitmaps
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  return coarse_tail<I>(c, gv, labels, n_aggs, c->h_ctr[kCtrLarge], 0, c_rowptr, c_colind, c_colind_cap, c_nnz, st);
}

// The same coarse graph without a host round trip: the large aggregates go
// through one bitmap batch sized on the host from n_aggs, whose count is read
// on the device; the output capacity is checked on the device.  More large
// aggregates than one batch holds set kErrLargeOverflow; the caller then
// finishes the remaining batches (coarsen_fast_needs_retry,
// coarsen_fast_finish).
// The part of the fast coarse graph that needs the labels but not the
// aggregate count, so that it can be queued before the host learns n_aggs:
// the member counts and degree sums per aggregate (over every possible
// aggregate id: n words) and, for graphs dense enough that the
// candidate/merge path is likely (average degree >= kEarlyCandDegree), the
// per-vertex candidate labels.  Returns whether the candidates were queued.
constexpr int kEarlyCandDegree = 20;

template <typename I>
static int coarse_prelude_t(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, bool* cand_ready,
                            cudaStream_t st, bool hist_done) {
  Scratch& s = c->s;
  const GraphView<I> gv = gview_of<I>(g);
  const int64_t n = g.n;
  *cand_ready = false;
  if (n == 0) return MIS2_OK;
  timer_begin(c, kKcCoarse, st);
  if (!hist_done) {
    MIS2_CUDA(cudaMemsetAsync(s.agg_cnt, 0, n * sizeof(int32_t), st));
    MIS2_CUDA(cudaMemsetAsync(s.ub, 0, n * sizeof(int32_t), st));
    launch_k(c, k_coarse_hist<I>, grid_for(c, n, kBlock), kBlock, st, gv, labels, s.agg_cnt, s.ub);
    c->launches++;
  }
  if (g.nnz >= (int64_t)kEarlyCandDegree * n) {
    launch_k(c, k_coarse_cand<I>, grid_for(c, (n + 31) / 32, kBlock / 32, 8), kBlock, st, gv, labels, s.cand);
    c->launches++;
    *cand_ready = true;
  }
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

int coarsen_prelude(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, bool* cand_ready, cudaStream_t st,
                    bool hist_done) {
  return g.rp64 ? coarse_prelude_t<int64_t>(c, g, labels, cand_ready, st, hist_done)
                : coarse_prelude_t<int32_t>(c, g, labels, cand_ready, st, hist_done);
}

template <typename I>
static int coarsen_fast_t(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                          int32_t* c_colind, int64_t c_colind_cap, cudaStream_t st, bool prelude_done,
                          bool cand_ready, bool ctr_fresh) {
  Scratch& s = c->s;
  GraphView<I> gv;
  gv.rowptr = static_cast<const I*>(g.rowptr);
  gv.colind = g.colind;
  gv.n = g.n;
  gv.nnz = g.nnz;
  gv.vec = g.vec ? 1 : 0;
  gv.pad = 0;
  const int64_t n = g.n;
  if (!ctr_fresh) MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrCnnz, 0, sizeof(int32_t), st));
  if (n_aggs == 0) {
    MIS2_CUDA(cudaMemsetAsync(c_rowptr, 0, sizeof(int32_t), st));
    return MIS2_OK;
  }
  timer_begin(c, kKcCoarse, st);
  if (!prelude_done) {
    MIS2_CUDA(cudaMemsetAsync(s.agg_cnt, 0, n_aggs * sizeof(int32_t), st));
    MIS2_CUDA(cudaMemsetAsync(s.ub, 0, n_aggs * sizeof(int32_t), st));
  }
  if (!ctr_fresh) {
    MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrLarge, 0, 2 * sizeof(int32_t), st));
    MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrLargeKb, 0, sizeof(int32_t), st));
  }
  if (!prelude_done) {
    launch_k(c, k_coarse_hist<I>, grid_for(c, n, kBlock), kBlock, st, gv, labels, s.agg_cnt, s.ub);
    c->launches++;
  }
  timer_end(c, st);
  MIS2_TRY(exclusive_scan_i32(c, s.agg_cnt, n_aggs, s.agg_ptr, nullptr, st, s.cursor));
  MIS2_TRY(exclusive_scan_i32(c, s.ub, n_aggs, s.ub_ptr, nullptr, st));
  timer_begin(c, kKcCoarse, st);
  launch_k(c, k_coarse_scatter, grid_for(c, n, kBlock), kBlock, st, n, labels, s.cursor, s.members);
  // the batched path pays off when small aggregates are common: average
  // entries per aggregate at most half the sub-batch
  const bool small_on = n_aggs < ((int64_t)1 << kSmallLabelBits) && g.nnz <= (int64_t)(kSmallEntries / 2) * n_aggs;
  if (small_on) {
    if (!ctr_fresh) MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrCoarseRest, 0, sizeof(int32_t), st));
    launch_k(c, k_coarse_small<I>, grid_for(c, (n_aggs + kSmallWindow - 1) / kSmallWindow, kBlock / 32, 8), kBlock,
             st, gv, labels, n_aggs, s.agg_ptr, s.members, s.ub, s.ub_ptr, s.tmp, s.c_cnt, s.left_mid,
             s.ctr + kCtrCoarseRest);
    c->launches++;
  }
  MIS2_TRY(coarse_rows_launch<I>(c, gv, labels, n_aggs, small_on, st, cand_ready, ctr_fresh));
  const int64_t words = (n_aggs + 31) / 32;
  const int32_t slots = bitmap_slots(c, n_aggs);
  launch_k(c, k_large_chunks, 1, kBlock, st, s.large, 0, slots, s.agg_ptr, s.chunk_off, s.ctr + kCtrLarge,
                                       s.ctr + kCtrLargeKb, s.ctr + kCtrErr, s.ctr + kCtrGiant);
  launch_k(c, k_large_zero, c->sm_count * 2, kBlock, st, s.bitmaps, words, s.ctr + kCtrLargeKb);
  launch_k(c, k_large_or<I>, c->sm_count * 8, kBlock, st, gv, labels, s.agg_ptr, s.members, s.large, 0, slots,
                                                    s.chunk_off, s.bitmaps, words, s.ctr + kCtrLargeKb, s.giant_v,
                                                    s.giant_slot, s.ctr + kCtrGiant);
  launch_k(c, k_giant_pieces<I>, 1, kBlock, st, gv, s.giant_v, s.ctr + kCtrGiant, s.giant_off);
  launch_k(c, k_giant_or<I>, c->sm_count * 8, kBlock, st, gv, labels, s.large, 0, s.giant_v, s.giant_slot,
                                                    s.ctr + kCtrGiant, s.giant_off, s.bitmaps, words);
  const int nseg = emit_segments(c, n_aggs);
  launch_k(c, k_large_count, c->sm_count * 4, kBlock, st, slots, s.bitmaps, words, nseg, s.cursor,
           s.ctr + kCtrLargeKb);
  launch_k(c, k_large_emit, c->sm_count * 4, kBlock, st, s.large, 0, slots, s.ub_ptr, s.bitmaps, words, nseg, s.cursor,
           s.tmp, s.c_cnt, s.ctr + kCtrLargeKb);
  c->launches += 8;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  MIS2_TRY(exclusive_scan_i32(c, s.c_cnt, n_aggs, c_rowptr, s.ctr + kCtrCnnz, st));
  timer_begin(c, kKcCoarse, st);
  launch_k(c, k_coarse_pack, grid_for(c, n_aggs, kBlock / 32, 8), kBlock, st, n_aggs, s.ub_ptr, s.c_cnt, c_rowptr, s.tmp,
                                                                        c_colind, s.ctr + kCtrErr,
                                                                        s.ctr + kCtrCnnz, c_colind_cap);
  launch_k(c, k_pack_chunks, 1, kBlock, st, s.large, s.ctr + kCtrLarge, s.c_cnt, s.chunk_off, s.ctr + kCtrErr,
           s.ctr + kCtrCnnz, c_colind_cap);
  launch_k(c, k_coarse_pack_long, c->sm_count * 4, kBlock, st, s.large, s.ctr + kCtrLarge, s.chunk_off, s.ub_ptr,
           s.c_cnt, c_rowptr, s.tmp, c_colind, s.ctr + kCtrErr, s.ctr + kCtrCnnz, c_colind_cap);
  c->launches += 3;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

int coarsen_fast(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                 int32_t* c_colind, int64_t c_colind_cap, cudaStream_t st, bool prelude_done, bool cand_ready,
                 bool ctr_fresh) {
  return g.rp64 ? coarsen_fast_t<int64_t>(c, g, labels, n_aggs, c_rowptr, c_colind, c_colind_cap, st, prelude_done,
                                          cand_ready, ctr_fresh)
                : coarsen_fast_t<int32_t>(c, g, labels, n_aggs, c_rowptr, c_colind, c_colind_cap, st, prelude_done,
                                          cand_ready, ctr_fresh);
}

bool coarsen_fast_needs_retry(const mis2_ctx* c) { return (c->h_ctr[kCtrErr] & kErrLargeOverflow) != 0; }

// After a single-batch pass that overflowed (counters read back into
// c->h_ctr): the remaining large aggregates, the row offsets and the packing.
int coarsen_fast_finish(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                        int32_t* c_colind, int64_t c_colind_cap, int64_t* c_nnz, cudaStream_t st) {
  const int32_t n_large = c->h_ctr[kCtrLarge];
  const int32_t done = bitmap_slots(c, n_aggs);
  MIS2_CUDA(cudaMemsetAsync(c->s.ctr + kCtrErr, 0, sizeof(int32_t), st));
  if (g.rp64)
    return coarse_tail<int64_t>(c, gview_of<int64_t>(g), labels, n_aggs, n_large, done, c_rowptr, c_colind,
                                c_colind_cap, c_nnz, st);
  return coarse_tail<int32_t>(c, gview_of<int32_t>(g), labels, n_aggs, n_large, done, c_rowptr, c_colind,
                              c_colind_cap, c_nnz, st);
}

int coarsen_impl(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                 int32_t* c_colind, int64_t c_colind_cap, int64_t* c_nnz, cudaStream_t st) {
  return g.rp64 ? coarsen_t<int64_t>(c, g, labels, n_aggs, c_rowptr, c_colind, c_colind_cap, c_nnz, st)
                : coarsen_t<int32_t>(c, g, labels, n_aggs, c_rowptr, c_colind, c_colind_cap, c_nnz, st);
}

}  // namespace mis2
