// mis_rows.cuh -- the per-row work of one round of Algorithm 1 (Section
// III-A), written once and used both by the standalone kernels (host-driven
// round loop) and by the persistent device-loop kernel.
//
//   column: M_v = min(T_w : w in N[v]); IN -> OUT; keep v in worklist2 iff
//           M_v != OUT                      ("Refresh column status")
//   decide: OUT if some M_w = OUT, else IN if every M_w = T_v, else stay
//           undecided and take the next round's tuple right away
//           ("Decide IN/OUT of set" fused with the next "Refresh row status")
//
// Rows are visited by a group of G lanes (class 0), a warp (class 1) or a
// whole block (class 2); compaction of both worklists happens in the same
// pass through warp-aggregated appends (Section V-B).
//
// Subgraph runs (aggregation phase 2) need no special case here: vertices
// outside the subgraph hold T = OUT, which never lowers a minimum, and
// M = 0, which no column step can produce (IN maps to OUT), so decide reads
// M = 0 as "not a neighbour" in both of its tests.
#pragma once

#include "common.cuh"

namespace mis2 {

struct RowLists {
  int32_t* l[kClasses];
};

// Lane-per-row rows (G = 1): the warp first copies the column indices of
// its 32 rows into shared memory, one row at a time with 4-byte asynchronous
// copies, so every copy instruction touches one or two cache lines (per-lane
// loads of 32 different rows touch 32); then each lane issues its row's
// neighbour gathers back to back from its own slot.
constexpr int kLaneRowMax = 32;          // entries staged per row
constexpr int kRowSlot = kLaneRowMax + 1;  // padded slot: lane i reads bank (i + k) % 32
constexpr int kStageWarpWords = 32 * kRowSlot;

// Worklist appends of the lane-per-row passes collect in a per-warp
// shared-memory buffer and reach the global list in batches: one atomic per
// ~kAppendBuf entries instead of one per 32 rows.  (Every warp of the grid
// appends to the same counter, and same-address atomics serialise.)
constexpr int kAppendBuf = 256;
constexpr int kWarpSmemWords = kStageWarpWords + kAppendBuf;

struct WarpAppender {
  int32_t* buf;
  int32_t* list;
  int32_t* cnt;
  int n;
  __device__ __forceinline__ void flush() {
    __syncwarp();
    if (n == 0) return;
    const int lane = lane_id();
    int base = 0;
    if (lane == 0) base = atomicAdd(cnt, n);
    base = __shfl_sync(kFull, base, 0);
    if (list != nullptr)  // null list: count only
      for (int i = lane; i < n; i += 32) list[base + i] = buf[i];
    __syncwarp();
    n = 0;
  }
  // every lane of the warp calls this
  __device__ __forceinline__ void push(bool want, int32_t v) {
    const unsigned b = __ballot_sync(kFull, want);
    if (want) buf[n + __popc(b & ((1u << lane_id()) - 1u))] = v;
    n += __popc(b);
    if (n > kAppendBuf - 32) flush();
  }
};

// Stage each lane's row colind[s, s + len) (len <= kLaneRowMax, or len < 0:
// not staged) in the warp's shared area and return where this lane's row
// starts there.  When the 32 rows lie in ascending order in colind with
// little in between (worklists that still hold runs of consecutive vertices,
// possibly with holes), the whole span moves with 16-byte copies, 512
// contiguous bytes per instruction, gaps included; otherwise each row moves with
// one coalesced 4-byte copy per entry, into padded per-lane slots (4 rows
// per copy instruction when no row is longer than 8, 2 when none is longer
// than 16).  Every lane of the warp must call this; on return every staged
// row is visible to its lane, and *width (when given) holds 8, 16 or 32: the
// smallest of them bounding every staged row of the warp.  `nnz` bounds the
// 16-byte copies to the colind allocation.
__device__ __forceinline__ const int32_t* stage_rows_warp(const int32_t* __restrict__ colind, int64_t nnz, bool vec,
                                                          int64_t s, int len, int32_t* area, int* width = nullptr) {
  const int lane = lane_id();
  const int ml = (int)__reduce_max_sync(kFull, (unsigned)(len > 0 ? len : 0));
  const int wd = ml <= 8 ? 8 : (ml <= 16 ? 16 : 32);
  if (width != nullptr) *width = wd;
  const int64_t s_next = __shfl_down_sync(kFull, s, 1);
  const int64_t e = s + (len > 0 ? len : 0);
  const bool ordered = lane == 31 || e <= s_next;
  const int64_t s0 = __shfl_sync(kFull, s, 0);
  const int64_t e31 = __shfl_sync(kFull, e, 31);
  const int64_t a = s0 & ~int64_t(3);
  const int64_t nq = (e31 - a + 3) >> 2;
  // copied words at most 1.5x the staged ones (plus alignment slack)
  const int64_t useful = __reduce_add_sync(kFull, (unsigned)(len > 0 ? len : 0));
  if (vec && __all_sync(kFull, len >= 0 && ordered) && nq * 4 <= kStageWarpWords && a + nq * 4 <= nnz &&
      2 * nq * 4 <= 3 * useful + 64) {
    for (int64_t q = lane; q < nq; q += 32) cp_async16(area + 4 * q, colind + a + 4 * q);
    cp_async_wait_all();
    __syncwarp();
    return area + (s - a);
  }
  if (wd == 8) {
#pragma unroll
    for (int j0 = 0; j0 < 32; j0 += 4) {
      const int j = j0 + (lane >> 3), c = lane & 7;
      const int64_t sj = __shfl_sync(kFull, s, j);
      const int lj = __shfl_sync(kFull, len, j);
      if (c < lj) cp_async4(area + j * kRowSlot + c, colind + sj + c);
    }
  } else if (wd == 16) {
#pragma unroll 4
    for (int j0 = 0; j0 < 32; j0 += 2) {
      const int j = j0 + (lane >> 4), c = lane & 15;
      const int64_t sj = __shfl_sync(kFull, s, j);
      const int lj = __shfl_sync(kFull, len, j);
      if (c < lj) cp_async4(area + j * kRowSlot + c, colind + sj + c);
    }
  } else {
#pragma unroll 4
    for (int j = 0; j < 32; j++) {
      const int64_t sj = __shfl_sync(kFull, s, j);
      const int lj = __shfl_sync(kFull, len, j);
      if (lane < lj) cp_async4(area + j * kRowSlot + lane, colind + sj + lane);
    }
  }
  cp_async_wait_all();
  __syncwarp();
  return area + lane * kRowSlot;
}

// min(m, T[row[k]] for k < len) with W unrolled gathers (len <= W); between()
// runs after the gathers are issued, before their values are used.
template <int W, bool NC, typename F>
__device__ __forceinline__ uint32_t gather_min(const uint32_t* T, const int32_t* row, int len, uint32_t m,
                                               F&& between) {
  uint32_t t[W];
#pragma unroll
  for (int k = 0; k < W; k++) t[k] = k < len ? ld<NC>(T + row[k]) : kOut;
  between();
#pragma unroll
  for (int k = 0; k < W; k++) m = min(m, t[k]);
  return m;
}

// The decide tests over M[row[k]], k < len (len <= W): any OUT, all equal to
// t or 0 (masked neighbours of a phase-2 MIS-2).  Each such M is OUT, 0 or
// at most t = T_v (v lies in every neighbour's closed neighbourhood, whose
// minimum M is, and T_v has not changed since), so "any OUT" is max == OUT
// and, when there is none, "all t or 0" is min(M - 1) >= t - 1 (0 wraps to
// the largest value).  t >= 1 for an undecided vertex.
template <int W, bool NC, typename F>
__device__ __forceinline__ void gather_decide(const uint32_t* M, const int32_t* row, int len, uint32_t t,
                                              bool& any_out, bool& all_eq, F&& between) {
  uint32_t mw[W];
#pragma unroll
  for (int k = 0; k < W; k++) mw[k] = k < len ? ld<NC>(M + row[k]) : t;
  between();
  uint32_t mx = 0u, mn = ~0u;
#pragma unroll
  for (int k = 0; k < W; k++) {
    mx = max(mx, mw[k]);
    mn = min(mn, mw[k] - 1u);
  }
  any_out |= mx == kOut;
  all_eq &= mn >= t - 1u;
}

template <typename I, bool NC>
__device__ __forceinline__ void column_lane_rows(const GraphView<I>& g, const uint32_t* T, uint32_t* M,
                                                 const int32_t* wl_in, int n_in, int32_t* wl_out, int32_t* cnt_out,
                                                 int64_t* dsum, int64_t warp_begin, int64_t warp_stride,
                                                 int32_t* stage_warp) {
  const int lane = lane_id();
  WarpAppender app{stage_warp + kStageWarpWords, wl_out, cnt_out, 0};
  int64_t dacc = 0;
  // the next iteration's vertex and row bounds are loaded while this
  // iteration's gathers are in flight
  // contiguous batch ranges per warp: the kept rows leave in long ascending
  // runs, so the next round's batches still stage as one span
  const int64_t nbat = ((int64_t)n_in + 31) / 32;
  const int64_t per = (nbat + warp_stride - 1) / warp_stride;
  int64_t base = warp_begin * per * 32;
  const int64_t end = min((int64_t)n_in, (warp_begin + 1) * per * 32);
  bool an = base + lane < end;
  int32_t vn = 0;
  int64_t sn = 0, en = 0;
  if (an) {
    vn = ld<false>(wl_in + base + lane);
    row_range(g, vn, sn, en);
  }
  for (; base < end; base += 32) {
    const bool active = an;
    const int32_t v = vn;
    const int64_t s = sn, e = en;
    const int len = active && e - s <= kLaneRowMax ? (int)(e - s) : -1;
    int wd;
    const int32_t* mine = stage_rows_warp(g.colind, g.nnz, g.vec, s, len, stage_warp, &wd);
    const int64_t inext = base + 32 + lane;
    an = inext < end;
    if (an) vn = ld<false>(wl_in + inext);
    uint32_t m = kOut;
    if (active) {
      m = ld<NC>(T + v);
      if (len >= 0) {
        auto nb = [&]() {
          if (an) row_range(g, vn, sn, en);
        };
        if (wd == 8) m = gather_min<8, NC>(T, mine, len, m, nb);
        else if (wd == 16) m = gather_min<16, NC>(T, mine, len, m, nb);
        else m = gather_min<32, NC>(T, mine, len, m, nb);
      } else {
        if (an) row_range(g, vn, sn, en);
        visit_row<1>(g.colind, g.nnz, s, e, 0, g.vec, [&](int32_t w) { m = min(m, ld<NC>(T + w)); });
      }
    } else if (an) {
      row_range(g, vn, sn, en);
    }
    bool keep = false;
    if (active) {
      if (m == kIn) m = kOut;
      M[v] = m;
      keep = m != kOut;
    }
    __syncwarp();  // staged rows are rewritten by the next iteration's copies
    app.push(keep, v);
    dacc += active ? e - s : 0;
  }
  app.flush();
  if (dsum != nullptr) warp_accumulate(dacc, dsum);
}

template <typename I, bool NC, bool GUARD = false>
__device__ __forceinline__ void decide_lane_rows(const GraphView<I>& g, uint32_t* T, const uint32_t* M,
                                                 const int32_t* wl_in, int n_in, int32_t* wl_out, int32_t* cnt_out,
                                                 int64_t* dsum, const PrioCfg& p, uint32_t next_iter,
                                                 int64_t warp_begin, int64_t warp_stride, int32_t* stage_warp) {
  const int lane = lane_id();
  WarpAppender app{stage_warp + kStageWarpWords, wl_out, cnt_out, 0};
  int64_t dacc = 0;
  // contiguous batch ranges per warp: the kept rows leave in long ascending
  // runs, so the next round's batches still stage as one span
  const int64_t nbat = ((int64_t)n_in + 31) / 32;
  const int64_t per = (nbat + warp_stride - 1) / warp_stride;
  int64_t base = warp_begin * per * 32;
  const int64_t end = min((int64_t)n_in, (warp_begin + 1) * per * 32);
  bool an = base + lane < end;
  // GUARD (visiting every vertex, no worklists): vertices already IN or OUT
  // are skipped before their rows are read
  auto undecided = [&](int32_t x) {
    const uint32_t tv = ld<false>(T + x);
    return tv != kIn && tv != kOut;
  };
  int32_t vn = 0;
  int64_t sn = 0, en = 0;
  if (an) {
    vn = ld<false>(wl_in + base + lane);
    if (GUARD) an = undecided(vn);
    if (an) row_range(g, vn, sn, en);
  }
  for (; base < end; base += 32) {
    const bool active = an;
    const int32_t v = vn;
    const int64_t s = sn, e = en;
    const int len = active && e - s <= kLaneRowMax ? (int)(e - s) : -1;
    int wd;
    const int32_t* mine = stage_rows_warp(g.colind, g.nnz, g.vec, s, len, stage_warp, &wd);
    const int64_t inext = base + 32 + lane;
    an = inext < end;
    if (an) vn = ld<false>(wl_in + inext);
    if (GUARD && an) an = undecided(vn);
    bool keep = false;
    if (active) {
      const uint32_t t = ld<false>(T + v);
      const uint32_t mv = ld<NC>(M + v);
      bool any_out = mv == kOut, all_eq = mv == t;
      if (len >= 0) {
        auto nb = [&]() {
          if (an) row_range(g, vn, sn, en);
        };
        if (wd == 8) gather_decide<8, NC>(M, mine, len, t, any_out, all_eq, nb);
        else if (wd == 16) gather_decide<16, NC>(M, mine, len, t, any_out, all_eq, nb);
        else gather_decide<32, NC>(M, mine, len, t, any_out, all_eq, nb);
      } else {
        if (an) row_range(g, vn, sn, en);
        visit_row<1>(g.colind, g.nnz, s, e, 0, g.vec, [&](int32_t w) {
          const uint32_t x = ld<NC>(M + w);
          any_out |= x == kOut;
          all_eq &= (x == t) | (x == 0u);
        });
      }
      uint32_t nt;
      if (any_out) {
        nt = kOut;
      } else if (all_eq) {
        nt = kIn;
      } else {
        nt = make_tuple(p, next_iter, (uint32_t)v);
        keep = true;
      }
      T[v] = nt;
    } else if (an) {
      row_range(g, vn, sn, en);
    }
    __syncwarp();
    app.push(keep, v);
    dacc += active ? e - s : 0;
  }
  app.flush();
  if (dsum != nullptr) warp_accumulate(dacc, dsum);
}

template <int G, typename I, bool NC>
__device__ __forceinline__ void column_group_rows(const GraphView<I>& g, const uint32_t* T, uint32_t* M,
                                                  const int32_t* wl_in, int n_in, int32_t* wl_out,
                                                  int32_t* cnt_out, int64_t* dsum, int64_t warp_begin,
                                                  int64_t warp_stride) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  int64_t dacc = 0;
  for (int64_t base = warp_begin * RPW; base < n_in; base += warp_stride * RPW) {
    const int64_t i = base + sub;
    const bool active = i < n_in;
    int32_t v = 0;
    uint32_t m = kOut;
    int64_t len = 0;
    if (active) {
      v = ld<false>(wl_in + i);
      int64_t s, e;
      row_range(g, v, s, e);
      len = e - s;
      m = ld<NC>(T + v);
      visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) { m = min(m, ld<NC>(T + w)); });
    }
    m = group_min<G>(m);
    bool keep = false;
    if (active && lg == 0) {
      if (m == kIn) m = kOut;
      M[v] = m;
      keep = m != kOut;
    }
    warp_append(keep, v, wl_out, cnt_out);
    dacc += lg == 0 ? len : 0;
  }
  if (dsum != nullptr) warp_accumulate(dacc, dsum);
}

template <int G, typename I, bool NC, bool GUARD = false>
__device__ __forceinline__ void decide_group_rows(const GraphView<I>& g, uint32_t* T, const uint32_t* M,
                                                  const int32_t* wl_in, int n_in, int32_t* wl_out,
                                                  int32_t* cnt_out, int64_t* dsum, const PrioCfg& p,
                                                  uint32_t next_iter, int64_t warp_begin,
                                                  int64_t warp_stride) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  int64_t dacc = 0;
  for (int64_t base = warp_begin * RPW; base < n_in; base += warp_stride * RPW) {
    const int64_t i = base + sub;
    bool active = i < n_in;
    int32_t v = 0;
    uint32_t t = 0;
    bool any_out = false, all_eq = true;
    int64_t len = 0;
    if (active) {
      v = ld<false>(wl_in + i);
      t = ld<false>(T + v);
      if (GUARD && (t == kIn || t == kOut)) active = false;
    }
    if (active) {
      int64_t s, e;
      row_range(g, v, s, e);
      len = e - s;
      const uint32_t mv = ld<NC>(M + v);
      any_out = mv == kOut;
      all_eq = mv == t;
      visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) {
        const uint32_t mw = ld<NC>(M + w);
        any_out |= mw == kOut;
        all_eq &= (mw == t) | (mw == 0u);
      });
    }
    any_out = group_any<G>(any_out);
    all_eq = group_all<G>(all_eq);
    bool keep = false;
    if (active && lg == 0) {
      uint32_t nt;
      if (any_out) {
        nt = kOut;
      } else if (all_eq) {
        nt = kIn;
      } else {
        nt = make_tuple(p, next_iter, (uint32_t)v);
        keep = true;
      }
      T[v] = nt;
    }
    warp_append(keep, v, wl_out, cnt_out);
    dacc += lg == 0 ? len : 0;
  }
  if (dsum != nullptr) warp_accumulate(dacc, dsum);
}

template <typename I, bool NC>
__device__ __forceinline__ void column_block_rows(const GraphView<I>& g, const uint32_t* T, uint32_t* M,
                                                  const int32_t* wl_in, int n_in, int32_t* wl_out,
                                                  int32_t* cnt_out, int64_t* dsum, int64_t blk_begin,
                                                  int64_t blk_stride, uint32_t* sh) {
  for (int64_t i = blk_begin; i < n_in; i += blk_stride) {
    const int32_t v = ld<false>(wl_in + i);
    int64_t s, e;
    row_range(g, v, s, e);
    uint32_t m = threadIdx.x == 0 ? ld<NC>(T + v) : kOut;
    visit_row<kBlock>(g.colind, g.nnz, s, e, threadIdx.x, g.vec,
                      [&](int32_t w) { m = min(m, ld<NC>(T + w)); });
    m = block_min_u32(m, sh);
    if (threadIdx.x == 0) {
      if (m == kIn) m = kOut;
      M[v] = m;
      if (m != kOut) {
        const int32_t pos = atomicAdd(cnt_out, 1);
        if (wl_out != nullptr) wl_out[pos] = v;
      }
      if (dsum != nullptr) atomicAdd(reinterpret_cast<unsigned long long*>(dsum), (unsigned long long)(e - s));
    }
  }
}

template <typename I, bool NC, bool GUARD = false>
__device__ __forceinline__ void decide_block_rows(const GraphView<I>& g, uint32_t* T, const uint32_t* M,
                                                  const int32_t* wl_in, int n_in, int32_t* wl_out,
                                                  int32_t* cnt_out, int64_t* dsum, const PrioCfg& p,
                                                  uint32_t next_iter, int64_t blk_begin,
                                                  int64_t blk_stride, uint32_t* sh) {
  for (int64_t i = blk_begin; i < n_in; i += blk_stride) {
    const int32_t v = ld<false>(wl_in + i);
    const uint32_t t = ld<false>(T + v);
    if (GUARD && (t == kIn || t == kOut)) continue;  // the same value in every thread
    int64_t s, e;
    row_range(g, v, s, e);
    bool any_out = false, all_eq = true;
    if (threadIdx.x == 0) {
      const uint32_t mv = ld<NC>(M + v);
      any_out = mv == kOut;
      all_eq = mv == t;
    }
    visit_row<kBlock>(g.colind, g.nnz, s, e, threadIdx.x, g.vec, [&](int32_t w) {
      const uint32_t mw = ld<NC>(M + w);
      any_out |= mw == kOut;
      all_eq &= (mw == t) | (mw == 0u);
    });
    // OR of any_out into bit 0, AND of all_eq through the count of failures
    const int bad = __syncthreads_count(!all_eq);
    const int outs = __syncthreads_count(any_out);
    if (threadIdx.x == 0) {
      uint32_t nt;
      if (outs > 0) {
        nt = kOut;
      } else if (bad == 0) {
        nt = kIn;
      } else {
        nt = make_tuple(p, next_iter, (uint32_t)v);
        const int32_t pos = atomicAdd(cnt_out, 1);
        if (wl_out != nullptr) wl_out[pos] = v;
      }
      T[v] = nt;
      if (dsum != nullptr) atomicAdd(reinterpret_cast<unsigned long long*>(dsum), (unsigned long long)(e - s));
    }
    __syncthreads();
    (void)sh;
  }
}

// Round-0 set-up: T_v for every vertex of the (sub)graph, OUT / M = 0 for
// the others, and worklist 1 filled per row class (Algorithm 1: worklist1 =
// worklist2 = all vertices; worklist 2 is written too when wl2.l[0] is not
// null, else only its sizes, since its round-0 content equals worklist 1's).
// labels == null: whole graph; otherwise the subgraph {v : labels[v] == -1}.
// Each block takes a contiguous vertex range and appends its members of a
// class as one ascending run (one reservation per block and class), so the
// lists start as long ascending runs: the passes stage 32 consecutive rows
// as one span, and keep that order in their outputs.  Within the block each
// thread owns a contiguous sub-range, so one block scan of the per-thread
// class counts places every entry; the row bounds of a thread's vertices are
// loaded kInitBatch at a time, so their latencies overlap.  Every thread of
// the block must call this.
constexpr int kInitBatch = 16;

template <typename I>
__device__ __forceinline__ void mis_init_rows(const GraphView<I>& g, const int32_t* labels, const PrioCfg& p,
                                              uint32_t* T, uint32_t* M, RowLists wl1, RowLists wl2,
                                              int32_t* c1, int32_t* c2, int32_t warp_degree,
                                              int32_t block_degree) {
  __shared__ int sh_scan[40];
  __shared__ int32_t sh_base1[kClasses], sh_base2[kClasses];
  const int64_t per = (g.n + gridDim.x - 1) / gridDim.x;
  const int64_t v0 = min(g.n, (int64_t)blockIdx.x * per), v1 = min(g.n, v0 + per);
  const int64_t q = (v1 - v0 + blockDim.x - 1) / blockDim.x;
  const int64_t t0 = min(v1, v0 + (int64_t)threadIdx.x * q), t1 = min(v1, t0 + q);
  // class of each vertex of [b, b + kInitBatch) ∩ [t0, t1) (-1: outside the
  // (sub)graph or the range), from the kInitBatch + 1 consecutive row
  // offsets rowptr[b ..], all loaded before any is used
  auto classes = [&](int64_t b, int (&cls)[kInitBatch]) {
    I rp[kInitBatch + 1];
    int32_t lab[kInitBatch];
#pragma unroll
    for (int k = 0; k <= kInitBatch; k++) rp[k] = b + k <= t1 ? __ldg(g.rowptr + b + k) : (I)0;
#pragma unroll
    for (int k = 0; k < kInitBatch; k++) lab[k] = (labels != nullptr && b + k < t1) ? ld<false>(labels + b + k) : -1;
#pragma unroll
    for (int k = 0; k < kInitBatch; k++)
      cls[k] = (b + k < t1 && lab[k] == -1) ? row_class((int64_t)(rp[k + 1] - rp[k]), warp_degree, block_degree) : -1;
  };
  int cnt[kClasses] = {0, 0, 0};
  for (int64_t b = t0; b < t1; b += kInitBatch) {
    int cls[kInitBatch];
    classes(b, cls);
#pragma unroll
    for (int k = 0; k < kInitBatch; k++) {
      const int64_t v = b + k;
      if (v >= t1) break;
      if (cls[k] >= 0) {
        T[v] = make_tuple(p, 0u, (uint32_t)v);
        cnt[0] += cls[k] == 0;
        cnt[1] += cls[k] == 1;
        cnt[2] += cls[k] == 2;
      } else {
        T[v] = kOut;
        M[v] = 0u;
      }
    }
  }
  int pos[kClasses];
#pragma unroll
  for (int k = 0; k < kClasses; k++) {
    int total;
    pos[k] = block_exclusive_scan(cnt[k], sh_scan, &total);
    if (threadIdx.x == 0) {
      sh_base1[k] = total > 0 ? atomicAdd(c1 + k, total) : 0;
      sh_base2[k] = total > 0 ? atomicAdd(c2 + k, total) : 0;
    }
  }
  __syncthreads();
  const bool both = wl2.l[0] != nullptr;
  for (int64_t b = t0; b < t1; b += kInitBatch) {
    int cls[kInitBatch];
    classes(b, cls);
#pragma unroll
    for (int k = 0; k < kInitBatch; k++) {
      const int c = cls[k];
      if (c < 0) continue;
      const int at = c == 0 ? pos[0]++ : (c == 1 ? pos[1]++ : pos[2]++);
      int32_t* L1 = c == 0 ? wl1.l[0] : (c == 1 ? wl1.l[1] : wl1.l[2]);
      L1[sh_base1[c] + at] = (int32_t)(b + k);
      if (both) {
        int32_t* L2 = c == 0 ? wl2.l[0] : (c == 1 ? wl2.l[1] : wl2.l[2]);
        L2[sh_base2[c] + at] = (int32_t)(b + k);
      }
    }
  }
}

}  // namespace mis2
