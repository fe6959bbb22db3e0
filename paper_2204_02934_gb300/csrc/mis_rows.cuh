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

// Lane-per-row rows (G = 1) stage their column indices in shared memory with
// asynchronous 16-byte copies issued all at once, then issue every neighbour
// gather back to back: a row costs about two memory latencies instead of one
// per 16-byte chunk.
constexpr int kLaneRowMax = 32;                          // entries staged per lane
constexpr int kStageInt4 = (kLaneRowMax + 3) / 4 + 1;   // 9 int4 cover 32 entries at any alignment
constexpr int kStageWarpInt4 = 32 * kStageInt4;

// Stage colind[s, e) into `my`; returns the word offset of colind[s] inside
// the staged words, or -1 when the row does not fit (too long, buffer not
// 16-byte aligned, or the last 16-byte chunk would pass nnz).
template <typename I>
__device__ __forceinline__ int stage_row(const GraphView<I>& g, int64_t s, int64_t e, int4* my) {
  if (!g.vec || e - s > kLaneRowMax) return -1;
  const int64_t a = s & ~int64_t(3);
  const int nq = (int)((e - a + 3) >> 2);
  if (a + 4 * (int64_t)nq > g.nnz) return -1;
#pragma unroll
  for (int k = 0; k < kStageInt4; k++)
    if (k < nq) cp_async16(my + k, g.colind + a + 4 * k);
  return (int)(s - a);
}

template <typename I, bool NC>
__device__ __forceinline__ void column_lane_rows(const GraphView<I>& g, const uint32_t* T, uint32_t* M,
                                                 const int32_t* wl_in, int n_in, int32_t* wl_out, int32_t* cnt_out,
                                                 int64_t* dsum, int64_t warp_begin, int64_t warp_stride,
                                                 int4* stage_warp) {
  const int lane = lane_id();
  int4* my = stage_warp + lane * kStageInt4;
  const int32_t* myw = reinterpret_cast<const int32_t*>(my);
  for (int64_t base = warp_begin * 32; base < n_in; base += warp_stride * 32) {
    const int64_t i = base + lane;
    const bool active = i < n_in;
    int32_t v = 0;
    int64_t s = 0, e = 0;
    int off = -1;
    if (active) {
      v = ld<false>(wl_in + i);
      row_range(g, v, s, e);
      off = stage_row(g, s, e, my);
    }
    cp_async_wait_all();
    uint32_t m = kOut;
    if (active) {
      m = ld<NC>(T + v);
      if (off >= 0) {
        const int len = (int)(e - s);
#pragma unroll
        for (int k = 0; k < kLaneRowMax; k++)
          if (k < len) m = min(m, ld<NC>(T + myw[off + k]));
      } else {
        visit_row<1>(g.colind, g.nnz, s, e, 0, g.vec, [&](int32_t w) { m = min(m, ld<NC>(T + w)); });
      }
    }
    bool keep = false;
    if (active) {
      if (m == kIn) m = kOut;
      M[v] = m;
      keep = m != kOut;
    }
    warp_append(keep, v, wl_out, cnt_out);
    if (dsum != nullptr) warp_accumulate(e - s, dsum);
  }
}

template <typename I, bool NC>
__device__ __forceinline__ void decide_lane_rows(const GraphView<I>& g, uint32_t* T, const uint32_t* M,
                                                 const int32_t* wl_in, int n_in, int32_t* wl_out, int32_t* cnt_out,
                                                 int64_t* dsum, const PrioCfg& p, uint32_t next_iter,
                                                 int64_t warp_begin, int64_t warp_stride, int4* stage_warp) {
  const int lane = lane_id();
  int4* my = stage_warp + lane * kStageInt4;
  const int32_t* myw = reinterpret_cast<const int32_t*>(my);
  for (int64_t base = warp_begin * 32; base < n_in; base += warp_stride * 32) {
    const int64_t i = base + lane;
    const bool active = i < n_in;
    int32_t v = 0;
    int64_t s = 0, e = 0;
    int off = -1;
    if (active) {
      v = ld<false>(wl_in + i);
      row_range(g, v, s, e);
      off = stage_row(g, s, e, my);
    }
    cp_async_wait_all();
    bool keep = false;
    if (active) {
      const uint32_t t = ld<false>(T + v);
      const uint32_t mv = ld<NC>(M + v);
      bool any_out = mv == kOut, all_eq = mv == t;
      if (off >= 0) {
        const int len = (int)(e - s);
#pragma unroll
        for (int k = 0; k < kLaneRowMax; k++) {
          if (k < len) {
            const uint32_t mw = ld<NC>(M + myw[off + k]);
            any_out |= mw == kOut;
            all_eq &= (mw == t) | (mw == 0u);
          }
        }
      } else {
        visit_row<1>(g.colind, g.nnz, s, e, 0, g.vec, [&](int32_t w) {
          const uint32_t mw = ld<NC>(M + w);
          any_out |= mw == kOut;
          all_eq &= (mw == t) | (mw == 0u);
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
    }
    warp_append(keep, v, wl_out, cnt_out);
    if (dsum != nullptr) warp_accumulate(e - s, dsum);
  }
}

template <int G, typename I, bool NC>
__device__ __forceinline__ void column_group_rows(const GraphView<I>& g, const uint32_t* T, uint32_t* M,
                                                  const int32_t* wl_in, int n_in, int32_t* wl_out,
                                                  int32_t* cnt_out, int64_t* dsum, int64_t warp_begin,
                                                  int64_t warp_stride) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
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
    if (dsum != nullptr) warp_accumulate(lg == 0 ? len : 0, dsum);
  }
}

template <int G, typename I, bool NC>
__device__ __forceinline__ void decide_group_rows(const GraphView<I>& g, uint32_t* T, const uint32_t* M,
                                                  const int32_t* wl_in, int n_in, int32_t* wl_out,
                                                  int32_t* cnt_out, int64_t* dsum, const PrioCfg& p,
                                                  uint32_t next_iter, int64_t warp_begin,
                                                  int64_t warp_stride) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  for (int64_t base = warp_begin * RPW; base < n_in; base += warp_stride * RPW) {
    const int64_t i = base + sub;
    const bool active = i < n_in;
    int32_t v = 0;
    uint32_t t = 0;
    bool any_out = false, all_eq = true;
    int64_t len = 0;
    if (active) {
      v = ld<false>(wl_in + i);
      int64_t s, e;
      row_range(g, v, s, e);
      len = e - s;
      t = ld<false>(T + v);
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
    if (dsum != nullptr) warp_accumulate(lg == 0 ? len : 0, dsum);
  }
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
      if (m != kOut) wl_out[atomicAdd(cnt_out, 1)] = v;
      if (dsum != nullptr) atomicAdd(reinterpret_cast<unsigned long long*>(dsum), (unsigned long long)(e - s));
    }
  }
}

template <typename I, bool NC>
__device__ __forceinline__ void decide_block_rows(const GraphView<I>& g, uint32_t* T, const uint32_t* M,
                                                  const int32_t* wl_in, int n_in, int32_t* wl_out,
                                                  int32_t* cnt_out, int64_t* dsum, const PrioCfg& p,
                                                  uint32_t next_iter, int64_t blk_begin,
                                                  int64_t blk_stride, uint32_t* sh) {
  for (int64_t i = blk_begin; i < n_in; i += blk_stride) {
    const int32_t v = ld<false>(wl_in + i);
    int64_t s, e;
    row_range(g, v, s, e);
    const uint32_t t = ld<false>(T + v);
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
        wl_out[atomicAdd(cnt_out, 1)] = v;
      }
      T[v] = nt;
      if (dsum != nullptr) atomicAdd(reinterpret_cast<unsigned long long*>(dsum), (unsigned long long)(e - s));
    }
    __syncthreads();
    (void)sh;
  }
}

// Round-0 set-up: T_v for every vertex of the (sub)graph, OUT / M = 0 for
// the others, and both worklists filled per row class (Algorithm 1:
// worklist1 = worklist2 = all vertices).  labels == null: whole graph;
// otherwise the subgraph {v : labels[v] == -1}.
template <typename I>
__device__ __forceinline__ void mis_init_rows(const GraphView<I>& g, const int32_t* labels, const PrioCfg& p,
                                              uint32_t* T, uint32_t* M, RowLists wl1, RowLists wl2,
                                              int32_t* c1, int32_t* c2, int32_t warp_degree,
                                              int32_t block_degree, int64_t thread_begin,
                                              int64_t thread_stride) {
  const int lane = lane_id();
  for (int64_t base = thread_begin - lane; base < g.n; base += thread_stride) {
    const int64_t v = base + lane;
    int cls = -1;
    if (v < g.n) {
      const bool member = labels == nullptr || ld<false>(labels + v) == -1;
      if (member) {
        int64_t s, e;
        row_range(g, v, s, e);
        cls = row_class(e - s, warp_degree, block_degree);
        T[v] = make_tuple(p, 0u, (uint32_t)v);
      } else {
        T[v] = kOut;
        M[v] = 0u;
      }
    }
#pragma unroll
    for (int c = 0; c < kClasses; c++) {
      warp_append(cls == c, (int32_t)v, wl1.l[c], c1 + c);
      warp_append(cls == c, (int32_t)v, wl2.l[c], c2 + c);
    }
  }
}

}  // namespace mis2
