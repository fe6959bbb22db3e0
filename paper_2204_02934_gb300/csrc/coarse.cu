// coarse.cu -- coarse graph A_c of an aggregation (Section III-C, setup of
// Algorithm 4: one coarse vertex per aggregate, coarse edge A-B whenever a
// fine edge joins a member of A to a member of B, A != B).
//
// No global sort: vertices are bucketed by aggregate (counting sort), then
// each aggregate's neighbour labels are de-duplicated on chip.
//   - Aggregates whose members hold <= kWarpEntries entries: one warp.  A
//     first walk finds the label range and count; a narrow range (<= 4096
//     ids) goes through a shared-memory bitmap read out in order, few
//     entries (<= 1024) through a shared-memory bitonic sort.
//   - Everything else: one block with a global bitmap over all aggregate
//     ids.  Each first-time bit flip appends the label to a discovery list;
//     the list (the coarse row, unordered) is sorted in shared memory when it
//     fits, otherwise the bitmap is read out in order.  Bits are cleared
//     again, so the bitmap stays zero between aggregates.
// Member rows of <= 32 entries are staged lane-per-row with asynchronous
// copies; longer rows are walked by the whole warp.
// Rows land in a scratch buffer at the aggregate's degree-sum offset, then
// are packed behind the prefix sum of the row lengths.
#include <algorithm>

#include "internal.h"
#include "mis_rows.cuh"
#include "scan.cuh"

namespace mis2 {

constexpr int kCoarseWarps = 4;        // warps per block of the warp-per-aggregate kernel
constexpr int kBitmapWords = 128;      // 4096 ids per warp
constexpr int kSortCap = 1024;         // entries per warp
constexpr int kWarpEntries = 8192;     // larger aggregates go to the block kernel
constexpr int kBlockSortCap = 8192;    // discovery lists sorted in shared memory up to this size
static_assert(kBlockSortCap * 4 <= (kBlock / 32) * kStageWarpInt4 * 16, "sort buffer reuses the staging area");

template <typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_hist(GraphView<I> g, const int32_t* labels, int32_t* agg_cnt,
                                                        int32_t* ub) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = lane_id();
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < g.n; base += stride) {
    const int64_t v = base + lane;
    const int32_t a = v < g.n ? labels[v] : -1;
    const unsigned peers = __match_any_sync(kFull, a);
    if (a >= 0) {
      if (lane == __ffs(peers) - 1) atomicAdd(agg_cnt + a, __popc(peers));
      int64_t s, e;
      row_range(g, v, s, e);
      if (e > s) atomicAdd(ub + a, (int32_t)(e - s));
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_coarse_scatter(int64_t n, const int32_t* labels, int32_t* cursor,
                                                           int32_t* members) {
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

// Walk every fine entry of aggregate a (members [mb, me)) with one warp and
// call f(label) for each neighbour label != a.  Warp-uniform; f runs in the
// lane that holds the entry.
template <typename I, typename F>
__device__ __forceinline__ void walk_aggregate(const GraphView<I>& g, const int32_t* labels, const int32_t* members,
                                               int64_t mb, int64_t me, int32_t a, int4* stage_warp, F&& f) {
  const int lane = lane_id();
  int4* my = stage_warp + lane * kStageInt4;
  const int32_t* myw = reinterpret_cast<const int32_t*>(my);
  for (int64_t kb = mb; kb < me; kb += 32) {
    const int64_t k = kb + lane;
    int64_t s = 0, e = 0;
    int off = -1;
    const bool has = k < me;
    if (has) {
      row_range(g, members[k], s, e);
      off = stage_row(g, s, e, my);
    }
    cp_async_wait_all();
    if (off >= 0) {
      const int len = (int)(e - s);
      int32_t lab[kLaneRowMax];
#pragma unroll
      for (int j = 0; j < kLaneRowMax; j++) lab[j] = j < len ? labels[myw[off + j]] : a;
#pragma unroll
      for (int j = 0; j < kLaneRowMax; j++)
        if (lab[j] != a) f(lab[j]);
    }
    unsigned longm = __ballot_sync(kFull, has && off < 0);
    while (longm) {
      const int j = __ffs(longm) - 1;
      longm &= longm - 1;
      const int64_t sj = __shfl_sync(kFull, s, j), ej = __shfl_sync(kFull, e, j);
      visit_row<32>(g.colind, g.nnz, sj, ej, lane, g.vec, [&](int32_t w) {
        const int32_t l = labels[w];
        if (l != a) f(l);
      });
    }
  }
}

template <typename I>
__global__ void __launch_bounds__(kCoarseWarps * 32) k_coarse_rows(
    GraphView<I> g, const int32_t* labels, int64_t n_aggs, const int32_t* agg_ptr, const int32_t* members,
    const int32_t* ub, const int32_t* ub_ptr, int32_t* tmp, int32_t* c_cnt, int32_t* large, int32_t* large_cnt) {
  __shared__ int32_t sbuf[kCoarseWarps][kSortCap];
  __shared__ int4 stage[kCoarseWarps][kStageWarpInt4];
  __shared__ int32_t scnt[kCoarseWarps];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  int32_t* buf = sbuf[wib];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n_aggs; a += nw) {
    if (ub[a] > kWarpEntries) {
      if (lane == 0) large[atomicAdd(large_cnt, 1)] = (int32_t)a;
      continue;
    }
    const int64_t mb = agg_ptr[a], me = agg_ptr[a + 1];
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    int cnt = 0;
    walk_aggregate<I>(g, labels, members, mb, me, (int32_t)a, stage[wib], [&](int32_t l) {
      lo = min(lo, (uint32_t)l);
      hi = max(hi, (uint32_t)l);
      cnt++;
    });
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    cnt = (int)__reduce_add_sync(kFull, (unsigned)cnt);
    const int64_t out = ub_ptr[a];
    if (cnt == 0) {
      if (lane == 0) c_cnt[a] = 0;
      continue;
    }
    if (hi - lo < 32u * kBitmapWords) {
      uint32_t* bm = reinterpret_cast<uint32_t*>(buf);
      for (int j = lane; j < kBitmapWords; j += 32) bm[j] = 0u;
      __syncwarp();
      walk_aggregate<I>(g, labels, members, mb, me, (int32_t)a, stage[wib], [&](int32_t l) {
        const uint32_t d = (uint32_t)l - lo;
        atomicOr(bm + (d >> 5), 1u << (d & 31));
      });
      __syncwarp();
      constexpr int WPL = kBitmapWords / 32;  // words per lane
      uint32_t wv[WPL];
      int pc = 0;
#pragma unroll
      for (int q = 0; q < WPL; q++) {
        wv[q] = bm[lane * WPL + q];
        pc += __popc(wv[q]);
      }
      int incl = pc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      int pos = incl - pc;
#pragma unroll
      for (int q = 0; q < WPL; q++) {
        uint32_t w = wv[q];
        while (w) {
          const int bit = __ffs(w) - 1;
          w &= w - 1;
          tmp[out + pos++] = (int32_t)(lo + (uint32_t)((lane * WPL + q) * 32 + bit));
        }
      }
      const int total = __shfl_sync(kFull, incl, 31);
      if (lane == 0) c_cnt[a] = total;
      __syncwarp();
      continue;
    }
    if (cnt <= kSortCap) {
      if (lane == 0) scnt[wib] = 0;
      __syncwarp();
      walk_aggregate<I>(g, labels, members, mb, me, (int32_t)a, stage[wib],
                        [&](int32_t l) { buf[atomicAdd(scnt + wib, 1)] = l; });
      __syncwarp();
      int P = 32;
      while (P < cnt) P <<= 1;
      for (int i = cnt + lane; i < P; i += 32) buf[i] = 0x7FFFFFFF;
      __syncwarp();
      for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = lane; i < P; i += 32) {
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
          __syncwarp();
        }
      }
      int total = 0;
      for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        const bool keep = i < cnt && (i == 0 || buf[i - 1] != buf[i]);
        const unsigned b = __ballot_sync(kFull, keep);
        if (keep) tmp[out + total + __popc(b & ((1u << lane) - 1u))] = buf[i];
        total += __popc(b);
      }
      if (lane == 0) c_cnt[a] = total;
      __syncwarp();
      continue;
    }
    if (lane == 0) large[atomicAdd(large_cnt, 1)] = (int32_t)a;
  }
}

// Block per large aggregate; `bitmaps` holds one zeroed bitmap of `words`
// words per block.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_large(GraphView<I> g, const int32_t* labels,
                                                         const int32_t* agg_ptr, const int32_t* members,
                                                         const int32_t* ub_ptr, const int32_t* large,
                                                         const int32_t* large_cnt, uint32_t* bitmaps, int64_t words,
                                                         int32_t* tmp, int32_t* c_cnt) {
  __shared__ int4 stage[kBlock / 32][kStageWarpInt4];
  int32_t* sorted = reinterpret_cast<int32_t*>(&stage[0][0]);  // reused once the walk is done
  __shared__ int disc;
  __shared__ int sh[40];
  uint32_t* bm = bitmaps + (int64_t)blockIdx.x * words;
  const int64_t nl = *large_cnt;
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  for (int64_t li = blockIdx.x; li < nl; li += gridDim.x) {
    const int32_t a = large[li];
    const int64_t mb = agg_ptr[a], me = agg_ptr[a + 1];
    const int64_t out = ub_ptr[a];
    if (threadIdx.x == 0) disc = 0;
    __syncthreads();
    // each warp walks a contiguous share of the members
    const int64_t per = (me - mb + (kBlock / 32) - 1) / (kBlock / 32);
    const int64_t w0 = mb + wib * per, w1 = min(me, w0 + per);
    walk_aggregate<I>(g, labels, members, w0, max(w0, w1), a, stage[wib], [&](int32_t l) {
      const uint32_t bit = 1u << (l & 31);
      const uint32_t old = atomicOr(bm + (l >> 5), bit);
      if ((old & bit) == 0u) tmp[out + atomicAdd(&disc, 1)] = l;
    });
    __syncthreads();
    const int D = disc;
    if (D <= kBlockSortCap) {
      int P = 1;
      while (P < D) P <<= 1;
      for (int i = threadIdx.x; i < P; i += blockDim.x) sorted[i] = i < D ? tmp[out + i] : 0x7FFFFFFF;
      __syncthreads();
      for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = threadIdx.x; i < P; i += blockDim.x) {
            const int ixj = i ^ j;
            if (ixj > i) {
              const int32_t x = sorted[i], y = sorted[ixj];
              const bool up = (i & k) == 0;
              if ((x > y) == up) {
                sorted[i] = y;
                sorted[ixj] = x;
              }
            }
          }
          __syncthreads();
        }
      }
      for (int i = threadIdx.x; i < D; i += blockDim.x) {
        const int32_t l = sorted[i];
        tmp[out + i] = l;
        bm[l >> 5] = 0u;  // clear for the next aggregate (idempotent per word)
      }
    } else {
      // read the whole bitmap out in order, clearing it
      int64_t run = 0;
      for (int64_t wb = 0; wb < words; wb += blockDim.x) {
        const int64_t wi = wb + threadIdx.x;
        uint32_t w = wi < words ? bm[wi] : 0u;
        int total;
        int pos = block_exclusive_scan(__popc(w), sh, &total);
        if (w != 0u) bm[wi] = 0u;
        while (w) {
          const int bit = __ffs(w) - 1;
          w &= w - 1;
          tmp[out + run + pos++] = (int32_t)(wi * 32 + bit);
        }
        run += total;
      }
    }
    if (threadIdx.x == 0) c_cnt[a] = D;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kBlock) k_coarse_pack(int64_t n_aggs, const int32_t* ub_ptr, const int32_t* c_cnt,
                                                        const int32_t* c_rowptr, const int32_t* tmp,
                                                        int32_t* c_colind) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n_aggs; a += nw) {
    const int64_t src = ub_ptr[a], dst = c_rowptr[a];
    const int len = c_cnt[a];
    for (int i = lane; i < len; i += 32) c_colind[dst + i] = tmp[src + i];
  }
}

// ------------------------------------------------------------------ host side
int coarse_bitmap_blocks(const mis2_ctx* c) {
  const int64_t words = (std::max<int64_t>(c->max_n, 1) + 31) / 32;
  const int64_t cap = ((int64_t)256 << 20) / (words * 4);
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c->sm_count * 2, cap));
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
  k_coarse_hist<I><<<grid_for(c, n, kBlock), kBlock, 0, st>>>(gv, labels, s.agg_cnt, s.ub);
  c->launches++;
  timer_end(c, st);
  MIS2_TRY(exclusive_scan_i32(c, s.agg_cnt, n_aggs, s.agg_ptr, nullptr, st));
  MIS2_TRY(exclusive_scan_i32(c, s.ub, n_aggs, s.ub_ptr, nullptr, st));
  timer_begin(c, kKcCoarse, st);
  MIS2_CUDA(cudaMemcpyAsync(s.cursor, s.agg_ptr, n_aggs * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  k_coarse_scatter<<<grid_for(c, n, kBlock), kBlock, 0, st>>>(n, labels, s.cursor, s.members);
  const int blocks = grid_for(c, n_aggs, kCoarseWarps, 16);
  k_coarse_rows<I><<<blocks, kCoarseWarps * 32, 0, st>>>(gv, labels, n_aggs, s.agg_ptr, s.members, s.ub, s.ub_ptr,
                                                         s.tmp, s.c_cnt, s.large, s.ctr + kCtrLarge);
  const int64_t words = (n_aggs + 31) / 32;
  const int nb = coarse_bitmap_blocks(c);
  MIS2_CUDA(cudaMemsetAsync(s.bitmaps, 0, (size_t)nb * words * sizeof(uint32_t), st));
  k_coarse_large<I><<<nb, kBlock, 0, st>>>(gv, labels, s.agg_ptr, s.members, s.ub_ptr, s.large, s.ctr + kCtrLarge,
                                           s.bitmaps, words, s.tmp, s.c_cnt);
  c->launches += 3;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  MIS2_TRY(exclusive_scan_i32(c, s.c_cnt, n_aggs, c_rowptr, s.ctr + kCtrCnnz, st));
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  const int64_t total = c->h_ctr[kCtrCnnz];
  if (total > c_colind_cap) return MIS2_ERR_INVALID_ARG;
  timer_begin(c, kKcCoarse, st);
  k_coarse_pack<<<grid_for(c, n_aggs, kBlock / 32, 8), kBlock, 0, st>>>(n_aggs, s.ub_ptr, s.c_cnt, c_rowptr, s.tmp,
                                                                        c_colind);
  c->launches++;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  *c_nnz = total;
  return MIS2_OK;
}

int coarsen_impl(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, int64_t n_aggs, int32_t* c_rowptr,
                 int32_t* c_colind, int64_t c_colind_cap, int64_t* c_nnz, cudaStream_t st) {
  return g.rp64 ? coarsen_t<int64_t>(c, g, labels, n_aggs, c_rowptr, c_colind, c_colind_cap, c_nnz, st)
                : coarsen_t<int32_t>(c, g, labels, n_aggs, c_rowptr, c_colind, c_colind_cap, c_nnz, st);
}

}  // namespace mis2
