// coarse.cu -- coarse graph A_c of an aggregation (Section III-C, setup of
// Algorithm 4: one coarse vertex per aggregate, coarse edge A-B whenever a
// fine edge joins a member of A to a member of B, A != B).
//
// No global sort: vertices are bucketed by aggregate (counting sort), then
// each aggregate's neighbour labels are de-duplicated on chip:
//   - narrow label range (<= 4096 ids): a per-warp bitmap, read out in order;
//   - few entries (<= 1024): a per-warp bitonic sort in shared memory;
//   - otherwise: a block walks the label range in 32768-bit windows.
// Rows land in a scratch buffer at the aggregate's degree-sum offset, then
// are packed behind the prefix sum of the row lengths.
#include <algorithm>

#include "internal.h"
#include "scan.cuh"

namespace mis2 {

constexpr int kBitmapWords = 128;    // 4096 ids per warp
constexpr int kSortCap = 1024;       // entries per warp
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr int kLargeWords = 1024;    // 32768 ids per block window

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

// Walk every fine entry of aggregate a's members with G lanes per member
// row; f(label) is called for neighbour labels != a.  Warp-uniform.
template <int G, typename I, typename F>
__device__ __forceinline__ void walk_aggregate(const GraphView<I>& g, const int32_t* labels, const int32_t* members,
                                               int64_t mb, int64_t me, int32_t a, F&& f) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  for (int64_t kb = mb; kb < me; kb += RPW) {
    const int64_t k = kb + sub;
    if (k < me) {
      const int32_t u = members[k];
      int64_t s, e;
      row_range(g, u, s, e);
      visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) {
        const int32_t l = labels[w];
        if (l != a) f(l);
      });
    }
  }
}

template <int G, typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_rows(GraphView<I> g, const int32_t* labels, int64_t n_aggs,
                                                        const int32_t* agg_ptr, const int32_t* members,
                                                        const int32_t* ub_ptr, int32_t* tmp, int32_t* c_cnt,
                                                        int32_t* lo_arr, int32_t* hi_arr, int32_t* large,
                                                        int32_t* large_cnt) {
  __shared__ int32_t sbuf[kWarpsPerBlock][kSortCap];
  __shared__ int32_t scnt[kWarpsPerBlock];
  const int lane = lane_id(), wib = threadIdx.x >> 5;
  int32_t* buf = sbuf[wib];
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; a < n_aggs; a += nw) {
    const int64_t mb = agg_ptr[a], me = agg_ptr[a + 1];
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    int cnt = 0;
    walk_aggregate<G, I>(g, labels, members, mb, me, (int32_t)a, [&](int32_t l) {
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
      walk_aggregate<G, I>(g, labels, members, mb, me, (int32_t)a, [&](int32_t l) {
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
      walk_aggregate<G, I>(g, labels, members, mb, me, (int32_t)a, [&](int32_t l) {
        buf[atomicAdd(scnt + wib, 1)] = l;
      });
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
    if (lane == 0) {
      lo_arr[a] = (int32_t)lo;
      hi_arr[a] = (int32_t)hi;
      large[atomicAdd(large_cnt, 1)] = (int32_t)a;
    }
  }
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_large(GraphView<I> g, const int32_t* labels,
                                                         const int32_t* agg_ptr, const int32_t* members,
                                                         const int32_t* ub_ptr, const int32_t* lo_arr,
                                                         const int32_t* hi_arr, const int32_t* large,
                                                         const int32_t* large_cnt, int32_t* tmp, int32_t* c_cnt) {
  __shared__ uint32_t bm[kLargeWords];
  __shared__ int sh[40];
  const int64_t nl = *large_cnt;
  constexpr int WPT = kLargeWords / kBlock;  // words per thread
  for (int64_t li = blockIdx.x; li < nl; li += gridDim.x) {
    const int32_t a = large[li];
    const int64_t mb = agg_ptr[a], me = agg_ptr[a + 1];
    const int64_t lo = lo_arr[a], hi = hi_arr[a];
    const int64_t out = ub_ptr[a];
    int64_t run = 0;
    for (int64_t wb = lo; wb <= hi; wb += 32 * kLargeWords) {
      for (int j = threadIdx.x; j < kLargeWords; j += blockDim.x) bm[j] = 0u;
      __syncthreads();
      // each warp takes every 8th member row
      const int lane = lane_id(), wib = threadIdx.x >> 5;
      for (int64_t k = mb + wib; k < me; k += kWarpsPerBlock) {
        const int32_t u = members[k];
        int64_t s, e;
        row_range(g, u, s, e);
        visit_row<32>(g.colind, g.nnz, s, e, lane, g.vec, [&](int32_t w) {
          const int32_t l = labels[w];
          if (l != a && l >= wb && l < wb + 32 * kLargeWords) {
            const int64_t d = l - wb;
            atomicOr(bm + (d >> 5), 1u << (d & 31));
          }
        });
      }
      __syncthreads();
      uint32_t wv[WPT];
      int pc = 0;
#pragma unroll
      for (int q = 0; q < WPT; q++) {
        wv[q] = bm[threadIdx.x * WPT + q];
        pc += __popc(wv[q]);
      }
      int total;
      int pos = block_exclusive_scan(pc, sh, &total);
#pragma unroll
      for (int q = 0; q < WPT; q++) {
        uint32_t w = wv[q];
        while (w) {
          const int bit = __ffs(w) - 1;
          w &= w - 1;
          tmp[out + run + pos++] = (int32_t)(wb + (int64_t)(threadIdx.x * WPT + q) * 32 + bit);
        }
      }
      run += total;
      __syncthreads();
    }
    if (threadIdx.x == 0) c_cnt[a] = (int32_t)run;
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
  const int G = pick_group_lanes(c, g);
  const int blocks = grid_for(c, n_aggs, kWarpsPerBlock, 8);
#define MIS2_CR(GG)                                                                                           \
  k_coarse_rows<GG, I><<<blocks, kBlock, 0, st>>>(gv, labels, n_aggs, s.agg_ptr, s.members, s.ub_ptr, s.tmp, \
                                                  s.c_cnt, s.lo, s.hi, s.large, s.ctr + kCtrLarge)
  switch (G) {
    case 1: MIS2_CR(1); break;
    case 2: MIS2_CR(2); break;
    case 4: MIS2_CR(4); break;
    case 8: MIS2_CR(8); break;
    case 16: MIS2_CR(16); break;
    default: MIS2_CR(32); break;
  }
#undef MIS2_CR
  k_coarse_large<I><<<c->sm_count * 2, kBlock, 0, st>>>(gv, labels, s.agg_ptr, s.members, s.ub_ptr, s.lo, s.hi,
                                                         s.large, s.ctr + kCtrLarge, s.tmp, s.c_cnt);
  c->launches += 3;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  MIS2_TRY(exclusive_scan_i32(c, s.c_cnt, n_aggs, c_rowptr, s.ctr + kCtrCnnz, st));
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  const int64_t total = c->h_ctr[kCtrCnnz];
  if (total > c_colind_cap) return MIS2_ERR_INVALID_ARG;
  timer_begin(c, kKcCoarse, st);
  k_coarse_pack<<<grid_for(c, n_aggs, kWarpsPerBlock, 8), kBlock, 0, st>>>(n_aggs, s.ub_ptr, s.c_cnt, c_rowptr,
                                                                            s.tmp, c_colind);
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
