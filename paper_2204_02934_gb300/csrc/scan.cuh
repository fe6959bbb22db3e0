// scan.cuh -- ordered (stable) compaction and exclusive prefix sums over
// large index ranges: per-tile counts, then a per-tile rewrite.  Up to
// kScanDirectTiles tiles, each tile's block of the rewrite adds up the counts
// of the tiles before it itself (two launches); above that a one-block scan
// of the tile counts runs in between (three).  Used for the root list
// (ascending vertex ids), the phase-2 root ranking and the CSR row pointers
// of the coarse graph.  Within a tile, item k of thread t is item
// k * kBlock + t, so that every load and store of the items is coalesced
// across the warp; the order of a tile's items is (k, warp, lane), and the
// rewrite ranks them in that order (a ballot or a warp scan per k, then the
// 64 (k, warp) totals scanned by one warp).
#pragma once

#include "common.cuh"

namespace mis2 {

constexpr int kScanIpt = 8;                    // items per thread
constexpr int kScanTile = kBlock * kScanIpt;   // items per tile

constexpr int64_t kScanDirectTiles = 4096;   // 8.4 M items
constexpr int kScanWarps = kBlock / 32;
static_assert(kScanIpt * kScanWarps == 64, "one warp scans a tile's (k, warp) totals two to a lane");

inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// Offset of tile `tile` in the rewrite: tile_cnt already scanned (three
// launches), or the sum of the raw counts tile_cnt[0, tile) taken by the
// whole block (direct mode).  Every thread of the block must call this.
__device__ __forceinline__ int tile_offset(const int32_t* tile_cnt, int64_t tile, bool direct, int* sh) {
  if (!direct) return tile_cnt[tile];
  int x = 0;
  for (int64_t t = threadIdx.x; t < tile; t += blockDim.x) x += tile_cnt[t];
  return block_sum_i32(x, sh);
}

// In place: wcnt[k * kScanWarps + w] (the count of item k over warp w of one
// tile) becomes the exclusive prefix over the tile's (k, w) order; returns
// the tile total.  Every thread of the block calls it; starts with a barrier
// (the counts' writes are then visible) and ends with one.
__device__ __forceinline__ int tile_warp_offsets(int* wcnt, int* total_sh) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int a = wcnt[lane], b = wcnt[32 + lane];
    int ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ya = __shfl_up_sync(kFull, ia, o), yb = __shfl_up_sync(kFull, ib, o);
      if (lane >= o) {
        ia += ya;
        ib += yb;
      }
    }
    const int ta = __shfl_sync(kFull, ia, 31);
    wcnt[lane] = ia - a;
    wcnt[32 + lane] = ta + ib - b;
    if (lane == 31) *total_sh = ta + ib;
  }
  __syncthreads();
  return *total_sh;
}

// Pred: struct with `__device__ bool operator()(int64_t i) const`.
template <class Pred>
__global__ void __launch_bounds__(kBlock) k_tile_count(int64_t n, Pred pred, int32_t* tile_cnt) {
  pdl_enter();
  __shared__ int sh[40];
  for (int64_t tile = blockIdx.x; tile * kScanTile < n; tile += gridDim.x) {
    int c = 0;
    const int64_t base = tile * kScanTile + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + (int64_t)k * kBlock;
      if (i < n && pred(i)) c++;
    }
    c = block_sum_i32(c, sh);
    if (threadIdx.x == 0) tile_cnt[tile] = c;
  }
}

// Val: struct with `__device__ int operator()(int64_t i) const`.
template <class Val>
__global__ void __launch_bounds__(kBlock) k_tile_sum(int64_t n, Val val, int32_t* tile_cnt) {
  pdl_enter();
  __shared__ int sh[40];
  for (int64_t tile = blockIdx.x; tile * kScanTile < n; tile += gridDim.x) {
    int c = 0;
    const int64_t base = tile * kScanTile + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + (int64_t)k * kBlock;
      if (i < n) c += val(i);
    }
    c = block_sum_i32(c, sh);
    if (threadIdx.x == 0) tile_cnt[tile] = c;
  }
}

// In-place exclusive scan of tile_cnt[0, ntiles) by one block; the grand
// total goes to *total (device) when total is not null.
__global__ void __launch_bounds__(1024) k_scan_tile_counts(int32_t* tile_cnt, int64_t ntiles, int32_t* total);

// Pred as above; Emit: `__device__ void operator()(int64_t i, int32_t pos, bool keep) const`
// is called for every i < n in ascending order of pos among kept items.
// direct: tile_off holds the raw tile counts (see tile_offset), and the
// block of the last tile writes the grand total to *total (when not null).
template <class Pred, class Emit>
__global__ void __launch_bounds__(kBlock) k_tile_compact(int64_t n, Pred pred, const int32_t* tile_off,
                                                          Emit emit, bool direct, int32_t* total_out) {
  pdl_enter();
  __shared__ int sh[40];
  __shared__ int wcnt[kScanIpt * kScanWarps];
  __shared__ int total_sh;
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (int64_t tile = blockIdx.x; tile * kScanTile < n; tile += gridDim.x) {
    const int64_t base = tile * kScanTile + threadIdx.x;
    bool keep[kScanIpt];
    int rank[kScanIpt];
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + (int64_t)k * kBlock;
      keep[k] = i < n && pred(i);
      const unsigned b = __ballot_sync(kFull, keep[k]);
      rank[k] = __popc(b & below);
      if (lane == 0) wcnt[k * kScanWarps + w] = __popc(b);
    }
    const int off = tile_offset(tile_off, tile, direct, sh);
    const int total = tile_warp_offsets(wcnt, &total_sh);
    if (direct && total_out != nullptr && threadIdx.x == 0 && (tile + 1) * kScanTile >= n) *total_out = off + total;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + (int64_t)k * kBlock;
      if (i < n) emit(i, off + wcnt[k * kScanWarps + w] + rank[k], keep[k]);
    }
    __syncthreads();  // wcnt and total_sh are rewritten for the next tile
  }
}

// Exclusive scan of val(i) into out[i] (i < n), with out[n] = total.
// direct and *total_out: as for k_tile_compact; out2 (or null) receives a
// copy of out[0, n).
template <class Val, typename O>
__global__ void __launch_bounds__(kBlock) k_tile_scan_write(int64_t n, Val val, const int32_t* tile_off,
                                                             O* out, O* out2, bool direct, int32_t* total_out) {
  pdl_enter();
  __shared__ int sh[40];
  __shared__ int wcnt[kScanIpt * kScanWarps];
  __shared__ int total_sh;
  const int lane = lane_id(), w = threadIdx.x >> 5;
  for (int64_t tile = blockIdx.x; tile * kScanTile < n; tile += gridDim.x) {
    const int64_t base = tile * kScanTile + threadIdx.x;
    int ex[kScanIpt];  // exclusive prefix of item k within its warp
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + (int64_t)k * kBlock;
      const int v = i < n ? val(i) : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      ex[k] = incl - v;
      if (lane == 31) wcnt[k * kScanWarps + w] = incl;
    }
    const int off = tile_offset(tile_off, tile, direct, sh);
    const int total = tile_warp_offsets(wcnt, &total_sh);
    const bool last = (tile + 1) * kScanTile >= n;
    if (direct && total_out != nullptr && threadIdx.x == 0 && last) *total_out = off + total;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + (int64_t)k * kBlock;
      if (i < n) {
        const int pos = off + wcnt[k * kScanWarps + w] + ex[k];
        out[i] = (O)pos;
        if (out2 != nullptr) out2[i] = (O)pos;
      }
    }
    if (last && threadIdx.x == 0) out[n] = (O)(off + total);
    __syncthreads();  // wcnt and total_sh are rewritten for the next tile
  }
}

}  // namespace mis2
