// scan.cuh -- ordered (stable) compaction and exclusive prefix sums over
// large index ranges: per-tile counts, then a per-tile rewrite.  Up to
// kScanDirectTiles tiles, each tile's block of the rewrite adds up the counts
// of the tiles before it itself (two launches); above that a one-block scan
// of the tile counts runs in between (three).  Used for the root list
// (ascending vertex ids), the phase-2 root ranking and the CSR row pointers
// of the coarse graph.
#pragma once

#include "common.cuh"

namespace mis2 {

constexpr int kScanIpt = 8;                    // items per thread
constexpr int kScanTile = kBlock * kScanIpt;   // items per tile

constexpr int64_t kScanDirectTiles = 4096;   // 8.4 M items

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

// Pred: struct with `__device__ bool operator()(int64_t i) const`.
template <class Pred>
__global__ void __launch_bounds__(kBlock) k_tile_count(int64_t n, Pred pred, int32_t* tile_cnt) {
  pdl_enter();
  __shared__ int sh[40];
  for (int64_t tile = blockIdx.x; tile * kScanTile < n; tile += gridDim.x) {
    int c = 0;
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanIpt;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + k;
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
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanIpt;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + k;
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
  for (int64_t tile = blockIdx.x; tile * kScanTile < n; tile += gridDim.x) {
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanIpt;
    bool keep[kScanIpt];
    int c = 0;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + k;
      keep[k] = i < n && pred(i);
      c += keep[k];
    }
    const int off = tile_offset(tile_off, tile, direct, sh);
    int total;
    int pos = block_exclusive_scan(c, sh, &total) + off;
    if (direct && total_out != nullptr && threadIdx.x == 0 && (tile + 1) * kScanTile >= n) *total_out = off + total;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + k;
      if (i < n) {
        emit(i, pos, keep[k]);
        pos += keep[k];
      }
    }
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
  for (int64_t tile = blockIdx.x; tile * kScanTile < n; tile += gridDim.x) {
    const int64_t base = tile * kScanTile + (int64_t)threadIdx.x * kScanIpt;
    int v[kScanIpt];
    int c = 0;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + k;
      v[k] = i < n ? val(i) : 0;
      c += v[k];
    }
    const int off = tile_offset(tile_off, tile, direct, sh);
    int total;
    int pos = block_exclusive_scan(c, sh, &total) + off;
    if (direct && total_out != nullptr && threadIdx.x == 0 && (tile + 1) * kScanTile >= n) *total_out = off + total;
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + k;
      if (i < n) {
        out[i] = (O)pos;
        if (out2 != nullptr) out2[i] = (O)pos;
      }
      pos += v[k];
    }
    if (base <= n - 1 && n - 1 < base + kScanIpt) out[n] = (O)pos;  // thread holding the last item
  }
}

}  // namespace mis2
