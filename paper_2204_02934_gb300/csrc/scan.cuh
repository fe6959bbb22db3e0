// scan.cuh -- ordered (stable) compaction and exclusive prefix sums over
// large index ranges: per-tile counts, one-block scan of the tile counts,
// then a per-tile rewrite.  Used for the root list (ascending vertex ids),
// the phase-2 root ranking and the CSR row pointers of the coarse graph.
#pragma once

#include "common.cuh"

namespace mis2 {

constexpr int kScanIpt = 8;                    // items per thread
constexpr int kScanTile = kBlock * kScanIpt;   // items per tile

inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// Pred: struct with `__device__ bool operator()(int64_t i) const`.
template <class Pred>
__global__ void __launch_bounds__(kBlock) k_tile_count(int64_t n, Pred pred, int32_t* tile_cnt) {
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
template <class Pred, class Emit>
__global__ void __launch_bounds__(kBlock) k_tile_compact(int64_t n, Pred pred, const int32_t* tile_off,
                                                          Emit emit) {
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
    int total;
    int pos = block_exclusive_scan(c, sh, &total) + tile_off[tile];
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
template <class Val, typename O>
__global__ void __launch_bounds__(kBlock) k_tile_scan_write(int64_t n, Val val, const int32_t* tile_off,
                                                             O* out) {
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
    int total;
    int pos = block_exclusive_scan(c, sh, &total) + tile_off[tile];
#pragma unroll
    for (int k = 0; k < kScanIpt; k++) {
      const int64_t i = base + k;
      if (i < n) out[i] = (O)pos;
      pos += v[k];
    }
    if (base <= n - 1 && n - 1 < base + kScanIpt) out[n] = (O)pos;  // thread holding the last item
  }
}

}  // namespace mis2
