// group.cu -- stable grouping of the indices 0..n-1 by an integer key in
// [0, n_keys): list holds the indices of key 0, then of key 1, ..., each run
// ascending, and ptr[k] the start of key k's run.  It serves the two lists of
// cluster multicolor Gauss-Seidel (Algorithm 4): the clusters of each colour
// and the fine rows of each cluster.  An LSD radix sort of (key, index)
// pairs, 8 bits a pass; each pass is stable, so the runs stay ascending.
// Per pass: a per-tile digit histogram (digit-major, so one exclusive scan
// gives every (digit, tile) its output offset), then a scatter that ranks
// the items of a tile in index order (warp match on the digit, running
// per-warp digit counters in shared memory).
#include "internal.h"

namespace mis2 {

namespace {

constexpr int kRadix = 256;
constexpr int kRadixIpt = 8;                     // items per thread
constexpr int kRadixTile = kBlock * kRadixIpt;   // items per tile (one block)
constexpr int kWarps = kBlock / 32;
constexpr int kWarpSpan = kRadixTile / kWarps;   // consecutive items of one warp
static_assert(kRadix == kBlock, "one thread per digit in the cross-warp prefix");

__device__ __forceinline__ int digit_of(int32_t key, int shift) { return (int)(((uint32_t)key >> shift) & 255u); }

// cnt[d * n_tiles + t] = number of items of tile t whose digit is d.  With
// n_keys > 0 (first pass) a key outside [0, n_keys) sets err.
__global__ void __launch_bounds__(kBlock) k_radix_count(int64_t n, const int32_t* keys, int shift, int64_t n_tiles,
                                                        int64_t n_keys, int32_t* cnt, int32_t* err) {
  __shared__ int32_t hist[kRadix];
  bool bad = false;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = t * kRadixTile;
#pragma unroll
    for (int k = 0; k < kRadixIpt; k++) {
      const int64_t i = base + (int64_t)k * kBlock + threadIdx.x;
      if (i < n) {
        const int32_t key = keys[i];
        bad |= n_keys > 0 && (key < 0 || key >= n_keys);
        atomicAdd(hist + digit_of(key, shift), 1);
      }
    }
    __syncthreads();
    cnt[(int64_t)threadIdx.x * n_tiles + t] = hist[threadIdx.x];
    __syncthreads();
  }
  if (bad) atomicOr(err, kErrBadGraph);
}

// Stable scatter: item i of tile t with digit d goes to off[d * n_tiles + t]
// plus its rank among the tile's items of digit d that precede it.  vals_in
// null: the value is i itself; keys_out null: keys are not carried on.
__global__ void __launch_bounds__(kBlock) k_radix_scatter(int64_t n, const int32_t* keys_in, const int32_t* vals_in,
                                                          int shift, int64_t n_tiles, const int32_t* off,
                                                          int32_t* keys_out, int32_t* vals_out) {
  __shared__ int32_t wcnt[kWarps][kRadix];
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    for (int d = lane; d < kRadix; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const int64_t base = t * kRadixTile + (int64_t)w * kWarpSpan;
    int dig[kRadixIpt], rank[kRadixIpt];
#pragma unroll
    for (int k = 0; k < kRadixIpt; k++) {
      const int64_t i = base + (int64_t)k * 32 + lane;
      const int d = i < n ? digit_of(keys_in[i], shift) : kRadix;  // tail lanes match only each other
      const unsigned peers = __match_any_sync(kFull, d);
      const int prior = d < kRadix ? wcnt[w][d] : 0;
      dig[k] = d;
      rank[k] = prior + __popc(peers & below);
      __syncwarp();
      if (d < kRadix && (peers & below) == 0) wcnt[w][d] = prior + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // exclusive prefix of the per-warp counts across warps, per digit
    {
      int32_t run = 0;
#pragma unroll
      for (int ww = 0; ww < kWarps; ww++) {
        const int32_t x = wcnt[ww][threadIdx.x];
        wcnt[ww][threadIdx.x] = run;
        run += x;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRadixIpt; k++) {
      const int64_t i = base + (int64_t)k * 32 + lane;
      if (i < n) {
        const int d = dig[k];
        const int64_t pos = (int64_t)off[(int64_t)d * n_tiles + t] + wcnt[w][d] + rank[k];
        vals_out[pos] = vals_in ? vals_in[i] : (int32_t)i;
        if (keys_out) keys_out[pos] = keys_in[i];
      }
    }
    __syncthreads();
  }
}

// ptr[k] = the first position of the sorted keys holding a key >= k (the
// start of key k's run; empty runs included), for k in [0, n_keys].
__global__ void __launch_bounds__(kBlock) k_run_starts(int64_t n, const int32_t* sorted, int64_t n_keys,
                                                       int32_t* ptr) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= n_keys; k += stride) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)sorted[mid] < k) lo = mid + 1;
      else hi = mid;
    }
    ptr[k] = (int32_t)lo;
  }
}

}  // namespace

int64_t group_scratch_words(int64_t n) { return (int64_t)kRadix * ((n + kRadixTile - 1) / kRadixTile) + 1; }

int group_by_key(mis2_ctx* c, const int32_t* keys, int64_t n, int64_t n_keys, int32_t* ptr, int32_t* list,
                 cudaStream_t st) {
  Scratch& s = c->s;
  int32_t* err = s.ctr + kCtrErr;
  MIS2_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  if (n == 0) {
    MIS2_CUDA(cudaMemsetAsync(ptr, 0, (n_keys + 1) * sizeof(int32_t), st));
    return MIS2_OK;
  }
  // the sort: enough 8-bit passes for the largest key
  int bits = 0;
  while (bits < 31 && ((int64_t)1 << bits) < n_keys) bits++;
  const int passes = bits <= 8 ? 1 : (bits + 7) / 8;
  const int64_t n_tiles = (n + kRadixTile - 1) / kRadixTile;
  const int blocks = grid_for(c, n_tiles, 1, 4);
  int32_t* kbuf[2] = {reinterpret_cast<int32_t*>(s.M), s.roots2};
  int32_t* vbuf[2] = {s.tent, s.qlist};
  const int32_t* kin = keys;
  const int32_t* vin = nullptr;
  for (int p = 0; p < passes; p++) {
    int32_t* kout = kbuf[p & 1];
    int32_t* vout = p == passes - 1 ? list : vbuf[p & 1];
    k_radix_count<<<blocks, kBlock, 0, st>>>(n, kin, 8 * p, n_tiles, p == 0 ? n_keys : 0, s.radix, err);
    MIS2_TRY(exclusive_scan_i32(c, s.radix, kRadix * n_tiles, s.radix, nullptr, st));
    k_radix_scatter<<<blocks, kBlock, 0, st>>>(n, kin, vin, 8 * p, n_tiles, s.radix, kout, vout);
    c->launches += 2;
    MIS2_CUDA(cudaGetLastError());
    kin = kout;
    vin = vout;
  }
  // run starts from the sorted keys (no atomics on the keys of big groups)
  k_run_starts<<<grid_for(c, n_keys + 1, kBlock), kBlock, 0, st>>>(n, kin, n_keys, ptr);
  c->launches++;
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

}  // namespace mis2
