// teams.cuh -- walks for the host-driven round kernels (distance-k MIS, the
// colouring) over rows split by length: a warp picks, 32 vertices at a time,
// the ones still in play and hands them to its G-lane groups; listed medium
// and heavy rows go to a "team" of TPR threads (a warp or the whole block)
// each, with the team reductions below.
#pragma once

#include "common.cuh"

namespace mis2 {

// Every warp of the grid walks [0, n) 32 vertices at a time; the vertices
// with pick(v) go to the warp's G-lane groups, 32 / G at a time.  body(v)
// runs on every lane of the warp in step (v = -1 for an idle group), so it
// may use warp-wide collectives.  PACK false: no packing, each group takes
// the next vertex in turn (more warps in flight when n is small).
template <int G, bool PACK, class Pick, class Body>
__device__ __forceinline__ void for_picked(int64_t n, Pick&& pick, Body&& body) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), sub = lane / G;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if constexpr (!PACK) {
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW; base < n;
         base += nw * RPW) {
      const int64_t v = base + sub;
      body(v < n && pick(v) ? v : (int64_t)-1);
    }
  } else {
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += nw * 32) {
      const int64_t vl = base + lane;
      unsigned mask = __ballot_sync(kFull, vl < n && pick(vl));
      while (mask != 0u) {  // warp-uniform
        unsigned mm = mask;
        for (int i = 0; i < sub; i++) mm &= mm - 1u;
        const int64_t v = mm != 0u ? base + __ffs(mm) - 1 : -1;
#pragma unroll
        for (int i = 0; i < RPW; i++) mask &= mask - 1u;
        body(v);
      }
    }
  }
}

// Team reductions: TPR = 32 (a warp) or kBlock (the block; `sh` holds 33
// words and every thread of the block calls).
template <int TPR>
__device__ __forceinline__ bool team_any(bool p) {
  if constexpr (TPR == 32) return __any_sync(kFull, p);
  else return __syncthreads_or(p) != 0;
}

template <int TPR>
__device__ __forceinline__ uint32_t team_min(uint32_t x, uint32_t* sh) {
  if constexpr (TPR == 32) return __reduce_min_sync(kFull, x);
  else return block_min_u32(x, sh);
}

template <int TPR>
__device__ __forceinline__ uint32_t team_or(uint32_t x, uint32_t* sh) {
  x = __reduce_or_sync(kFull, x);
  if constexpr (TPR == 32) {
    return x;
  } else {
    if (threadIdx.x == 0) sh[32] = 0u;
    __syncthreads();
    if (lane_id() == 0 && x != 0u) atomicOr(sh + 32, x);
    __syncthreads();
    const uint32_t r = sh[32];
    __syncthreads();
    return r;
  }
}

// The team's place in the grid: rank of the thread in its team, the team's
// index and the number of teams.
template <int TPR>
struct Team {
  int tid;
  int64_t index, count;
  __device__ __forceinline__ Team() {
    constexpr int per_block = kBlock / TPR;
    tid = TPR == 32 ? lane_id() : (int)threadIdx.x;
    index = (int64_t)blockIdx.x * per_block + (TPR == 32 ? (threadIdx.x >> 5) : 0);
    count = (int64_t)gridDim.x * per_block;
  }
};

}  // namespace mis2
