// grid_sync.cuh -- what the persistent cooperative kernels (the MIS-2 round
// loop, the colouring round loop) need to separate their phases: a bounded
// grid-wide barrier and the acquire / release / volatile accesses around it.
#pragma once

#include "internal.h"

namespace mis2 {

__device__ __forceinline__ int ld_acquire_i32(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_i32(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int32_t* p) { return *reinterpret_cast<const volatile int32_t*>(p); }
__device__ __forceinline__ int64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (int64_t)t;
}

// Grid barrier on a monotonic arrival counter: the k-th barrier of a launch
// (epoch k, counted by every block) completes when the counter reaches
// base + k * gridDim.x, base being the counter's value when the launch
// started (0 after a reset; the caller passes it, since blocks that start
// late cannot read it from the counter).  Each block adds 1 after a fence and polls with
// acquire loads; there is no reset step on the critical path.
// Returns false (in every thread of the block) when this block gave up
// waiting or another block already reported a timeout.
// ts (optional): ts[0] = latest arrival time, ts[1] = block 0's departure
// time (globaltimer, ns).
__device__ __forceinline__ bool grid_barrier(int32_t* count, int32_t& epoch, int32_t* err, int64_t spin_limit,
                                             int64_t* ts = nullptr, int32_t extra = 0, uint32_t base = 0u) {
  __shared__ int ok;
  __syncthreads();
  epoch++;
  if (threadIdx.x == 0) {
    ok = 1;
    if (ts != nullptr) atomicMax(reinterpret_cast<unsigned long long*>(ts), (unsigned long long)global_ns());
    __threadfence();
    atomicAdd(count, 1);
    const uint32_t target = base + (uint32_t)epoch * gridDim.x + (uint32_t)extra;
    int64_t spins = 0;
    while ((int32_t)((uint32_t)ld_acquire_i32(count) - target) < 0) {
      if (++spins > spin_limit || (ld_volatile_i32(err) & kErrTimeout)) {
        atomicOr(err, kErrTimeout);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    if (ts != nullptr && blockIdx.x == 0) ts[1] = global_ns();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace mis2
