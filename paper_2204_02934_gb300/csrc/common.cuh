// common.cuh -- device-side building blocks shared by the MIS-2, aggregation
// and coarse-graph kernels: the packed status tuple, the priority hash, CSR
// row traversal by a group of lanes, group/warp/block reductions and
// warp-aggregated worklist appends.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mis2.h"

namespace mis2 {

constexpr uint32_t kIn = 0u;            // Section V-C: IN is the smallest tuple
constexpr uint32_t kOut = 0xFFFFFFFFu;  // and OUT the largest
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kClasses = 3;             // row classes: 0 group, 1 warp, 2 block
constexpr int kBlock = 256;             // threads of every row kernel

// ----------------------------------------------------------------- priorities
// f = xorshift64* (Vigna, ACM TOMS 2016: xorshift triple 12/25/27, then a
// multiply by 0x2545F4914F6CDD1D); the Table I ablation also offers plain
// xorshift: the same xorshift stage without the multiply (Section V-A calls
// xorshift* xorshift followed by a linear congruential step).
// h(iter, v) = f(f(iter) ^ f(v) ^ seed) (Section V-A; seed 0 is the paper's
// formula).
__host__ __device__ __forceinline__ uint64_t xorshift_star64(uint64_t x) {
  x ^= x >> 12;
  x ^= x << 25;
  x ^= x >> 27;
  return x * 0x2545F4914F6CDD1Dull;
}
__host__ __device__ __forceinline__ uint64_t xorshift64(uint64_t x) {
  x ^= x >> 12;
  x ^= x << 25;
  x ^= x >> 27;
  return x;
}

// Everything a kernel needs to build T_v for a round.  For a batch of
// graphs stored as one block-diagonal union, gid maps a union vertex to its
// graph, whose own id bits and first union vertex give the tuple that graph
// would get on its own (tuples are only ever compared inside one graph).
struct PrioCfg {
  uint64_t seed;
  const uint32_t* table;  // test hook (Fig. 1): per-round priorities, or null
  int64_t table_n;        // row length of the table
  const int32_t* gid;     // batch: graph of each union vertex, or null
  const int64_t* voff;    // batch: first union vertex of each graph
  const int32_t* gbits;   // batch: id bits of each graph
  int32_t table_rounds;
  int32_t b;              // id bits, b = ceil(log2(n + 2))
  int32_t variant;        // MIS2_HASH_*
  int32_t pad;
};

// Section V-C, Eq. 1: (priority << b) | (v + 1) evaluated in the 32-bit
// status word, the priority being the hash truncated to 32 bits: its low
// 32 - b bits survive the shift.  2^b >= n + 2 keeps the result away from
// IN (0) and OUT.
__device__ __forceinline__ uint32_t make_tuple(const PrioCfg& p, uint32_t iter, uint32_t v) {
  uint32_t prio;
  int b = p.b;
  if (p.gid != nullptr) {
    const int32_t g = p.gid[v];
    v -= (uint32_t)p.voff[g];
    b = p.gbits[g];
  }
  if (p.table != nullptr && (int32_t)iter < p.table_rounds) {
    prio = p.table[(int64_t)iter * p.table_n + v];
  } else {
    uint64_t h;
    if (p.variant == MIS2_HASH_XORSHIFT) {
      h = xorshift64(xorshift64((uint64_t)iter) ^ xorshift64((uint64_t)v) ^ p.seed);
    } else {
      const uint64_t it = p.variant == MIS2_HASH_FIXED ? 0ull : (uint64_t)iter;
      h = xorshift_star64(xorshift_star64(it) ^ xorshift_star64((uint64_t)v) ^ p.seed);
    }
    prio = (uint32_t)h;
  }
  return (b >= 32 ? 0u : (prio << b)) | (v + 1u);
}

__host__ __device__ inline int id_bits(int64_t n) {
  int b = 0;
  while (((uint64_t)1 << b) < (uint64_t)n + 2u) b++;
  return b;
}

// ----------------------------------------------------------------- graph view
template <typename I>
struct GraphView {
  const I* rowptr;
  const int32_t* colind;
  int64_t n;
  int64_t nnz;
  int32_t vec;  // colind 16-byte aligned: int4 loads allowed
  int32_t pad;
};

template <typename I>
__device__ __forceinline__ void row_range(const GraphView<I>& g, int64_t v, int64_t& s, int64_t& e) {
  s = (int64_t)__ldg(g.rowptr + v);
  e = (int64_t)__ldg(g.rowptr + v + 1);
}

// Loads of arrays written earlier in the same launch (persistent kernels)
// must not take the non-coherent path; standalone kernels may.
template <bool NC, typename T>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

// Visit colind[s, e) with the G lanes of a group (lane lg of the group).
// With `vec`, 16-byte loads start at the aligned-down row start; an int4 is
// only loaded when it lies wholly inside colind[0, nnz).
template <int G, typename F>
__device__ __forceinline__ void visit_row(const int32_t* __restrict__ colind, int64_t nnz, int64_t s,
                                          int64_t e, int lg, bool vec, F&& f) {
  if (vec) {
    for (int64_t p = (s & ~int64_t(3)) + 4 * lg; p < e; p += 4 * G) {
      if (p + 4 <= nnz) {
        const int4 q = __ldg(reinterpret_cast<const int4*>(colind + p));
        if (p >= s) f(q.x);
        if (p + 1 >= s && p + 1 < e) f(q.y);
        if (p + 2 >= s && p + 2 < e) f(q.z);
        if (p + 3 < e) f(q.w);
      } else {
        for (int k = 0; k < 4; k++) {
          const int64_t q = p + k;
          if (q >= s && q < e) f(__ldg(colind + q));
        }
      }
    }
  } else {
    for (int64_t p = s + lg; p < e; p += G) f(__ldg(colind + p));
  }
}

// 16-byte global -> shared copies that bypass L1 (LDGSTS); each thread waits
// for its own copies only.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ----------------------------------------------------------------- reductions
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may be scheduled while the preceding kernel of its stream is
// still running.  pdl_enter() waits until that kernel has completed and its
// writes are visible (it returns at once for a kernel launched without the
// attribute), then lets the next kernel's blocks be scheduled.  Every kernel
// that launch_k starts calls it before touching global memory.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) return kFull;
  else return ((1u << G) - 1u) << (lane_id() & ~(G - 1));
}

template <int G>
__device__ __forceinline__ uint32_t group_min(uint32_t x) {
  if constexpr (G == 32) {
    return __reduce_min_sync(kFull, x);
  } else {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(kFull, x, o));
    return x;
  }
}

template <int G>
__device__ __forceinline__ uint32_t group_max(uint32_t x) {
  if constexpr (G == 32) {
    return __reduce_max_sync(kFull, x);
  } else {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(kFull, x, o));
    return x;
  }
}

template <int G>
__device__ __forceinline__ int group_sum(int x) {
  if constexpr (G == 32) {
    return (int)__reduce_add_sync(kFull, (unsigned)x);
  } else {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
  }
}

template <int G>
__device__ __forceinline__ bool group_any(bool p) {
  const unsigned b = __ballot_sync(kFull, p);
  return (b & group_mask<G>()) != 0u;
}

template <int G>
__device__ __forceinline__ bool group_all(bool p) {
  const unsigned b = __ballot_sync(kFull, p);
  const unsigned m = group_mask<G>();
  return (b & m) == m;
}

// Append v (where want) to list, one atomic per warp; warp order is kept.
// Every lane of the warp must call this.
__device__ __forceinline__ void warp_append(bool want, int32_t v, int32_t* list, int32_t* cnt) {
  const unsigned b = __ballot_sync(kFull, want);
  if (b == 0u) return;
  const int lane = lane_id();
  const int leader = __ffs(b) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(cnt, __popc(b));
  base = __shfl_sync(kFull, base, leader);
  if (want && list != nullptr) list[base + __popc(b & ((1u << lane) - 1u))] = v;
}

// Add x over the warp into *acc with one 64-bit atomic (acc may be null).
// *p read by one thread of the block and shared: one L2 request per block
// where every warp of a large grid would otherwise read the same word.  Every
// thread of the block must call it, in uniform control flow.
__device__ __forceinline__ int32_t block_load(const int32_t* p) {
  __shared__ int32_t v;
  __syncthreads();
  if (threadIdx.x == 0) v = *p;
  __syncthreads();
  return v;
}
__device__ __forceinline__ int64_t block_load(const int64_t* p) {
  __shared__ int64_t v;
  __syncthreads();
  if (threadIdx.x == 0) v = *p;
  __syncthreads();
  return v;
}

__device__ __forceinline__ void warp_accumulate(int64_t x, int64_t* acc) {
  if (acc == nullptr) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  if (lane_id() == 0 && x != 0) atomicAdd(reinterpret_cast<unsigned long long*>(acc), (unsigned long long)x);
}

// Block-wide reductions for kBlock threads; `sh` holds >= 32 words.  They
// end with a barrier, so `sh` may be reused right after.
__device__ __forceinline__ uint32_t block_min_u32(uint32_t x, uint32_t* sh) {
  x = __reduce_min_sync(kFull, x);
  if (lane_id() == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t y = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : kOut;
    y = __reduce_min_sync(kFull, y);
    if (threadIdx.x == 0) sh[32] = y;
  }
  __syncthreads();
  const uint32_t r = sh[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ uint32_t block_max_u32(uint32_t x, uint32_t* sh) {
  x = __reduce_max_sync(kFull, x);
  if (lane_id() == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t y = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0u;
    y = __reduce_max_sync(kFull, y);
    if (threadIdx.x == 0) sh[32] = y;
  }
  __syncthreads();
  const uint32_t r = sh[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int block_sum_i32(int x, int* sh) {
  x = (int)__reduce_add_sync(kFull, (unsigned)x);
  if (lane_id() == 0) sh[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x < 32) {
    int y = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
    y = (int)__reduce_add_sync(kFull, (unsigned)y);
    if (threadIdx.x == 0) sh[32] = y;
  }
  __syncthreads();
  const int r = sh[32];
  __syncthreads();
  return r;
}

// Exclusive block scan of x over kBlock threads; returns the prefix and
// the block total in *total.  Ends with a barrier.
__device__ __forceinline__ int block_exclusive_scan(int x, int* sh, int* total) {
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int w = lane < nw ? sh[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < nw) sh[lane] = wi - w;
    if (lane == nw - 1) sh[32] = wi;
  }
  __syncthreads();
  const int r = sh[warp] + incl - x;
  *total = sh[32];
  __syncthreads();
  return r;
}

// Row class by degree: 0 = group of G lanes, 1 = warp, 2 = block.
__device__ __forceinline__ int row_class(int64_t deg, int32_t warp_degree, int32_t block_degree) {
  return deg >= block_degree ? 2 : (deg >= warp_degree ? 1 : 0);
}

}  // namespace mis2
