// galerkin.cu -- the two pieces a multilevel method takes from an
// aggregation after the coarse graph (Section III-B: residuals are restricted
// to the coarse system and its solution interpolated back): the coarse edge
// weights (how many fine entries join two aggregates: the off-diagonal of
// P^T A P for the 0/1 adjacency and prolongator) and the tentative
// prolongator itself.
#include "internal.h"

namespace mis2 {

namespace {

// Coarse position of the fine entry (u in aggregate a, v in aggregate b):
// binary search for b in the ascending coarse row of a; -1 for an entry
// inside one aggregate; a missing coarse entry sets err.
__device__ __forceinline__ int32_t coarse_pos(int32_t a, int32_t b, const int32_t* c_rowptr, const int32_t* c_colind,
                                              int32_t* err) {
  if (b == a) return -1;
  const int32_t r1 = c_rowptr[a + 1];
  int32_t lo = c_rowptr[a], hi = r1;  // first position with c_colind >= b
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (c_colind[mid] < b) lo = mid + 1;
    else hi = mid;
  }
  if (lo < r1 && c_colind[lo] == b) return lo;
  atomicOr(err, kErrBadGraph);  // not the coarse graph of these labels
  return -1;
}

// Lanes of a warp that hit the same coarse entry add once, together.
__device__ __forceinline__ void add_combined(int32_t pos, int32_t* c_weights) {
  const unsigned peers = __match_any_sync(kFull, pos);
  if (pos >= 0 && (peers & ((1u << lane_id()) - 1u)) == 0) atomicAdd(c_weights + pos, __popc(peers));
}

constexpr int kWeightChunk = 256;  // fine entries per warp task

// chunk_row[c] = the row holding fine entry c * kWeightChunk.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_chunk_rows(GraphView<I> g, int32_t* chunk_row) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += stride) {
    int64_t s, e;
    row_range(g, v, s, e);
    for (int64_t c = (s + kWeightChunk - 1) / kWeightChunk; c * kWeightChunk < e; c++) chunk_row[c] = (int32_t)v;
  }
}

// Warp per chunk of kWeightChunk consecutive fine entries, so that a hub row
// is shared among many warps: every entry (u, v) whose endpoints lie in
// different aggregates adds 1 to its coarse entry.  The row of each entry:
// when the chunk spans at most 32 rows, a binary search over the row ends
// held one per lane (shuffles); else a binary search over rowptr between
// the rows of this chunk's and the next chunk's first entries.  Integer
// atomics: the sums do not depend on the order of the additions.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_weights(GraphView<I> g, const int32_t* chunk_row,
                                                           const int32_t* labels, const int32_t* c_rowptr,
                                                           const int32_t* c_colind, int32_t* c_weights,
                                                           int32_t* err) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_chunks = (g.nnz + kWeightChunk - 1) / kWeightChunk;
  for (int64_t ch = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < n_chunks; ch += nw) {
    const int64_t k0 = ch * kWeightChunk, k1 = min(g.nnz, k0 + kWeightChunk);
    // every entry of the chunk lies in rows u_first .. u_last (u_last may
    // overshoot: rows past the chunk's last entry start at or after k1)
    const int64_t u_first = chunk_row[ch];
    const int64_t u_last = ch + 1 < n_chunks ? chunk_row[ch + 1] : g.n - 1;
    const bool narrow = u_last - u_first < 32;  // warp-uniform
    // narrow: lane l holds the end of row u_first + l, relative to k0
    int32_t end_rel = 0x7FFFFFFF;
    if (narrow && u_first + lane <= u_last) end_rel = (int32_t)((int64_t)__ldg(g.rowptr + u_first + lane + 1) - k0);
    int64_t u = u_first;
    for (int j = lane; j < kWeightChunk; j += 32) {  // warp-uniform trip count
      const int64_t k = k0 + j;
      if (narrow) {
        int pos = 0;  // rows of the chunk ending at or before k
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int32_t x = __shfl_sync(kFull, end_rel, pos + step - 1);
          if (x <= j) pos += step;
        }
        u = u_first + pos;
      } else if (k < k1 && (int64_t)__ldg(g.rowptr + u + 1) <= k) {
        int64_t a = u + 1, b = u_last;  // the last r in (u, u_last] with rowptr[r] <= k
        while (a < b) {
          const int64_t mid = (a + b + 1) >> 1;
          if ((int64_t)__ldg(g.rowptr + mid) <= k) a = mid;
          else b = mid - 1;
        }
        u = a;
      }
      const int32_t pos = k < k1 ? coarse_pos(labels[u], labels[g.colind[k]], c_rowptr, c_colind, err) : -1;
      add_combined(pos, c_weights);
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_agg_sizes(int64_t n, const int32_t* labels, int32_t* size) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) atomicAdd(size + labels[v], 1);
}

// P[v, labels[v]] = 1, or 1/sqrt(|aggregate|) (IEEE double sqrt and
// division, correctly rounded).
__global__ void __launch_bounds__(kBlock) k_prolongator(int64_t n, const int32_t* labels, const int32_t* size,
                                                        int normalize, int32_t* p_rowptr, int32_t* p_colind,
                                                        double* p_values) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
    p_rowptr[v] = (int32_t)v;
    if (v == n) continue;
    const int32_t a = labels[v];
    p_colind[v] = a;
    p_values[v] = normalize ? 1.0 / sqrt((double)size[a]) : 1.0;
  }
}

}  // namespace

int coarse_weights_impl(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const int32_t* c_rowptr,
                        const int32_t* c_colind, int64_t c_nnz, int32_t* c_weights, cudaStream_t st) {
  int32_t* err = c->s.ctr + kCtrErr;
  MIS2_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  if (c_nnz > 0) MIS2_CUDA(cudaMemsetAsync(c_weights, 0, c_nnz * sizeof(int32_t), st));
  if (g.n > 0 && g.nnz > 0) {
    const int64_t n_chunks = (g.nnz + kWeightChunk - 1) / kWeightChunk;  // <= nnz / 256 + 1 words of tmp
    const int blocks = grid_for(c, n_chunks, kBlock / 32);
    int32_t* chunk_row = c->s.tmp;
    GraphView<int32_t> g32;
    GraphView<int64_t> g64;
    if (g.rp64) {
      g64.rowptr = static_cast<const int64_t*>(g.rowptr);
      g64.colind = g.colind;
      g64.n = g.n;
      g64.nnz = g.nnz;
      g64.vec = g.vec ? 1 : 0;
      g64.pad = 0;
      k_chunk_rows<int64_t><<<grid_for(c, g.n, kBlock), kBlock, 0, st>>>(g64, chunk_row);
      k_coarse_weights<int64_t><<<blocks, kBlock, 0, st>>>(g64, chunk_row, labels, c_rowptr, c_colind, c_weights,
                                                           err);
    } else {
      g32.rowptr = static_cast<const int32_t*>(g.rowptr);
      g32.colind = g.colind;
      g32.n = g.n;
      g32.nnz = g.nnz;
      g32.vec = g.vec ? 1 : 0;
      g32.pad = 0;
      k_chunk_rows<int32_t><<<grid_for(c, g.n, kBlock), kBlock, 0, st>>>(g32, chunk_row);
      k_coarse_weights<int32_t><<<blocks, kBlock, 0, st>>>(g32, chunk_row, labels, c_rowptr, c_colind, c_weights,
                                                           err);
    }
    c->launches += 2;
    MIS2_CUDA(cudaGetLastError());
  }
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, c->s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  return (c->h_ctr[kCtrErr] & kErrBadGraph) ? MIS2_ERR_BAD_GRAPH : MIS2_OK;
}

int prolongator_impl(mis2_ctx* c, const int32_t* labels, int64_t n, int64_t n_aggs, int normalize,
                     int32_t* p_rowptr, int32_t* p_colind, double* p_values, cudaStream_t st) {
  int32_t* size = c->s.agg_cnt;  // n + 1 words of scratch
  if (n_aggs > 0) MIS2_CUDA(cudaMemsetAsync(size, 0, n_aggs * sizeof(int32_t), st));
  if (n > 0) {
    k_agg_sizes<<<grid_for(c, n, kBlock), kBlock, 0, st>>>(n, labels, size);
    c->launches++;
  }
  k_prolongator<<<grid_for(c, n + 1, kBlock), kBlock, 0, st>>>(n, labels, size, normalize, p_rowptr, p_colind,
                                                                p_values);
  c->launches++;
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

}  // namespace mis2
