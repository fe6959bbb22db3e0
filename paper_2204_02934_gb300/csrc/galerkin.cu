// galerkin.cu -- the two pieces a multilevel method takes from an
// aggregation after the coarse graph (Section III-B: residuals are restricted
// to the coarse system and its solution interpolated back): the coarse edge
// weights (how many fine entries join two aggregates: the off-diagonal of
// P^T A P for the 0/1 adjacency and prolongator) and the tentative
// prolongator itself.
#include "internal.h"

namespace mis2 {

namespace {

// Warp per fine row u: every entry (u, v) whose endpoints lie in different
// aggregates adds 1 to its coarse entry, found by binary search in the
// ascending coarse row of u's aggregate.  Integer atomics: the sums do not
// depend on the order of the additions.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_coarse_weights(GraphView<I> g, const int32_t* labels,
                                                           const int32_t* c_rowptr, const int32_t* c_colind,
                                                           int32_t* c_weights, int32_t* err) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < g.n; u += nw) {
    const int32_t a = labels[u];
    int64_t s, e;
    row_range(g, u, s, e);
    const int32_t r0 = c_rowptr[a], r1 = c_rowptr[a + 1];
    for (int64_t k = s + lane; k < e; k += 32) {
      const int32_t b = labels[g.colind[k]];
      if (b == a) continue;
      int32_t lo = r0, hi = r1;  // first position with c_colind >= b
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (c_colind[mid] < b) lo = mid + 1;
        else hi = mid;
      }
      if (lo < r1 && c_colind[lo] == b) atomicAdd(c_weights + lo, 1);
      else atomicOr(err, kErrBadGraph);  // not the coarse graph of these labels
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
  if (g.n > 0) {
    const int blocks = grid_for(c, g.n, kBlock / 32);
    GraphView<int32_t> g32;
    GraphView<int64_t> g64;
    if (g.rp64) {
      g64.rowptr = static_cast<const int64_t*>(g.rowptr);
      g64.colind = g.colind;
      g64.n = g.n;
      g64.nnz = g.nnz;
      g64.vec = g.vec ? 1 : 0;
      g64.pad = 0;
      k_coarse_weights<int64_t><<<blocks, kBlock, 0, st>>>(g64, labels, c_rowptr, c_colind, c_weights, err);
    } else {
      g32.rowptr = static_cast<const int32_t*>(g.rowptr);
      g32.colind = g.colind;
      g32.n = g.n;
      g32.nnz = g.nnz;
      g32.vec = g.vec ? 1 : 0;
      g32.pad = 0;
      k_coarse_weights<int32_t><<<blocks, kBlock, 0, st>>>(g32, labels, c_rowptr, c_colind, c_weights, err);
    }
    c->launches++;
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
