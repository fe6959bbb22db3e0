// checks.cu -- input validation of the debug mode (mis2_config.debug_checks):
// the CSR is well formed and symmetric, and roots handed to mis2_aggregate
// form a distance-2 independent set (Section III: no two roots within two
// hops), ascending.  Every check reads the inputs without indexing memory
// by an unchecked value: the row bounds are validated before any row is
// walked, the root ids before any root's row is read.
#include "internal.h"

namespace mis2 {

namespace {

__device__ __forceinline__ uint64_t mix_pair(uint64_t a, uint64_t b) {
  // SplitMix64 finaliser of the ordered pair
  uint64_t z = (a << 32) ^ b ^ 0x9E3779B97F4A7C15ull;
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// rowptr[0] == 0, rowptr[n] == nnz, rowptr non-decreasing.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_check_rowptr(const I* rowptr, int64_t n, int64_t nnz, int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
    const int64_t r = (int64_t)rowptr[v];
    bool bad = (v == 0 && r != 0) || (v == n && r != nnz) || r < 0 || r > nnz;
    if (v < n && (int64_t)rowptr[v + 1] < r) bad = true;
    if (bad) atomicOr(err, kErrBadGraph);
  }
}

// Column indices in [0, n); symmetry through two order-independent sums of a
// hash of every entry (v, w) and of its mirror (w, v): the multisets of
// entries and of mirrored entries agree exactly when the graph is symmetric,
// and then the sums agree; an asymmetric graph makes them differ unless the
// 64-bit hash collides.  Warp per row; rows already validated.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_check_rows(GraphView<I> g, int32_t* err, unsigned long long* sums) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint64_t h_fwd = 0, h_rev = 0;
  bool bad = false;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n; v += nw) {
    int64_t s, e;
    row_range(g, v, s, e);
    for (int64_t k = s + lane; k < e; k += 32) {
      const int32_t w = g.colind[k];
      if (w < 0 || w >= g.n) {
        bad = true;
        continue;
      }
      h_fwd += mix_pair((uint64_t)v, (uint64_t)w);
      h_rev += mix_pair((uint64_t)w, (uint64_t)v);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    h_fwd += __shfl_xor_sync(kFull, h_fwd, o);
    h_rev += __shfl_xor_sync(kFull, h_rev, o);
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(err, kErrBadGraph);
  if (lane == 0) {
    atomicAdd(sums, (unsigned long long)h_fwd);
    atomicAdd(sums + 1, (unsigned long long)h_rev);
  }
}

// Root ids in [0, n) and strictly ascending.
__global__ void __launch_bounds__(kBlock) k_check_root_ids(const int32_t* roots, int64_t n_roots, int64_t n,
                                                           int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_roots; j += stride) {
    const int32_t r = roots[j];
    if (r < 0 || r >= n || (j > 0 && roots[j - 1] >= r)) atomicOr(err, kErrBadGraph);
  }
}

// cnt[u] += 1 for every u in the closed neighbourhood of every root: two
// roots within two hops share a vertex there (or one lies next to the
// other), so some count reaches 2.  Warp per root.
template <typename I>
__global__ void __launch_bounds__(kBlock) k_count_root_balls(GraphView<I> g, const int32_t* roots, int64_t n_roots,
                                                             int32_t* cnt) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n_roots; j += nw) {
    const int32_t r = roots[j];
    int64_t s, e;
    row_range(g, r, s, e);
    if (lane == 0) atomicAdd(cnt + r, 1);
    for (int64_t k = s + lane; k < e; k += 32) {
      const int32_t u = g.colind[k];
      if (u != r) atomicAdd(cnt + u, 1);
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_check_labels(const int32_t* labels, int64_t n, int64_t n_aggs,
                                                         int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    if (labels[v] < 0 || labels[v] >= n_aggs) atomicOr(err, kErrBadGraph);
}

__global__ void __launch_bounds__(kBlock) k_check_counts(const int32_t* cnt, int64_t n, int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) bad |= cnt[v] > 1;
  if (bad) atomicOr(err, kErrBadGraph);
}

template <typename I>
GraphView<I> view(const GraphArgs& g) {
  GraphView<I> v;
  v.rowptr = static_cast<const I*>(g.rowptr);
  v.colind = g.colind;
  v.n = g.n;
  v.nnz = g.nnz;
  v.vec = g.vec ? 1 : 0;
  v.pad = 0;
  return v;
}

int read_err(mis2_ctx* c, cudaStream_t st) {
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, c->s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  return c->h_ctr[kCtrErr] & kErrBadGraph ? MIS2_ERR_BAD_GRAPH : MIS2_OK;
}

}  // namespace

int check_graph(mis2_ctx* c, const GraphArgs& g, cudaStream_t st) {
  Scratch& s = c->s;
  int32_t* err = s.ctr + kCtrErr;
  unsigned long long* sums = reinterpret_cast<unsigned long long*>(s.ctr + kCtrCheckSums);
  MIS2_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(sums, 0, 2 * sizeof(unsigned long long), st));
  const int blocks = grid_for(c, g.n + 1, kBlock);
  if (g.rp64) k_check_rowptr<int64_t><<<blocks, kBlock, 0, st>>>(static_cast<const int64_t*>(g.rowptr), g.n, g.nnz, err);
  else k_check_rowptr<int32_t><<<blocks, kBlock, 0, st>>>(static_cast<const int32_t*>(g.rowptr), g.n, g.nnz, err);
  MIS2_CUDA(cudaGetLastError());
  MIS2_TRY(read_err(c, st));
  if (g.n > 0) {
    const int wb = grid_for(c, g.n, kBlock / 32);
    if (g.rp64) k_check_rows<int64_t><<<wb, kBlock, 0, st>>>(view<int64_t>(g), err, sums);
    else k_check_rows<int32_t><<<wb, kBlock, 0, st>>>(view<int32_t>(g), err, sums);
    MIS2_CUDA(cudaGetLastError());
  }
  MIS2_TRY(read_err(c, st));
  const uint64_t* h = reinterpret_cast<const uint64_t*>(c->h_ctr + kCtrCheckSums);
  if (h[0] != h[1]) return MIS2_ERR_BAD_GRAPH;
  return MIS2_OK;
}

int check_roots(mis2_ctx* c, const GraphArgs& g, const int32_t* roots, int64_t n_roots, cudaStream_t st) {
  Scratch& s = c->s;
  int32_t* err = s.ctr + kCtrErr;
  MIS2_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  if (n_roots == 0) return MIS2_OK;
  k_check_root_ids<<<grid_for(c, n_roots, kBlock), kBlock, 0, st>>>(roots, n_roots, g.n, err);
  MIS2_CUDA(cudaGetLastError());
  MIS2_TRY(read_err(c, st));
  int32_t* cnt = s.aggsize;  // n words, rewritten by aggregation afterwards
  MIS2_CUDA(cudaMemsetAsync(cnt, 0, g.n * sizeof(int32_t), st));
  const int wb = grid_for(c, n_roots, kBlock / 32);
  if (g.rp64) k_count_root_balls<int64_t><<<wb, kBlock, 0, st>>>(view<int64_t>(g), roots, n_roots, cnt);
  else k_count_root_balls<int32_t><<<wb, kBlock, 0, st>>>(view<int32_t>(g), roots, n_roots, cnt);
  k_check_counts<<<grid_for(c, g.n, kBlock), kBlock, 0, st>>>(cnt, g.n, err);
  MIS2_CUDA(cudaGetLastError());
  return read_err(c, st);
}

int check_labels(mis2_ctx* c, const int32_t* labels, int64_t n, int64_t n_aggs, cudaStream_t st) {
  int32_t* err = c->s.ctr + kCtrErr;
  MIS2_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  if (n == 0) return MIS2_OK;
  k_check_labels<<<grid_for(c, n, kBlock), kBlock, 0, st>>>(labels, n, n_aggs, err);
  MIS2_CUDA(cudaGetLastError());
  return read_err(c, st);
}

}  // namespace mis2
