// misk.cu -- distance-k maximal independent sets, the generalisation of
// Algorithm 1 (Section II: distance-k independence; Section III-A: each
// column step spreads statuses one hop, decide reads one more).  Every round
// spreads two quantities hop by hop over closed neighbourhoods:
//   B(j)_v  some IN vertex within distance j of v,
//   P(j)_v  the smallest undecided tuple within distance j of v (OUT if none),
// from B(0)_v = [T_v = IN], P(0)_v = T_v for undecided v (else OUT); an
// undecided v then becomes OUT if B(k)_v, IN if P(k)_v = T_v, and keeps
// competing otherwise with a fresh tuple.  For k = 2 this is Algorithm 1.
// Host-driven rounds over every vertex (no worklists): one refresh kernel,
// k - 1 spread kernels, one decide kernel and one count read per round.
#include "internal.h"
#include "mis_rows.cuh"

namespace mis2 {

namespace {

// Round refresh (Algorithm 1's row refresh, fused with hop 0): undecided
// vertices (every vertex in round 0) draw h(iter, v).
__global__ void __launch_bounds__(kBlock) k_misk_refresh(int64_t n, uint32_t* T, PrioCfg p, uint32_t iter,
                                                         uint8_t* B0, uint32_t* P0) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    uint32_t t = T[v];
    const bool decided = iter > 0 && (t == kIn || t == kOut);
    if (!decided) {
      t = make_tuple(p, iter, (uint32_t)v);
      T[v] = t;
    }
    B0[v] = (uint8_t)(decided && t == kIn);
    P0[v] = decided ? kOut : t;
  }
}

// One hop: B_out = OR of B_in over N[v], P_out = min of P_in over N[v].
// G lanes per row.
template <int G, typename I>
__global__ void __launch_bounds__(kBlock) k_misk_spread(GraphView<I> g, const uint8_t* Bi, const uint32_t* Pi,
                                                        uint8_t* Bo, uint32_t* Po) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW; base < g.n; base += nw * RPW) {
    const int64_t v = base + sub;
    bool bl = false;
    uint32_t m = kOut;
    if (v < g.n) {
      if (lg == 0) {
        bl = Bi[v] != 0;
        m = Pi[v];
      }
      int64_t s, e;
      row_range(g, v, s, e);
      visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) {
        bl |= Bi[w] != 0;
        m = min(m, Pi[w]);
      });
    }
    bl = group_any<G>(bl);
    m = group_min<G>(m);
    if (v < g.n && lg == 0) {
      Bo[v] = (uint8_t)bl;
      Po[v] = m;
    }
  }
}

// The last hop, as decide: undecided v becomes OUT if B(k)_v, IN if
// P(k)_v = T_v.  Counts the vertices still undecided.
template <int G, typename I>
__global__ void __launch_bounds__(kBlock) k_misk_decide(GraphView<I> g, uint32_t* T, const uint8_t* Bi,
                                                        const uint32_t* Pi, int32_t* undecided) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t left = 0;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW; base < g.n; base += nw * RPW) {
    const int64_t v = base + sub;
    uint32_t t = kIn;
    if (v < g.n) t = T[v];
    const bool active = v < g.n && t != kIn && t != kOut;
    bool bl = false;
    uint32_t m = kOut;
    if (active) {
      if (lg == 0) {
        bl = Bi[v] != 0;
        m = Pi[v];
      }
      int64_t s, e;
      row_range(g, v, s, e);
      visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) {
        bl |= Bi[w] != 0;
        m = min(m, Pi[w]);
      });
    }
    bl = group_any<G>(bl);
    m = group_min<G>(m);
    if (active && lg == 0) {
      if (bl) T[v] = kOut;
      else if (m == t) T[v] = kIn;
      else left++;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) left += __shfl_xor_sync(kFull, left, o);
  if (lane == 0 && left > 0) atomicAdd(undecided, left);
}

template <int G, typename I>
int misk_rounds_t(mis2_ctx* c, const GraphView<I>& gv, int k, const PrioCfg& p, cudaStream_t st, int32_t* rounds) {
  Scratch& s = c->s;
  uint32_t* P[2] = {s.M, reinterpret_cast<uint32_t*>(s.tent)};
  uint8_t* B[2] = {s.qflag, reinterpret_cast<uint8_t*>(s.aggsize)};
  int32_t* cnt = s.ctr + kCtrRoots;  // undecided count of the round
  const int rb = grid_for(c, gv.n, kBlock);
  const int wb = grid_for(c, gv.n, kBlock / 32 * (32 / G));
  int r = 0;
  for (;; r++) {
    if (r > gv.n) return MIS2_ERR_NO_PROGRESS;
    k_misk_refresh<<<rb, kBlock, 0, st>>>(gv.n, s.T, p, (uint32_t)r, B[0], P[0]);
    int cur = 0;
    for (int j = 1; j <= k - 1; j++, cur ^= 1)
      k_misk_spread<G, I><<<wb, kBlock, 0, st>>>(gv, B[cur], P[cur], B[cur ^ 1], P[cur ^ 1]);
    MIS2_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t), st));
    k_misk_decide<G, I><<<wb, kBlock, 0, st>>>(gv, s.T, B[cur], P[cur], cnt);
    c->launches += 1 + k;
    MIS2_CUDA(cudaGetLastError());
    MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    if (c->h_ctr[kCtrRoots] == 0) break;
  }
  *rounds = r + 1;
  return MIS2_OK;
}

template <typename I>
int misk_t(mis2_ctx* c, const GraphArgs& g, int k, const PrioCfg& p, cudaStream_t st, int32_t* rounds) {
  GraphView<I> gv;
  gv.rowptr = static_cast<const I*>(g.rowptr);
  gv.colind = g.colind;
  gv.n = g.n;
  gv.nnz = g.nnz;
  gv.vec = g.vec ? 1 : 0;
  gv.pad = 0;
  const double avg = g.n > 0 ? (double)g.nnz / (double)g.n : 0.0;
  return avg < 40.0 ? misk_rounds_t<4, I>(c, gv, k, p, st, rounds) : misk_rounds_t<32, I>(c, gv, k, p, st, rounds);
}

}  // namespace

int misk_impl(mis2_ctx* c, const GraphArgs& g, int k, const PrioCfg& p, uint8_t* in_set, int32_t* roots,
              int64_t* n_roots, int32_t* n_rounds, cudaStream_t st) {
  int32_t r = 0;
  if (g.n > 0)
    MIS2_TRY(g.rp64 ? misk_t<int64_t>(c, g, k, p, st, &r) : misk_t<int32_t>(c, g, k, p, st, &r));
  MIS2_TRY(extract_in_set(c, g.n, in_set, roots, c->s.ctr + kCtrRoots, st));
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, c->s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  *n_roots = c->h_ctr[kCtrRoots];
  if (n_rounds) *n_rounds = r;
  c->stats.rounds = r;
  c->stats.n_roots = *n_roots;
  return MIS2_OK;
}

}  // namespace mis2
