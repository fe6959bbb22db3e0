// misk.cu -- distance-k maximal independent sets, the generalisation of
// Algorithm 1 (Section II: distance-k independence; Section III-A: each
// column step spreads statuses one hop, decide reads one more).  Every round
// spreads two quantities hop by hop over closed neighbourhoods:
//   B(j)_v  some IN vertex within distance j of v,
//   P(j)_v  the smallest undecided tuple within distance j of v (OUT if none),
// from B(0)_v = [T_v = IN], P(0)_v = T_v for undecided v (else OUT); an
// undecided v then becomes OUT if B(k)_v, IN if P(k)_v = T_v, and keeps
// competing otherwise with a fresh tuple.  For k = 2 this is Algorithm 1.
// Host-driven rounds: one refresh kernel, k - 1 spreads and a decide (the
// k-th hop fused with the decision, for the undecided vertices only) per
// round, then one count read.  Rows are split by length: short ones get G
// lanes each, medium ones a warp and long ones (hubs) a block, so that one
// long row does not hold a warp for the whole round.
#include <algorithm>

#include "internal.h"
#include "teams.cuh"

namespace mis2 {

namespace {

constexpr int64_t kMiskHeavy = 2048;

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

// One hop over the short rows: B_out = OR of B_in over N[v], P_out = min of
// P_in over N[v]; G lanes per row.  Longer rows get their own values only
// (the list kernels, run next, overwrite them).
template <int G, typename I>
__global__ void __launch_bounds__(kBlock) k_misk_spread(GraphView<I> g, int64_t light_max, const uint8_t* Bi,
                                                        const uint32_t* Pi, uint8_t* Bo, uint32_t* Po) {
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
      if (e - s <= light_max)
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

// The k-th hop fused with the decision, short rows, undecided vertices only:
// v becomes OUT if B(k)_v, IN if P(k)_v = T_v.  Counts the vertices still
// undecided.
template <int G, bool PACK, typename I>
__global__ void __launch_bounds__(kBlock) k_misk_decide(GraphView<I> g, int64_t light_max, uint32_t* T,
                                                        const uint8_t* Bi, const uint32_t* Pi, int32_t* undecided) {
  const int lg = lane_id() & (G - 1);
  int32_t left = 0;
  for_picked<G, PACK>(
      g.n,
      [&](int64_t v) {
        const uint32_t t = T[v];
        return t != kIn && t != kOut;
      },
      [&](int64_t v) {
        bool active = v >= 0;
        int64_t s = 0, e = 0;
        uint32_t t = 0;
        if (active) {
          row_range(g, v, s, e);
          active = e - s <= light_max;
          t = T[v];
        }
        bool bl = false;
        uint32_t m = kOut;
        if (active) {
          if (lg == 0) {
            bl = Bi[v] != 0;
            m = Pi[v];
          }
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
      });
  left = (int32_t)__reduce_add_sync(kFull, (unsigned)left);
  if (lane_id() == 0 && left > 0) atomicAdd(undecided, left);
}

// The listed (medium or heavy) rows, a team of TPR threads each: one hop
// (DECIDE false) or the fused last hop and decision (DECIDE true, undecided
// vertices only).
template <int TPR, bool DECIDE, typename I>
__global__ void __launch_bounds__(kBlock) k_misk_list(GraphView<I> g, const int32_t* list, const int32_t* n_list,
                                                      const uint8_t* Bi, const uint32_t* Pi, uint8_t* Bo,
                                                      uint32_t* Po, uint32_t* T, int32_t* undecided) {
  __shared__ uint32_t sh[33];
  const Team<TPR> tm;
  const int32_t nl = block_load(n_list);
  int32_t left = 0;
  for (int64_t j = tm.index; j < nl; j += tm.count) {  // team-uniform
    const int32_t v = list[j];
    uint32_t t = 0;
    if (DECIDE) {
      t = T[v];
      if (t == kIn || t == kOut) continue;  // team-uniform: only this team writes T[v]
    }
    int64_t s, e;
    row_range(g, v, s, e);
    bool bl = false;
    uint32_t m = kOut;
    for (int64_t k = s + tm.tid; k < e; k += TPR) {
      const int32_t w = __ldg(g.colind + k);
      bl |= Bi[w] != 0;
      m = min(m, Pi[w]);
    }
    bl = team_any<TPR>(bl);
    m = team_min<TPR>(m, sh);
    if (tm.tid == 0) {
      bl |= Bi[v] != 0;
      m = min(m, Pi[v]);
      if (DECIDE) {
        if (bl) T[v] = kOut;
        else if (m == t) T[v] = kIn;
        else left++;
      } else {
        Bo[v] = (uint8_t)bl;
        Po[v] = m;
      }
    }
  }
  if (DECIDE) {
    left = (int32_t)__reduce_add_sync(kFull, (unsigned)left);
    if (lane_id() == 0 && left > 0) atomicAdd(undecided, left);
  }
}

template <int G, typename I>
int misk_rounds_t(mis2_ctx* c, const GraphView<I>& gv, const GraphArgs& ga, int k, const PrioCfg& p,
                  cudaStream_t st, int32_t* rounds) {
  Scratch& s = c->s;
  const int64_t light_max = G == 32 ? kMiskHeavy : 64;
  LenLists rl;
  MIS2_TRY(classify_rows(c, ga, light_max, kMiskHeavy, &rl, st));
  // hop buffers (after the classification, which borrows qflag and aggsize)
  uint32_t* P[2] = {s.M, reinterpret_cast<uint32_t*>(s.tent)};
  uint8_t* B[2] = {s.qflag, reinterpret_cast<uint8_t*>(s.aggsize)};
  int32_t* cnt = s.ctr + kCtrRoots;  // undecided count of the round
  const int rb = grid_for(c, gv.n, kBlock);
  const int wb = grid_for(c, gv.n, kBlock / 32 * (32 / G));
  // the decide's packed walk (a warp per 32 vertices) once the graph fills the machine
  const bool pack = gv.n > (int64_t)c->sm_count * 2048;
  const int pb = pack ? grid_for(c, gv.n, kBlock) : wb;
  const int mb = rl.n_medium > 0 ? grid_for(c, rl.n_medium, kBlock / 32) : 0;
  const int hb = rl.n_heavy > 0 ? (int)std::min<int64_t>(rl.n_heavy, (int64_t)c->sm_count * 8) : 0;
  int r = 0;
  for (;; r++) {
    if (r > gv.n) return MIS2_ERR_NO_PROGRESS;
    k_misk_refresh<<<rb, kBlock, 0, st>>>(gv.n, s.T, p, (uint32_t)r, B[0], P[0]);
    c->launches++;
    int cur = 0;
    for (int j = 1; j <= k - 1; j++, cur ^= 1) {
      k_misk_spread<G, I><<<wb, kBlock, 0, st>>>(gv, light_max, B[cur], P[cur], B[cur ^ 1], P[cur ^ 1]);
      c->launches++;
      if (mb > 0) {
        k_misk_list<32, false, I><<<mb, kBlock, 0, st>>>(gv, rl.medium, rl.n_medium_dev, B[cur], P[cur], B[cur ^ 1],
                                                          P[cur ^ 1], nullptr, nullptr);
        c->launches++;
      }
      if (hb > 0) {
        k_misk_list<kBlock, false, I><<<hb, kBlock, 0, st>>>(gv, rl.heavy, rl.n_heavy_dev, B[cur], P[cur],
                                                              B[cur ^ 1], P[cur ^ 1], nullptr, nullptr);
        c->launches++;
      }
    }
    MIS2_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t), st));
    if (pack) k_misk_decide<G, true, I><<<pb, kBlock, 0, st>>>(gv, light_max, s.T, B[cur], P[cur], cnt);
    else k_misk_decide<G, false, I><<<pb, kBlock, 0, st>>>(gv, light_max, s.T, B[cur], P[cur], cnt);
    c->launches++;
    if (mb > 0) {
      k_misk_list<32, true, I><<<mb, kBlock, 0, st>>>(gv, rl.medium, rl.n_medium_dev, B[cur], P[cur], nullptr,
                                                       nullptr, s.T, cnt);
      c->launches++;
    }
    if (hb > 0) {
      k_misk_list<kBlock, true, I><<<hb, kBlock, 0, st>>>(gv, rl.heavy, rl.n_heavy_dev, B[cur], P[cur], nullptr,
                                                           nullptr, s.T, cnt);
      c->launches++;
    }
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
  return avg < 40.0 ? misk_rounds_t<4, I>(c, gv, g, k, p, st, rounds)
                    : misk_rounds_t<32, I>(c, gv, g, k, p, st, rounds);
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
