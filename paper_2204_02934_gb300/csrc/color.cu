// color.cu -- the colour sets of cluster multicolor Gauss-Seidel (Algorithm
// 4's setup: colorsets = color(A_c) on the coarse graph).  Jones-Plassmann
// rounds with the round-0 tuples of Eq. 1 as fixed priorities: an uncoloured
// vertex whose tuple is smaller than every uncoloured neighbour's takes the
// smallest colour no coloured neighbour holds.  Such vertices are pairwise
// non-adjacent, and each colours after all its smaller-tuple neighbours, so
// the result is the first-fit greedy colouring in ascending tuple order,
// whatever the schedule.  A neighbour coloured in the current round counts as
// uncoloured (round stamps), which keeps every round's decisions on the state
// before the round.  Host-driven rounds; then the vertices of each colour,
// ascending, by a stable grouping on the colour.
#include "internal.h"

namespace mis2 {

namespace {

constexpr int32_t kUncolored = 0x7FFFFFFF;

__global__ void __launch_bounds__(kBlock) k_color_init(int64_t n, PrioCfg p, uint32_t* prio, int32_t* col,
                                                       int32_t* when) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    prio[v] = make_tuple(p, 0u, (uint32_t)v);
    col[v] = -1;
    when[v] = kUncolored;
  }
}

// One Jones-Plassmann round, G lanes per vertex.  A vertex whose neighbours
// use every colour of the first window of 64 looks at the next window.
template <int G, typename I>
__global__ void __launch_bounds__(kBlock) k_color_round(GraphView<I> g, const uint32_t* prio, int32_t* col,
                                                        int32_t* when, int32_t round, int32_t* left,
                                                        int32_t* max_color) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t still = 0;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW; base < g.n; base += nw * RPW) {
    const int64_t v = base + sub;
    const bool active = v < g.n && when[v] == kUncolored;
    int64_t s = 0, e = 0;
    uint32_t pv = 0;
    if (active) {
      row_range(g, v, s, e);
      pv = prio[v];
    }
    // a smaller uncoloured neighbour (coloured this round counts as uncoloured)
    bool blocked = false;
    if (active)
      visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) {
        if (w != v && when[w] >= round && prio[w] < pv) blocked = true;
      });
    blocked = group_any<G>(blocked);
    const bool mine = active && !blocked;
    int32_t c = -1;
    // warp-uniform trip count: every lane takes part in the group reductions
    for (int32_t wbase = 0; __any_sync(kFull, mine && c < 0); wbase += 64) {
      uint32_t lo = 0, hi = 0;
      if (mine && c < 0)
        visit_row<G>(g.colind, g.nnz, s, e, lg, g.vec, [&](int32_t w) {
          if (w != v && when[w] < round) {
            const int32_t cw = col[w] - wbase;
            if (cw >= 0 && cw < 32) lo |= 1u << cw;
            else if (cw >= 32 && cw < 64) hi |= 1u << (cw - 32);
          }
        });
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        lo |= __shfl_xor_sync(kFull, lo, o);
        hi |= __shfl_xor_sync(kFull, hi, o);
      }
      if (mine && c < 0) {
        if (~lo != 0u) c = wbase + __ffs(~lo) - 1;
        else if (~hi != 0u) c = wbase + 32 + __ffs(~hi) - 1;
      }
    }
    if (mine && lg == 0) {
      col[v] = c;
      when[v] = round;
      atomicMax(max_color, c);
    }
    if (active && !mine && lg == 0) still++;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) still += __shfl_xor_sync(kFull, still, o);
  if (lane == 0 && still > 0) atomicAdd(left, still);
}

template <int G, typename I>
int color_rounds_t(mis2_ctx* c, const GraphView<I>& gv, const PrioCfg& p, int32_t* colors, cudaStream_t st,
                   int32_t* rounds, int32_t* n_colors) {
  Scratch& s = c->s;
  uint32_t* prio = s.M;
  int32_t* when = s.tent;
  int32_t* left = s.ctr + kCtrRoots;
  int32_t* maxc = s.ctr + kCtrM2;
  MIS2_CUDA(cudaMemsetAsync(maxc, 0xFF, sizeof(int32_t), st));
  k_color_init<<<grid_for(c, gv.n, kBlock), kBlock, 0, st>>>(gv.n, p, prio, colors, when);
  c->launches++;
  const int wb = grid_for(c, gv.n, kBlock / 32 * (32 / G));
  int32_t r = 0;
  for (;; r++) {
    if (r > gv.n) return MIS2_ERR_NO_PROGRESS;
    MIS2_CUDA(cudaMemsetAsync(left, 0, sizeof(int32_t), st));
    k_color_round<G, I><<<wb, kBlock, 0, st>>>(gv, prio, colors, when, r, left, maxc);
    c->launches++;
    MIS2_CUDA(cudaGetLastError());
    MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    if (c->h_ctr[kCtrRoots] == 0) break;
  }
  *rounds = r + 1;
  *n_colors = c->h_ctr[kCtrM2] + 1;
  return MIS2_OK;
}

template <typename I>
int color_t(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, int32_t* colors, cudaStream_t st, int32_t* rounds,
            int32_t* n_colors) {
  GraphView<I> gv;
  gv.rowptr = static_cast<const I*>(g.rowptr);
  gv.colind = g.colind;
  gv.n = g.n;
  gv.nnz = g.nnz;
  gv.vec = g.vec ? 1 : 0;
  gv.pad = 0;
  const double avg = g.n > 0 ? (double)g.nnz / (double)g.n : 0.0;
  return avg < 40.0 ? color_rounds_t<4, I>(c, gv, p, colors, st, rounds, n_colors)
                    : color_rounds_t<32, I>(c, gv, p, colors, st, rounds, n_colors);
}

}  // namespace

int color_impl(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, int32_t* colors, int32_t* color_ptr,
               int32_t* color_list, int32_t* n_colors, int32_t* n_rounds, cudaStream_t st) {
  int32_t r = 0, nc = 0;
  if (g.n > 0)
    MIS2_TRY(g.rp64 ? color_t<int64_t>(c, g, p, colors, st, &r, &nc) : color_t<int32_t>(c, g, p, colors, st, &r, &nc));
  *n_colors = nc;
  if (n_rounds) *n_rounds = r;
  // colour sets: the vertices grouped by colour, ascending within a colour
  MIS2_TRY(group_by_key(c, colors, g.n, nc, color_ptr, color_list, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  return MIS2_OK;
}

}  // namespace mis2
