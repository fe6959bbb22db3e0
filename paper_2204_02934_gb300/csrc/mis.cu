// mis.cu -- Algorithm 1 (Section III-A) with a host-driven round loop, plus
// the ordered compactions and prefix sums the other phases use.
#include <algorithm>

#include "internal.h"
#include "mis_rows.cuh"
#include "scan.cuh"

namespace mis2 {

// ------------------------------------------------------------------ kernels
template <typename I>
__global__ void __launch_bounds__(kBlock) k_mis_init(GraphView<I> g, const int32_t* labels, PrioCfg p,
                                                     uint32_t* T, uint32_t* M, RowLists wl1, RowLists wl2,
                                                     int32_t* c1, int32_t* c2, int32_t warp_degree,
                                                     int32_t block_degree) {
  mis_init_rows<I>(g, labels, p, T, M, wl1, wl2, c1, c2, warp_degree, block_degree);
}

// Trace words of a phase: W from the three class counts, D by atomics.
struct PhaseTrace {
  int64_t* w;      // null: no trace this round
  int64_t* d;
  const int32_t* cnt_all;
};

__device__ __forceinline__ void phase_prologue(int32_t* zero, const PhaseTrace& tr) {
  if (blockIdx.x == 0 && threadIdx.x < kClasses && zero != nullptr) zero[threadIdx.x] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && tr.w != nullptr)
    *tr.w = (int64_t)tr.cnt_all[0] + tr.cnt_all[1] + tr.cnt_all[2];
}

template <int G, typename I>
__global__ void __launch_bounds__(kBlock) k_column(GraphView<I> g, const uint32_t* T, uint32_t* M,
                                                   const int32_t* wl_in, const int32_t* cnt_in,
                                                   int32_t* wl_out, int32_t* cnt_out, int32_t* zero,
                                                   PhaseTrace tr) {
  phase_prologue(zero, tr);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  column_group_rows<G, I, true>(g, T, M, wl_in, block_load(cnt_in), wl_out, cnt_out, tr.d, warp,
                                nw);
}

template <int G, typename I, bool GUARD>
__global__ void __launch_bounds__(kBlock) k_decide(GraphView<I> g, uint32_t* T, const uint32_t* M,
                                                   const int32_t* wl_in, const int32_t* cnt_in,
                                                   int32_t* wl_out, int32_t* cnt_out, int32_t* zero,
                                                   PhaseTrace tr, PrioCfg p, uint32_t next_iter) {
  phase_prologue(zero, tr);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  decide_group_rows<G, I, true, GUARD>(g, T, M, wl_in, block_load(cnt_in), wl_out, cnt_out, tr.d, p, next_iter,
                                       warp, nw);
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_column_lane(GraphView<I> g, const uint32_t* T, uint32_t* M,
                                                        const int32_t* wl_in, const int32_t* cnt_in, int32_t* wl_out,
                                                        int32_t* cnt_out, int32_t* zero, PhaseTrace tr) {
  __shared__ __align__(16) int32_t stage[kBlock / 32][kWarpSmemWords];
  phase_prologue(zero, tr);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  column_lane_rows<I, true>(g, T, M, wl_in, block_load(cnt_in), wl_out, cnt_out, tr.d, warp, nw,
                            stage[threadIdx.x >> 5]);
}

template <typename I, bool GUARD>
__global__ void __launch_bounds__(kBlock) k_decide_lane(GraphView<I> g, uint32_t* T, const uint32_t* M,
                                                        const int32_t* wl_in, const int32_t* cnt_in, int32_t* wl_out,
                                                        int32_t* cnt_out, int32_t* zero, PhaseTrace tr, PrioCfg p,
                                                        uint32_t next_iter) {
  __shared__ __align__(16) int32_t stage[kBlock / 32][kWarpSmemWords];
  phase_prologue(zero, tr);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  decide_lane_rows<I, true, GUARD>(g, T, M, wl_in, block_load(cnt_in), wl_out, cnt_out, tr.d, p, next_iter, warp,
                                   nw, stage[threadIdx.x >> 5]);
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_column_block(GraphView<I> g, const uint32_t* T, uint32_t* M,
                                                         const int32_t* wl_in, const int32_t* cnt_in,
                                                         int32_t* wl_out, int32_t* cnt_out, int64_t* dsum) {
  __shared__ uint32_t sh[40];
  column_block_rows<I, true>(g, T, M, wl_in, block_load(cnt_in), wl_out, cnt_out, dsum, blockIdx.x, gridDim.x, sh);
}

template <typename I, bool GUARD>
__global__ void __launch_bounds__(kBlock) k_decide_block(GraphView<I> g, uint32_t* T, const uint32_t* M,
                                                         const int32_t* wl_in, const int32_t* cnt_in,
                                                         int32_t* wl_out, int32_t* cnt_out, int64_t* dsum,
                                                         PrioCfg p, uint32_t next_iter) {
  __shared__ uint32_t sh[40];
  decide_block_rows<I, true, GUARD>(g, T, M, wl_in, block_load(cnt_in), wl_out, cnt_out, dsum, p, next_iter,
                                    blockIdx.x, gridDim.x, sh);
}

__global__ void __launch_bounds__(1024) k_scan_tile_counts(int32_t* tile_cnt, int64_t ntiles, int32_t* total) {
  pdl_enter();
  __shared__ int sh[40];
  __shared__ int carry_sh;
  if (threadIdx.x == 0) carry_sh = 0;
  __syncthreads();
  const int lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int x = i < ntiles ? tile_cnt[i] : 0;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int w = lane < nw ? sh[lane] : 0;
      int wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += y;
      }
      if (lane < nw) sh[lane] = wi - w;
      if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    const int carry = carry_sh;
    if (i < ntiles) tile_cnt[i] = carry + sh[warp] + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) carry_sh = carry + sh[32];
    __syncthreads();
  }
  if (threadIdx.x == 0 && total != nullptr) *total = carry_sh;
}

struct PredIn {
  const uint32_t* T;
  __device__ bool operator()(int64_t i) const { return T[i] == kIn; }
};
struct EmitRoots {
  int32_t* roots;
  uint8_t* flags;
  LevelFill fill;
  __device__ void operator()(int64_t i, int32_t pos, bool keep) const {
    if (flags != nullptr) flags[i] = keep ? 1 : 0;
    if (keep && roots != nullptr) roots[pos] = (int32_t)i;
    if (fill.minus1 != nullptr) fill.minus1[i] = -1;
#pragma unroll
    for (int k = 0; k < 3; k++)
      if (fill.zero[k] != nullptr) fill.zero[k][i] = 0;
  }
};
struct PredFlag {
  const uint8_t* f;
  __device__ bool operator()(int64_t i) const { return f[i] != 0; }
};
struct EmitMapped {
  const int32_t* map;
  int32_t* out;
  __device__ void operator()(int64_t i, int32_t pos, bool keep) const {
    if (keep) out[pos] = map != nullptr ? map[i] : (int32_t)i;
  }
};
struct ValArr {
  const int32_t* a;
  __device__ int operator()(int64_t i) const { return a[i]; }
};

// ------------------------------------------------------------------ host side
int grid_for(const mis2_ctx* c, int64_t items, int items_per_block, int blocks_per_sm) {
  int64_t b = (items + items_per_block - 1) / items_per_block;
  b = std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)c->sm_count * blocks_per_sm));
  return (int)b;
}

// Row mapping from the average degree (measured on GB300 over 7-/27-point
// grids, 2-, 3- and 5-dof elasticity, random geometric graphs and R-MAT):
// below 40 a lane per row (32 independent rows in flight per warp) and a warp
// from 32 entries on; above it, rows of up to 255 entries stay with small
// lane groups (16 or 8 rows in flight per warp beat a warp per row, whose
// one row at a time leaves the loop latency-bound: 2.3-3.1x on those
// graphs), and only longer rows get a warp.
int pick_group_lanes(const mis2_ctx* c, const GraphArgs& g) {
  if (c->cfg.group_lanes > 0) return c->cfg.group_lanes;
  const double avg = g.n > 0 ? (double)g.nnz / (double)g.n : 0.0;
  if (avg < 40) return 1;
  if (avg < 128) return 2;
  return 4;
}

int pick_warp_degree(const mis2_ctx* c, const GraphArgs& g) {
  if (c->cfg.warp_degree > 0) return c->cfg.warp_degree;
  const double avg = g.n > 0 ? (double)g.nnz / (double)g.n : 0.0;
  return std::min(avg < 40 ? 32 : 256, (int)c->cfg.block_degree);
}

template <typename I>
static GraphView<I> view_of(const GraphArgs& g) {
  GraphView<I> v;
  v.rowptr = static_cast<const I*>(g.rowptr);
  v.colind = g.colind;
  v.n = g.n;
  v.nnz = g.nnz;
  v.vec = g.vec ? 1 : 0;
  v.pad = 0;
  return v;
}

template <typename I>
static void launch_column(mis2_ctx* c, const GraphView<I>& gv, int G, int cls, int blocks, const int32_t* wl_in,
                          const int32_t* cnt_in, int32_t* wl_out, int32_t* cnt_out, int32_t* zero,
                          PhaseTrace tr, cudaStream_t st) {
  c->launches++;
  if (cls == 2) {
    k_column_block<I><<<blocks, kBlock, 0, st>>>(gv, c->s.T, c->s.M, wl_in, cnt_in, wl_out, cnt_out, tr.d);
    return;
  }
  if (cls == 1) G = 32;
#define MIS2_COL(GG) \
  k_column<GG, I><<<blocks, kBlock, 0, st>>>(gv, c->s.T, c->s.M, wl_in, cnt_in, wl_out, cnt_out, zero, tr)
  switch (G) {
    case 1:
      k_column_lane<I><<<blocks, kBlock, 0, st>>>(gv, c->s.T, c->s.M, wl_in, cnt_in, wl_out, cnt_out, zero, tr);
      break;
    case 2: MIS2_COL(2); break;
    case 4: MIS2_COL(4); break;
    case 8: MIS2_COL(8); break;
    case 16: MIS2_COL(16); break;
    default: MIS2_COL(32); break;
  }
#undef MIS2_COL
}

template <typename I>
static void launch_decide(mis2_ctx* c, const GraphView<I>& gv, int G, int cls, int blocks, const int32_t* wl_in,
                          const int32_t* cnt_in, int32_t* wl_out, int32_t* cnt_out, int32_t* zero,
                          PhaseTrace tr, const PrioCfg& p, uint32_t next_iter, cudaStream_t st, bool guard) {
  c->launches++;
  if (cls == 2) {
    if (guard)
      k_decide_block<I, true><<<blocks, kBlock, 0, st>>>(gv, c->s.T, c->s.M, wl_in, cnt_in, wl_out, cnt_out, tr.d,
                                                         p, next_iter);
    else
      k_decide_block<I, false><<<blocks, kBlock, 0, st>>>(gv, c->s.T, c->s.M, wl_in, cnt_in, wl_out, cnt_out, tr.d,
                                                          p, next_iter);
    return;
  }
  if (cls == 1) G = 32;
#define MIS2_DEC(GG)                                                                                      \
  if (guard)                                                                                              \
    k_decide<GG, I, true><<<blocks, kBlock, 0, st>>>(gv, c->s.T, c->s.M, wl_in, cnt_in, wl_out, cnt_out, zero, \
                                                     tr, p, next_iter);                                        \
  else                                                                                                    \
    k_decide<GG, I, false><<<blocks, kBlock, 0, st>>>(gv, c->s.T, c->s.M, wl_in, cnt_in, wl_out, cnt_out, zero, \
                                                      tr, p, next_iter)
  switch (G) {
    case 1:
      if (guard)
        k_decide_lane<I, true><<<blocks, kBlock, 0, st>>>(gv, c->s.T, c->s.M, wl_in, cnt_in, wl_out, cnt_out, zero,
                                                          tr, p, next_iter);
      else
        k_decide_lane<I, false><<<blocks, kBlock, 0, st>>>(gv, c->s.T, c->s.M, wl_in, cnt_in, wl_out, cnt_out, zero,
                                                           tr, p, next_iter);
      break;
    case 2: MIS2_DEC(2); break;
    case 4: MIS2_DEC(4); break;
    case 8: MIS2_DEC(8); break;
    case 16: MIS2_DEC(16); break;
    default: MIS2_DEC(32); break;
  }
#undef MIS2_DEC
}

template <typename I>
static int rounds_host_t(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const PrioCfg& p,
                         int trace_phase, cudaStream_t st, int32_t* rounds) {
  Scratch& s = c->s;
  const GraphView<I> gv = view_of<I>(g);
  const int G = pick_group_lanes(c, g);
  int64_t* dtr = s.dtrace + (int64_t)trace_phase * MIS2_TRACE_CAP * 4;
  MIS2_CUDA(cudaMemsetAsync(s.ctr, 0, 18 * sizeof(int32_t), st));
  MIS2_CUDA(cudaMemsetAsync(dtr, 0, MIS2_TRACE_CAP * 4 * sizeof(int64_t), st));
  RowLists l1, l2;
  for (int k = 0; k < kClasses; k++) {
    l1.l[k] = s.wl1[0][k];
    l2.l[k] = s.wl2[0][k];
  }
  timer_begin(c, kKcInit, st);
  k_mis_init<I><<<grid_for(c, g.n, kBlock), kBlock, 0, st>>>(gv, labels, p, s.T, s.M, l1, l2,
                                                              s.ctr + ctr_c1(0, 0), s.ctr + ctr_c2(0, 0),
                                                              pick_warp_degree(c, g), c->cfg.block_degree);
  c->launches++;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  // no-worklist mode (ablation): every round visits the round-0 lists, whose
  // sizes are kept in ctr words kCtrInitSizes.. (the slots rotate)
  const bool nowl = (c->cfg.ablation & MIS2_ABLATE_NO_WORKLISTS) != 0;
  if (nowl) {
    MIS2_CUDA(cudaMemcpyAsync(s.ctr + kCtrInitSizes, s.ctr + ctr_c1(0, 0), kClasses * sizeof(int32_t),
                              cudaMemcpyDeviceToDevice, st));
    MIS2_CUDA(cudaMemcpyAsync(s.ctr + kCtrInitSizes + kClasses, s.ctr + ctr_c2(0, 0), kClasses * sizeof(int32_t),
                              cudaMemcpyDeviceToDevice, st));
  }
  // mis2_run_snapshots: the round's copy of T or M (stream-ordered)
  auto snap = [&](int round, int which, const uint32_t* src) -> int {
    if (c->snaps == nullptr || labels != nullptr || round >= c->snap_rounds) return MIS2_OK;
    MIS2_CUDA(cudaMemcpyAsync(c->snaps + ((int64_t)round * 3 + which) * g.n, src, (size_t)g.n * sizeof(uint32_t),
                              cudaMemcpyDeviceToDevice, st));
    return MIS2_OK;
  };
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  int32_t n1_0[kClasses], n2_0[kClasses];
  for (int k = 0; k < kClasses; k++) {
    n1_0[k] = c->h_ctr[ctr_c1(0, k)];
    n2_0[k] = c->h_ctr[ctr_c2(0, k)];
  }
  int r = 0;
  for (;;) {
    const int slot = r % 3, nslot = (r + 1) % 3, zslot = (r + 2) % 3;
    int64_t w1 = 0;
    int32_t n1[kClasses], n2[kClasses];
    for (int k = 0; k < kClasses; k++) {
      n1[k] = c->h_ctr[ctr_c1(slot, k)];
      n2[k] = c->h_ctr[ctr_c2(slot, k)];
      w1 += n1[k];
    }
    if (w1 == 0) break;
    if (r > g.n) return MIS2_ERR_NO_PROGRESS;
    MIS2_TRY(snap(r, 0, s.T));  // T after round r's row refresh
    if (nowl)
      for (int k = 0; k < kClasses; k++) {
        n1[k] = n1_0[k];
        n2[k] = n2_0[k];
      }
    const bool tr_on = r < MIS2_TRACE_CAP;
    int32_t* c1_in = nowl ? s.ctr + kCtrInitSizes : s.ctr + ctr_c1(slot, 0);
    int32_t* c2_in = nowl ? s.ctr + kCtrInitSizes + kClasses : s.ctr + ctr_c2(slot, 0);
    PhaseTrace tcol{tr_on ? dtr + r * 4 + 1 : nullptr, tr_on ? dtr + r * 4 + 3 : nullptr, c2_in};
    PhaseTrace tdec{tr_on ? dtr + r * 4 + 0 : nullptr, tr_on ? dtr + r * 4 + 2 : nullptr, c1_in};
    const int rp = nowl ? 0 : r & 1, wp = (r + 1) & 1;
    // column step over worklist2
    timer_begin(c, kKcColumn, st);
    for (int k = 0; k < kClasses; k++) {
      if (k > 0 && n2[k] == 0) continue;
      const int per_block = k == 0 ? kBlock / G : (k == 1 ? kBlock / 32 : 1);
      const int blocks = grid_for(c, n2[k], per_block, k == 2 ? 4 : 8);
      PhaseTrace t = tcol;
      if (k > 0) t.w = nullptr;
      launch_column<I>(c, gv, G, k, blocks, s.wl2[rp][k], c2_in + k, nowl ? nullptr : s.wl2[wp][k],
                       s.ctr + ctr_c2(nslot, k), k == 0 ? s.ctr + ctr_c1(nslot, 0) : nullptr, t, st);
    }
    timer_end(c, st);
    MIS2_TRY(snap(r, 1, s.M));
    // decide over worklist1 (with the next round's refresh)
    timer_begin(c, kKcDecide, st);
    for (int k = 0; k < kClasses; k++) {
      if (k > 0 && n1[k] == 0) continue;
      const int per_block = k == 0 ? kBlock / G : (k == 1 ? kBlock / 32 : 1);
      const int blocks = grid_for(c, n1[k], per_block, k == 2 ? 4 : 8);
      PhaseTrace t = tdec;
      if (k > 0) t.w = nullptr;
      launch_decide<I>(c, gv, G, k, blocks, s.wl1[rp][k], c1_in + k, nowl ? nullptr : s.wl1[wp][k],
                       s.ctr + ctr_c1(nslot, k), k == 0 ? s.ctr + ctr_c2(zslot, 0) : nullptr, t, p,
                       (uint32_t)(r + 1), st, nowl);
    }
    timer_end(c, st);
    MIS2_CUDA(cudaGetLastError());
    MIS2_TRY(snap(r, 2, s.T));
    MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    r++;
  }
  *rounds = r;
  return MIS2_OK;
}

int mis2_rounds_host(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const PrioCfg& p, int trace_phase,
                     cudaStream_t st, int32_t* rounds) {
  return g.rp64 ? rounds_host_t<int64_t>(c, g, labels, p, trace_phase, st, rounds)
                : rounds_host_t<int32_t>(c, g, labels, p, trace_phase, st, rounds);
}

int extract_in_set(mis2_ctx* c, int64_t n, uint8_t* flags, int32_t* roots, int32_t* count_dev, cudaStream_t st,
                   const LevelFill& fill) {
  if (n == 0) {
    MIS2_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(int32_t), st));
    return MIS2_OK;
  }
  const int64_t nt = scan_tiles(n);
  const int blocks = grid_for(c, nt, 1, 8);
  timer_begin(c, kKcCompact, st);
  const bool direct = nt <= kScanDirectTiles;
  launch_k(c, k_tile_count<PredIn>, blocks, kBlock, st, n, PredIn{c->s.T}, c->s.tile);
  if (!direct) launch_k(c, k_scan_tile_counts, 1, 1024, st, c->s.tile, nt, count_dev);
  launch_k(c, k_tile_compact<PredIn, EmitRoots>, blocks, kBlock, st, n, PredIn{c->s.T}, c->s.tile,
                                                               EmitRoots{roots, flags, fill}, direct, count_dev);
  c->launches += direct ? 2 : 3;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

int compact_flags(mis2_ctx* c, const uint8_t* flags, const int32_t* map, int64_t n, int32_t* out,
                  int32_t* count_dev, cudaStream_t st) {
  if (n == 0) {
    MIS2_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(int32_t), st));
    return MIS2_OK;
  }
  const int64_t nt = scan_tiles(n);
  const int blocks = grid_for(c, nt, 1, 8);
  timer_begin(c, kKcCompact, st);
  const bool direct = nt <= kScanDirectTiles;
  launch_k(c, k_tile_count<PredFlag>, blocks, kBlock, st, n, PredFlag{flags}, c->s.tile);
  if (!direct) launch_k(c, k_scan_tile_counts, 1, 1024, st, c->s.tile, nt, count_dev);
  launch_k(c, k_tile_compact<PredFlag, EmitMapped>, blocks, kBlock, st, n, PredFlag{flags}, c->s.tile,
                                                                  EmitMapped{map, out}, direct, count_dev);
  c->launches += direct ? 2 : 3;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

int exclusive_scan_i32(mis2_ctx* c, const int32_t* vals, int64_t n, int32_t* out, int32_t* total_dev,
                       cudaStream_t st, int32_t* out2) {
  if (n == 0) {
    MIS2_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
    if (total_dev) MIS2_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int32_t), st));
    return MIS2_OK;
  }
  const int64_t nt = scan_tiles(n);
  const int blocks = grid_for(c, nt, 1, 8);
  timer_begin(c, kKcCompact, st);
  const bool direct = nt <= kScanDirectTiles;
  launch_k(c, k_tile_sum<ValArr>, blocks, kBlock, st, n, ValArr{vals}, c->s.tile);
  if (!direct) launch_k(c, k_scan_tile_counts, 1, 1024, st, c->s.tile, nt, total_dev);
  launch_k(c, k_tile_scan_write<ValArr, int32_t>, blocks, kBlock, st, n, ValArr{vals}, c->s.tile, out, out2, direct,
           total_dev);
  c->launches += direct ? 2 : 3;
  timer_end(c, st);
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

}  // namespace mis2
