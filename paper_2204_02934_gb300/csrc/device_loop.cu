// device_loop.cu -- the whole round loop of Algorithm 1 in one persistent
// cooperative kernel: every block stays resident, phases are separated by a
// grid-wide barrier, and the loop ends when worklist1 is empty (read by all
// blocks right after the decide barrier).  No host synchronisation per
// round.  Every barrier wait is bounded: after spin_limit polls a block
// raises the timeout flag, all blocks leave, and the host reports
// MIS2_ERR_TIMEOUT instead of hanging.
//
// A launch leaves the counter words as the next launch needs them, so that
// back-to-back MIS-2 launches of a level need no clearing in between: the
// worklist sizes zero, the barrier's arrival count at its value with the
// base word (kCtrBarrier + 1) equal to it, and its trace rows zero from the
// round where it stopped on (each round clears the next round's row).
#include <algorithm>

#include "grid_sync.cuh"
#include "internal.h"
#include "mis_rows.cuh"

namespace mis2 {

// Minimum resident blocks per SM the loop kernel is compiled for (register
// budget: 65536 / (256 * MIS2_LOOP_MINB) per thread).
#ifndef MIS2_LOOP_MINB
#define MIS2_LOOP_MINB 2
#endif

struct LoopArgs {
  RowLists wl1[2];
  RowLists wl2[2];
  uint32_t* T;
  uint32_t* M;
  int32_t* ctr;
  int64_t* dtr;  // trace of this MIS-2 (MIS2_TRACE_CAP x 4)
  int64_t* ts;   // barrier timestamps (2 per barrier) or null
  const int32_t* labels;
  int64_t spin_limit;
  int32_t warp_degree;
  int32_t block_degree;
  int32_t max_rounds;
  int32_t rounds_slot;
  int32_t barrier_extra;  // arrivals awaited beyond the grid: 1 = forced timeout (test hook)
  int32_t no_worklists;   // visit every vertex every round (ablation)
  uint32_t* snaps;        // mis2_run_snapshots: per-round copies of T and M, or null
  int32_t snap_rounds;
};

// Copy n words grid-wide (mis2_run_snapshots); the source is not written in
// the phase that runs until the next grid barrier.
__device__ __forceinline__ void grid_copy(uint32_t* dst, const uint32_t* src, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

template <int G, typename I, bool NOWL>
__global__ void __launch_bounds__(kBlock, MIS2_LOOP_MINB) k_mis_loop(GraphView<I> g, PrioCfg p, LoopArgs a) {
  __shared__ uint32_t sh[40];
  __shared__ int32_t sh_n[2 * kClasses];
  __shared__ int32_t sh_n0[2 * kClasses];  // round-0 sizes: every vertex (no-worklist mode)
  __shared__ __align__(16) int32_t stage[kBlock / 32][kWarpSmemWords];
  int32_t* my_stage = stage[threadIdx.x >> 5];
  int32_t* ctr = a.ctr;
  int32_t* bar_count = ctr + kCtrBarrier;
  int32_t epoch = 0;
  int32_t* err = ctr + kCtrErr;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t warp = tid >> 5, nwarps = nthreads >> 5;

  int64_t* ts = a.ts;
  if (ts != nullptr && tid == 0) ts[0] = global_ns();  // block 0 starts
  // arrival count when the launch started: written by the previous launch
  // after its last barrier, read here before this launch's first one
  const uint32_t bar_base = (uint32_t)ld_volatile_i32(ctr + kCtrBarrier + 1);
  if (tid == 0 && a.dtr != nullptr)
    for (int k = 0; k < 4; k++) a.dtr[k] = 0;  // round 0's trace row
  // worklist 2 starts equal to worklist 1: round 0's column step reads the
  // worklist-1 lists, so only worklist 2's sizes are set here
  const RowLists none{{nullptr, nullptr, nullptr}};
  mis_init_rows<I>(g, a.labels, p, a.T, a.M, a.wl1[0], none, ctr + ctr_c1(0, 0), ctr + ctr_c2(0, 0),
                   a.warp_degree, a.block_degree);
  if (ts != nullptr && tid == 0) ts[1] = global_ns();  // block 0 has set up its vertices
  if (!grid_barrier(bar_count, epoch, err, a.spin_limit, ts ? ts + 2 : nullptr, a.barrier_extra, bar_base)) return;

  constexpr bool nowl = NOWL;
  int r = 0;
  for (;; r++) {
    const int slot = r % 3, nslot = (r + 1) % 3, zslot = (r + 2) % 3;
    // the worklist sizes: read once per block (one request instead of one
    // per warp on the same L2 line) and shared
    if (threadIdx.x < 2 * kClasses) {
      const int32_t x = ld_volatile_i32(ctr + (threadIdx.x < kClasses ? ctr_c1(slot, (int)threadIdx.x)
                                                                       : ctr_c2(slot, (int)threadIdx.x - kClasses)));
      sh_n[threadIdx.x] = x;
      if (r == 0) sh_n0[threadIdx.x] = x;
    }
    __syncthreads();
    int n1[kClasses], n2[kClasses];
    int w1 = 0, w2 = 0;
#pragma unroll
    for (int k = 0; k < kClasses; k++) {
      n1[k] = sh_n[k];
      n2[k] = sh_n[kClasses + k];
      w1 += n1[k];
      w2 += n2[k];
    }
    if (a.snaps != nullptr) {  // T after round r - 1's decide step, after round r's refresh
      if (r > 0 && r - 1 < a.snap_rounds) grid_copy(a.snaps + ((int64_t)(r - 1) * 3 + 2) * g.n, a.T, g.n);
      if (w1 > 0 && r < a.snap_rounds) grid_copy(a.snaps + (int64_t)r * 3 * g.n, a.T, g.n);
    }
    if (w1 == 0) break;
    if (nowl) {  // every vertex visited; n1/n2 above were the compacted counts
      w2 = 0;
#pragma unroll
      for (int k = 0; k < kClasses; k++) {
        n1[k] = sh_n0[k];
        n2[k] = sh_n0[kClasses + k];
        w2 += n2[k];
      }
    }
    if (r > a.max_rounds) {
      if (tid == 0) atomicOr(err, kErrNoProgress);
      break;
    }
    const bool tr_on = a.dtr != nullptr && r < MIS2_TRACE_CAP;
    int64_t* d2 = tr_on ? a.dtr + r * 4 + 3 : nullptr;
    int64_t* d1 = tr_on ? a.dtr + r * 4 + 2 : nullptr;
    const RowLists in2 = (nowl || r == 0) ? a.wl1[0] : a.wl2[r & 1], out2 = nowl ? none : a.wl2[(r + 1) & 1];
    const RowLists in1 = nowl ? a.wl1[0] : a.wl1[r & 1], out1 = nowl ? none : a.wl1[(r + 1) & 1];
    // ---- column step
    if (tid < kClasses) ctr[ctr_c1(nslot, (int)tid)] = 0;
    if (tid == 0 && tr_on) a.dtr[r * 4 + 1] = w2;
    if (tid == 0 && a.dtr != nullptr && r + 1 < MIS2_TRACE_CAP)
      for (int k = 0; k < 4; k++) a.dtr[(r + 1) * 4 + k] = 0;  // summed into during round r + 1
    if constexpr (G == 1)
      column_lane_rows<I, false>(g, a.T, a.M, in2.l[0], n2[0], out2.l[0], ctr + ctr_c2(nslot, 0), d2, warp, nwarps,
                                 my_stage);
    else
      column_group_rows<G, I, false>(g, a.T, a.M, in2.l[0], n2[0], out2.l[0], ctr + ctr_c2(nslot, 0), d2, warp,
                                     nwarps);
    if (n2[1] > 0)
      column_group_rows<32, I, false>(g, a.T, a.M, in2.l[1], n2[1], out2.l[1], ctr + ctr_c2(nslot, 1), d2, warp,
                                      nwarps);
    if (n2[2] > 0)
      column_block_rows<I, false>(g, a.T, a.M, in2.l[2], n2[2], out2.l[2], ctr + ctr_c2(nslot, 2), d2, blockIdx.x,
                                  gridDim.x, sh);
    const bool ts_on = ts != nullptr && r < MIS2_TRACE_CAP;
    if (!grid_barrier(bar_count, epoch, err, a.spin_limit, ts_on ? ts + 4 + 4 * r : nullptr, a.barrier_extra,
                      bar_base))
      return;
    if (a.snaps != nullptr && r < a.snap_rounds) grid_copy(a.snaps + ((int64_t)r * 3 + 1) * g.n, a.M, g.n);
    // ---- decide step (with the next round's row refresh)
    if (tid < kClasses) ctr[ctr_c2(zslot, (int)tid)] = 0;
    if (tid == 0 && tr_on) a.dtr[r * 4 + 0] = nowl ? n1[0] + n1[1] + n1[2] : w1;
    if constexpr (G == 1)
      decide_lane_rows<I, false, NOWL>(g, a.T, a.M, in1.l[0], n1[0], out1.l[0], ctr + ctr_c1(nslot, 0), d1, p,
                                 (uint32_t)(r + 1), warp, nwarps, my_stage);
    else
      decide_group_rows<G, I, false, NOWL>(g, a.T, a.M, in1.l[0], n1[0], out1.l[0], ctr + ctr_c1(nslot, 0), d1, p,
                                     (uint32_t)(r + 1), warp, nwarps);
    if (n1[1] > 0)
      decide_group_rows<32, I, false, NOWL>(g, a.T, a.M, in1.l[1], n1[1], out1.l[1], ctr + ctr_c1(nslot, 1), d1, p,
                                      (uint32_t)(r + 1), warp, nwarps);
    if (n1[2] > 0)
      decide_block_rows<I, false, NOWL>(g, a.T, a.M, in1.l[2], n1[2], out1.l[2], ctr + ctr_c1(nslot, 2), d1, p,
                                  (uint32_t)(r + 1), blockIdx.x, gridDim.x, sh);
    if (!grid_barrier(bar_count, epoch, err, a.spin_limit, ts_on ? ts + 6 + 4 * r : nullptr, a.barrier_extra,
                      bar_base))
      return;
  }
  // Every block has passed the last barrier, so every block has read the
  // base and no block writes a worklist size again; a block still to read
  // this round's sizes sees worklist 1 empty, as it is, and stops too.
  if (blockIdx.x == 0) {
    if (threadIdx.x < 18) ctr[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
      ctr[a.rounds_slot] = r;
      ctr[kCtrBarrier + 1] = (int32_t)(bar_base + (uint32_t)epoch * gridDim.x);
      if (a.dtr != nullptr)
        for (int k = r * 4; k < MIS2_TRACE_CAP * 4; k++) a.dtr[k] = 0;  // rows of rounds that did not run
    }
  }
}

template <int G, typename I>
static int launch_loop(mis2_ctx* c, GraphView<I> gv, PrioCfg p, LoopArgs la, cudaStream_t st) {
  auto kern = la.no_worklists ? k_mis_loop<G, I, true> : k_mis_loop<G, I, false>;
  int per_sm = 0;
  MIS2_TRY(resident_blocks_per_sm(c, (const void*)kern, kBlock, &per_sm));
  if (per_sm < 1) return MIS2_ERR_CUDA;
  const int want = c->cfg.loop_blocks_per_sm > 0 ? c->cfg.loop_blocks_per_sm : 2;
  const int blocks = c->sm_count * std::min(per_sm, want);
  c->device_loop_blocks = blocks;
  void* args[] = {&gv, &p, &la};
  if (c->coop_lock != nullptr) {
    std::lock_guard<std::mutex> lk(*c->coop_lock);
    MIS2_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(kBlock), args, 0, st));
    MIS2_CUDA(cudaEventRecord(c->coop_done, st));
    MIS2_CUDA(cudaEventSynchronize(c->coop_done));
  } else {
    MIS2_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(kBlock), args, 0, st));
  }
  c->launches++;
  return MIS2_OK;
}

template <typename I>
static int rounds_device_t(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const PrioCfg& p,
                           int trace_phase, cudaStream_t st, int32_t* rounds, bool sync, int rounds_slot) {
  Scratch& s = c->s;
  GraphView<I> gv;
  gv.rowptr = static_cast<const I*>(g.rowptr);
  gv.colind = g.colind;
  gv.n = g.n;
  gv.nnz = g.nnz;
  gv.vec = g.vec ? 1 : 0;
  gv.pad = 0;
  LoopArgs la;
  for (int b = 0; b < 2; b++)
    for (int k = 0; k < kClasses; k++) {
      la.wl1[b].l[k] = s.wl1[b][k];
      la.wl2[b].l[k] = s.wl2[b][k];
    }
  la.T = s.T;
  la.M = s.M;
  la.ctr = s.ctr;
  la.dtr = s.dtrace + (int64_t)trace_phase * MIS2_TRACE_CAP * 4;
  la.ts = c->cfg.timing == MIS2_TIMING_ALL ? s.loop_ts + (int64_t)trace_phase * kLoopTsWords : nullptr;
  la.labels = labels;
  la.spin_limit = c->cfg.spin_limit;
  la.warp_degree = pick_warp_degree(c, g);
  la.block_degree = c->cfg.block_degree;
  la.max_rounds = (int32_t)std::min<int64_t>(g.n, (int64_t)1 << 30);
  la.rounds_slot = rounds_slot;
  la.barrier_extra = (c->cfg.debug_checks & MIS2_DEBUG_FORCE_TIMEOUT) ? 1 : 0;
  la.no_worklists = (c->cfg.ablation & MIS2_ABLATE_NO_WORKLISTS) ? 1 : 0;
  la.snaps = labels == nullptr ? c->snaps : nullptr;
  la.snap_rounds = c->snap_rounds;
  // async: the counter words were cleared at the level's start, or left
  // ready by the level's previous loop launch (see the top of this file);
  // the other counters of the level (roots, errors) stay
  if (sync) MIS2_CUDA(cudaMemsetAsync(s.ctr, 0, kCtrWords * sizeof(int32_t), st));
  if (la.ts != nullptr) MIS2_CUDA(cudaMemsetAsync(la.ts, 0, kLoopTsWords * sizeof(int64_t), st));
  timer_begin(c, kKcDeviceLoop, st);
  int rc;
  switch (pick_group_lanes(c, g)) {
    case 1: rc = launch_loop<1, I>(c, gv, p, la, st); break;
    case 2: rc = launch_loop<2, I>(c, gv, p, la, st); break;
    case 4: rc = launch_loop<4, I>(c, gv, p, la, st); break;
    case 8: rc = launch_loop<8, I>(c, gv, p, la, st); break;
    case 16: rc = launch_loop<16, I>(c, gv, p, la, st); break;
    default: rc = launch_loop<32, I>(c, gv, p, la, st); break;
  }
  timer_end(c, st);
  if (rc != MIS2_OK) return rc;
  if (la.ts != nullptr)
    MIS2_CUDA(cudaMemcpyAsync(c->stats.loop_ns[trace_phase], la.ts, kLoopTsWords * sizeof(int64_t),
                              cudaMemcpyDeviceToHost, st));
  if (!sync) return MIS2_OK;
  MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MIS2_CUDA(cudaStreamSynchronize(st));
  if (c->h_ctr[kCtrErr] & kErrTimeout) return MIS2_ERR_TIMEOUT;
  if (c->h_ctr[kCtrErr] & kErrNoProgress) return MIS2_ERR_NO_PROGRESS;
  *rounds = c->h_ctr[rounds_slot];
  return MIS2_OK;
}

int mis2_rounds_device_async(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const PrioCfg& p,
                             int trace_phase, int rounds_slot, cudaStream_t st) {
  return g.rp64 ? rounds_device_t<int64_t>(c, g, labels, p, trace_phase, st, nullptr, false, rounds_slot)
                : rounds_device_t<int32_t>(c, g, labels, p, trace_phase, st, nullptr, false, rounds_slot);
}

int mis2_rounds_device(mis2_ctx* c, const GraphArgs& g, const int32_t* labels, const PrioCfg& p, int trace_phase,
                       cudaStream_t st, int32_t* rounds) {
  return g.rp64 ? rounds_device_t<int64_t>(c, g, labels, p, trace_phase, st, rounds, true, kCtrRounds)
                : rounds_device_t<int32_t>(c, g, labels, p, trace_phase, st, rounds, true, kCtrRounds);
}

}  // namespace mis2
