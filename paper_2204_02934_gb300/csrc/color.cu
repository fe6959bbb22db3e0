// color.cu -- the colour sets of cluster multicolor Gauss-Seidel (Algorithm
// 4's setup: colorsets = color(A_c) on the coarse graph).  Jones-Plassmann
// rounds with the round-0 tuples of Eq. 1 as fixed priorities: an uncoloured
// vertex whose tuple is smaller than every uncoloured neighbour's takes the
// smallest colour no coloured neighbour holds.  Such vertices are pairwise
// non-adjacent, and each colours after all its smaller-tuple neighbours, so
// the result is the first-fit greedy colouring in ascending tuple order,
// whatever the schedule.  A neighbour coloured in the current round counts as
// uncoloured (round stamps), which keeps every round's decisions on the state
// before the round.  Each vertex remembers where its last blocker was found
// and resumes there (entries before it are coloured or have larger tuples,
// for good), so the blocked checks of all rounds read each row about once.
// Rows are split by length: short ones get G lanes each, medium ones a warp
// and long ones (hubs) a block.  Rounds
// are launched in batches of kColorBatch with one count readback per batch
// (rounds after the last one find nothing to do), or, with the device loop,
// all in one persistent cooperative launch with a bounded grid barrier per
// round; then the vertices of each colour, ascending, by a stable grouping
// on the colour.
#include <algorithm>

#include "grid_sync.cuh"
#include "internal.h"
#include "teams.cuh"

namespace mis2 {

namespace {

constexpr int32_t kUncolored = 0x7FFFFFFF;
constexpr int64_t kColorHeavy = 2048;
constexpr int kColorBatch = 8;
constexpr int kScanU = 4;  // entries a lane tests per step of the blocked scan

__global__ void __launch_bounds__(kBlock) k_color_init(int64_t n, PrioCfg p, uint32_t* prio, int32_t* col,
                                                       int32_t* when, int32_t* resume, uint32_t* mlo, uint32_t* mhi) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    prio[v] = make_tuple(p, 0u, (uint32_t)v);
    col[v] = -1;
    when[v] = kUncolored;
    resume[v] = 0;
    mlo[v] = 0u;
    mhi[v] = 0u;
  }
}

// Does w keep v waiting this round?  (w uncoloured before the round, smaller
// tuple; self-loops ignored.)
__device__ __forceinline__ bool blocks_v(int32_t w, int64_t v, uint32_t pv, const uint32_t* prio,
                                        const int32_t* when, int32_t round) {
  return w != v && when[w] >= round && prio[w] < pv;
}

// One Jones-Plassmann round over the short rows, G lanes per uncoloured
// vertex.  The blocked scan also collects the colours (below 64) of the
// neighbours it finds coloured: a neighbour coloured before v has the
// smaller tuple (a larger one waits for v), so its colour is final and
// belongs to v's first-fit mask, kept per vertex (mlo / mhi) across rounds.
// When v is no longer blocked its mask is complete, and it takes the first
// free colour without a second pass over the row; only a vertex whose
// neighbours use all of 0..63 walks the row again, window by window.
template <int G, bool PACK, typename I>
__device__ __forceinline__ void color_light_pass(const GraphView<I>& g, int64_t light_max, const uint32_t* prio,
                                                 int32_t* col, int32_t* when, int32_t* resume, uint32_t* mlo,
                                                 uint32_t* mhi, int32_t round, int32_t* left, int32_t* max_color) {
  const int lg = lane_id() & (G - 1);
  int32_t still = 0;
  for_picked<G, PACK>(
      g.n, [&](int64_t v) { return when[v] == kUncolored; },
      [&](int64_t v) {
        bool active = v >= 0;
        int64_t s = 0, e = 0;
        uint32_t pv = 0;
        int32_t res = 0;
        if (active) {
          row_range(g, v, s, e);
          active = e - s <= light_max;
          pv = prio[v];
          res = resume[v];
        }
        const int32_t len = active ? (int32_t)(e - s) : 0;
        // a smaller uncoloured neighbour, from the resume point on; stop at
        // the first chunk that holds one
        bool blocked = false;
        uint32_t lo = 0, hi = 0;  // colours of the coloured neighbours met
        for (int32_t off = res;; off += G * kScanU) {
          const bool live = active && !blocked && off < len;
          if (!__any_sync(kFull, live)) break;
          bool h = false;
          if (live) {
            int32_t w[kScanU], tw[kScanU];  // all loads of the step first, then the tests
#pragma unroll
            for (int u = 0; u < kScanU; u++) {
              const int32_t q = off + lg + u * G;
              w[u] = q < len ? __ldg(g.colind + s + q) : (int32_t)v;  // v itself neither blocks nor counts
            }
#pragma unroll
            for (int u = 0; u < kScanU; u++) tw[u] = w[u] != v ? when[w[u]] : kUncolored;
#pragma unroll
            for (int u = 0; u < kScanU; u++) {
              if (w[u] == v) continue;
              if (tw[u] < round) {
                const int32_t cw = col[w[u]];
                if (cw < 32) lo |= 1u << cw;
                else if (cw < 64) hi |= 1u << (cw - 32);
              } else if (prio[w[u]] < pv) {
                h = true;
              }
            }
          }
          if (group_any<G>(h) && live) {
            blocked = true;
            res = off;
          }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
          lo |= __shfl_xor_sync(kFull, lo, o);
          hi |= __shfl_xor_sync(kFull, hi, o);
        }
        if (active) {
          lo |= mlo[v];
          hi |= mhi[v];
        }
        const bool mine = active && !blocked;
        int32_t c = -1;
        if (mine) {
          if (~lo != 0u) c = __ffs(~lo) - 1;
          else if (~hi != 0u) c = 32 + __ffs(~hi) - 1;
        }
        // colours from 64 on (rare): the row again, a window of 64 at a time;
        // warp-uniform trip count: every lane takes part in the group reductions
        for (int32_t wbase = 64; __any_sync(kFull, mine && c < 0); wbase += 64) {
          uint32_t lo = 0, hi = 0;
          if (mine && c < 0)
            for (int32_t off = lg; off < len; off += G) {
              const int32_t w = __ldg(g.colind + s + off);
              if (w != v && when[w] < round) {
                const int32_t cw = col[w] - wbase;
                if (cw >= 0 && cw < 32) lo |= 1u << cw;
                else if (cw >= 32 && cw < 64) hi |= 1u << (cw - 32);
              }
            }
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
        if (lg == 0) {
          if (mine) {
            col[v] = c;
            when[v] = round;
            atomicMax(max_color, c);
          } else if (active) {
            resume[v] = res;
            mlo[v] = lo;
            mhi[v] = hi;
            still++;
          }
        }
      });
  still = (int32_t)__reduce_add_sync(kFull, (unsigned)still);
  if (lane_id() == 0 && still > 0) atomicAdd(left, still);
}

template <int G, bool PACK, typename I>
__global__ void __launch_bounds__(kBlock) k_color_round(GraphView<I> g, int64_t light_max, const uint32_t* prio,
                                                        int32_t* col, int32_t* when, int32_t* resume, uint32_t* mlo,
                                                        uint32_t* mhi, int32_t round, int32_t* left,
                                                        int32_t* max_color) {
  color_light_pass<G, PACK, I>(g, light_max, prio, col, when, resume, mlo, mhi, round, left, max_color);
}

// One listed row with a team of TPR threads (a warp or the block): the
// blocked scan from the resume point, kScanU entries a thread per step, then
// the first-fit windows.  Returns true (on every thread) if v still waits.
template <int TPR, typename I>
__device__ __forceinline__ bool color_row_team(const GraphView<I>& g, int32_t v, int tid, const uint32_t* prio,
                                               int32_t* col, int32_t* when, int32_t* resume, int32_t round,
                                               int32_t* max_color, uint32_t* sh) {
  int64_t s, e;
  row_range(g, v, s, e);
  const uint32_t pv = prio[v];
  int64_t p = s + resume[v];
  for (; p < e; p += (int64_t)TPR * kScanU) {  // team-uniform
    int32_t w[kScanU];
#pragma unroll
    for (int u = 0; u < kScanU; u++) {
      const int64_t k = p + tid + (int64_t)u * TPR;
      w[u] = k < e ? __ldg(g.colind + k) : v;
    }
    bool h = false;
#pragma unroll
    for (int u = 0; u < kScanU; u++) h |= blocks_v(w[u], v, pv, prio, when, round);
    if (team_any<TPR>(h)) {
      if (tid == 0) resume[v] = (int32_t)(p - s);
      return true;
    }
  }
  int32_t c = -1;
  for (int32_t wbase = 0; c < 0; wbase += 64) {  // team-uniform
    uint32_t lo = 0, hi = 0;
    for (int64_t k = s + tid; k < e; k += TPR) {
      const int32_t w = __ldg(g.colind + k);
      if (w != v && when[w] < round) {
        const int32_t cw = col[w] - wbase;
        if (cw >= 0 && cw < 32) lo |= 1u << cw;
        else if (cw >= 32 && cw < 64) hi |= 1u << (cw - 32);
      }
    }
    lo = team_or<TPR>(lo, sh);
    hi = team_or<TPR>(hi, sh);
    if (~lo != 0u) c = wbase + __ffs(~lo) - 1;
    else if (~hi != 0u) c = wbase + 32 + __ffs(~hi) - 1;
  }
  if (tid == 0) {
    col[v] = c;
    when[v] = round;
    atomicMax(max_color, c);
  }
  return false;
}

// The same round for the medium rows: warp per row.
template <typename I>
__device__ __forceinline__ void color_medium_pass(const GraphView<I>& g, const int32_t* list, int32_t nl,
                                                  const uint32_t* prio, int32_t* col, int32_t* when,
                                                  int32_t* resume, int32_t round, int32_t* left,
                                                  int32_t* max_color) {
  const int lane = lane_id();
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t still = 0;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < nl; j += nw) {  // warp-uniform
    const int32_t v = list[j];
    if (when[v] != kUncolored) continue;  // warp-uniform: only this warp writes when[v]
    if (color_row_team<32, I>(g, v, lane, prio, col, when, resume, round, max_color, nullptr) && lane == 0) still++;
  }
  still = (int32_t)__reduce_add_sync(kFull, (unsigned)still);
  if (lane == 0 && still > 0) atomicAdd(left, still);
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_color_medium(GraphView<I> g, const int32_t* list, const int32_t* n_list,
                                                         const uint32_t* prio, int32_t* col, int32_t* when,
                                                         int32_t* resume, int32_t round, int32_t* left,
                                                         int32_t* max_color) {
  color_medium_pass<I>(g, list, block_load(n_list), prio, col, when, resume, round, left, max_color);
}

// The same round for the heavy rows: block per row.  `sh` holds 33 words.
template <typename I>
__device__ __forceinline__ void color_heavy_pass(const GraphView<I>& g, const int32_t* list, int32_t nl,
                                                 const uint32_t* prio, int32_t* col, int32_t* when, int32_t* resume,
                                                 int32_t round, int32_t* left, int32_t* max_color, uint32_t* sh) {
  int32_t still = 0;
  for (int64_t j = blockIdx.x; j < nl; j += gridDim.x) {  // block-uniform
    const int32_t v = list[j];
    if (when[v] != kUncolored) continue;  // block-uniform: only this block writes when[v]
    if (color_row_team<kBlock, I>(g, v, threadIdx.x, prio, col, when, resume, round, max_color, sh) &&
        threadIdx.x == 0)
      still++;
  }
  if (threadIdx.x == 0 && still > 0) atomicAdd(left, still);
}

template <typename I>
__global__ void __launch_bounds__(kBlock) k_color_heavy(GraphView<I> g, const int32_t* list, const int32_t* n_list,
                                                        const uint32_t* prio, int32_t* col, int32_t* when,
                                                        int32_t* resume, int32_t round, int32_t* left,
                                                        int32_t* max_color) {
  __shared__ uint32_t sh[33];
  color_heavy_pass<I>(g, list, block_load(n_list), prio, col, when, resume, round, left, max_color, sh);
}

// Every round in one persistent cooperative launch: the three passes of a
// round, one grid barrier, then every block reads the round's count of
// vertices still waiting and stops at zero.  Counts rotate over three slots:
// the slot zeroed in round r was last read right after barrier r - 1.
template <int G, bool PACK, typename I>
__global__ void __launch_bounds__(kBlock) k_color_loop(GraphView<I> g, int64_t light_max, const uint32_t* prio,
                                                       int32_t* col, int32_t* when, int32_t* resume, uint32_t* mlo,
                                                       uint32_t* mhi,
                                                       const int32_t* medium, const int32_t* n_medium,
                                                       const int32_t* heavy, const int32_t* n_heavy, int32_t* ctr,
                                                       int32_t* max_color, int64_t spin_limit, int32_t max_rounds,
                                                       int32_t barrier_extra) {
  __shared__ uint32_t sh[33];
  __shared__ int32_t sh_left;
  int32_t* left = ctr + kCtrColorLeft;
  int32_t epoch = 0;
  const int32_t nm = block_load(n_medium), nh = block_load(n_heavy);
  int32_t r = 0;
  for (;; r++) {
    int32_t* lr = left + r % 3;
    color_light_pass<G, PACK, I>(g, light_max, prio, col, when, resume, mlo, mhi, r, lr, max_color);
    if (nm > 0) color_medium_pass<I>(g, medium, nm, prio, col, when, resume, r, lr, max_color);
    if (nh > 0) color_heavy_pass<I>(g, heavy, nh, prio, col, when, resume, r, lr, max_color, sh);
    if (!grid_barrier(ctr + kCtrBarrier, epoch, ctr + kCtrErr, spin_limit, nullptr, barrier_extra)) return;
    if (threadIdx.x == 0) sh_left = ld_volatile_i32(lr);
    __syncthreads();
    const int32_t still = sh_left;
    __syncthreads();
    if (still == 0) break;
    if (r >= max_rounds) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(ctr + kCtrErr, kErrNoProgress);
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) left[(r + 2) % 3] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctr[kCtrRounds] = r + 1;
}

template <int G, typename I>
int color_rounds_t(mis2_ctx* c, const GraphView<I>& gv, const GraphArgs& ga, const PrioCfg& p, int32_t* colors,
                   cudaStream_t st, int32_t* rounds, int32_t* n_colors) {
  Scratch& s = c->s;
  const int64_t light_max = G == 32 ? kColorHeavy : 64;
  LenLists rl;
  MIS2_TRY(classify_rows(c, ga, light_max, kColorHeavy, &rl, st));
  uint32_t* prio = s.M;
  int32_t* when = s.tent;
  int32_t* resume = s.members;
  uint32_t* mlo = reinterpret_cast<uint32_t*>(s.ub);  // first-fit masks of the short rows
  uint32_t* mhi = reinterpret_cast<uint32_t*>(s.ub_ptr);
  int32_t* left = s.ctr + kCtrColorLeft;
  int32_t* maxc = s.ctr + kCtrM2;
  MIS2_CUDA(cudaMemsetAsync(maxc, 0xFF, sizeof(int32_t), st));
  const int rb = grid_for(c, gv.n, kBlock);
  k_color_init<<<rb, kBlock, 0, st>>>(gv.n, p, prio, colors, when, resume, mlo, mhi);
  c->launches++;
  // packed walk (a warp per 32 vertices) once the graph fills the machine
  const bool pack = gv.n > (int64_t)c->sm_count * 2048;
  const int wb = pack ? grid_for(c, gv.n, kBlock) : grid_for(c, gv.n, kBlock / 32 * (32 / G));
  const int mb = rl.n_medium > 0 ? grid_for(c, rl.n_medium, kBlock / 32) : 0;
  const int hb = rl.n_heavy > 0 ? (int)std::min<int64_t>(rl.n_heavy, (int64_t)c->sm_count * 8) : 0;
  if (c->cfg.loop == MIS2_LOOP_DEVICE) {
    // every round in one cooperative launch (all blocks resident)
    auto kern = pack ? k_color_loop<G, true, I> : k_color_loop<G, false, I>;
    int per_sm = 0;
    MIS2_TRY(resident_blocks_per_sm(c, (const void*)kern, kBlock, &per_sm));
    if (per_sm < 1) return MIS2_ERR_CUDA;
    const int want = c->cfg.loop_blocks_per_sm > 0 ? c->cfg.loop_blocks_per_sm : 6;
    const int blocks = c->sm_count * std::min(per_sm, want);
    MIS2_CUDA(cudaMemsetAsync(left, 0, 3 * sizeof(int32_t), st));
    MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrBarrier, 0, sizeof(int32_t), st));
    MIS2_CUDA(cudaMemsetAsync(s.ctr + kCtrErr, 0, sizeof(int32_t), st));
    const int64_t spin = c->cfg.spin_limit;
    const int32_t max_rounds = (int32_t)std::min<int64_t>(gv.n, (int64_t)1 << 30);
    const int32_t extra = (c->cfg.debug_checks & MIS2_DEBUG_FORCE_TIMEOUT) ? 1 : 0;  // test hook: the waits run out
    // cooperative launch through the typed form: the arguments are checked
    // against the kernel's parameters at compile time
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(blocks);
    lc.blockDim = dim3(kBlock);
    lc.dynamicSmemBytes = 0;
    lc.stream = st;
    lc.attrs = attr;
    lc.numAttrs = 1;
    auto launch = [&]() {
      return cudaLaunchKernelEx(&lc, kern, gv, light_max, (const uint32_t*)prio, colors, when, resume, mlo, mhi,
                                (const int32_t*)rl.medium, rl.n_medium_dev, (const int32_t*)rl.heavy, rl.n_heavy_dev,
                                s.ctr, maxc, spin, max_rounds, extra);
    };
    if (c->coop_lock != nullptr) {
      std::lock_guard<std::mutex> lk(*c->coop_lock);
      MIS2_CUDA(launch());
      MIS2_CUDA(cudaEventRecord(c->coop_done, st));
      MIS2_CUDA(cudaEventSynchronize(c->coop_done));
    } else {
      MIS2_CUDA(launch());
    }
    c->launches++;
    MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    if (c->h_ctr[kCtrErr] & kErrTimeout) return MIS2_ERR_TIMEOUT;
    if (c->h_ctr[kCtrErr] & kErrNoProgress) return MIS2_ERR_NO_PROGRESS;
    *rounds = c->h_ctr[kCtrRounds];
    *n_colors = c->h_ctr[kCtrM2] + 1;
    return MIS2_OK;
  }
  for (int32_t r0 = 0;; r0 += kColorBatch) {
    if (r0 > gv.n) return MIS2_ERR_NO_PROGRESS;
    MIS2_CUDA(cudaMemsetAsync(left, 0, kColorBatch * sizeof(int32_t), st));
    for (int b = 0; b < kColorBatch; b++) {
      if (pack)
        k_color_round<G, true, I><<<wb, kBlock, 0, st>>>(gv, light_max, prio, colors, when, resume, mlo, mhi,
                                                          r0 + b, left + b, maxc);
      else
        k_color_round<G, false, I><<<wb, kBlock, 0, st>>>(gv, light_max, prio, colors, when, resume, mlo, mhi,
                                                           r0 + b, left + b, maxc);
      c->launches++;
      if (mb > 0) {
        k_color_medium<I><<<mb, kBlock, 0, st>>>(gv, rl.medium, rl.n_medium_dev, prio, colors, when, resume, r0 + b,
                                                  left + b, maxc);
        c->launches++;
      }
      if (hb > 0) {
        k_color_heavy<I><<<hb, kBlock, 0, st>>>(gv, rl.heavy, rl.n_heavy_dev, prio, colors, when, resume, r0 + b,
                                                 left + b, maxc);
        c->launches++;
      }
    }
    MIS2_CUDA(cudaGetLastError());
    MIS2_CUDA(cudaMemcpyAsync(c->h_ctr + kCtrM2, s.ctr + kCtrM2, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaMemcpyAsync(c->h_ctr + kCtrColorLeft, left, kColorBatch * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < kColorBatch; b++)
      if (c->h_ctr[kCtrColorLeft + b] == 0) {
        *rounds = r0 + b + 1;
        *n_colors = c->h_ctr[kCtrM2] + 1;
        return MIS2_OK;
      }
  }
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
  return avg < 40.0 ? color_rounds_t<4, I>(c, gv, g, p, colors, st, rounds, n_colors)
                    : color_rounds_t<32, I>(c, gv, g, p, colors, st, rounds, n_colors);
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
