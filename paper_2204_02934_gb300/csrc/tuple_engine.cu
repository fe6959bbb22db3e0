// tuple_engine.cu -- Algorithm 1 through a plain engine, for the ablation of
// the packed status tuple (Section V-C; Fig. 2 measures the packing against
// unpacked tuples): host-driven rounds, ordered worklists rebuilt by
// compaction every round, G lanes per row.  The status tuple is either
// packed in one 32-bit word (Eq. 1) or unpacked as (status, priority, vertex
// id) in separate arrays compared field by field, with the packed tuple's
// 32 - b priority bits as priority.  Everything but the tuple is shared, so
// the two times isolate the packing.  Both variants compute exactly
// mis2_run's MIS-2.
#include "internal.h"

namespace mis2 {

namespace {

// Eq. 1's packed tuple: IN = 0 < undecided (priority << b | v + 1) < OUT.
struct PackedTuples {
  using V = uint32_t;
  uint32_t* T;
  uint32_t* M;
  __device__ __forceinline__ V t(int64_t w) const { return T[w]; }
  __device__ __forceinline__ V m(int64_t w) const { return M[w]; }
  __device__ __forceinline__ void set_t(int64_t v, V x) const { T[v] = x; }
  __device__ __forceinline__ void set_m(int64_t v, V x) const { M[v] = x; }
  __device__ __forceinline__ static V fresh(const PrioCfg& p, uint32_t iter, int64_t v) {
    return make_tuple(p, iter, (uint32_t)v);
  }
  __device__ __forceinline__ static bool undecided(V x) { return x != kIn && x != kOut; }
  __device__ __forceinline__ static bool is_in(V x) { return x == kIn; }
  __device__ __forceinline__ static bool is_out(V x) { return x == kOut; }
  __device__ __forceinline__ static V in() { return kIn; }
  __device__ __forceinline__ static V out() { return kOut; }
  __device__ __forceinline__ static bool lt(V a, V b) { return a < b; }
  __device__ __forceinline__ static bool eq(V a, V b) { return a == b; }
  template <int G>
  __device__ __forceinline__ static V gmin(V x) {
    return group_min<G>(x);
  }
};

// The unpacked tuple: status (0 IN, 1 undecided, 2 OUT; one byte), priority
// (32 bits) and vertex id in separate arrays.  A vertex's own tuple carries
// its own id, so T stores status and priority only; M stores all three.
struct UnpackedTuples {
  struct V {
    uint32_t s, p, i;
  };
  uint8_t* Ts;
  uint32_t* Tp;
  uint8_t* Ms;
  uint32_t* Mp;
  uint32_t* Mi;
  __device__ __forceinline__ V t(int64_t w) const { return V{Ts[w], Tp[w], (uint32_t)w}; }
  __device__ __forceinline__ V m(int64_t w) const { return V{Ms[w], Mp[w], Mi[w]}; }
  __device__ __forceinline__ void set_t(int64_t v, V x) const {
    Ts[v] = (uint8_t)x.s;
    Tp[v] = x.p;
  }
  __device__ __forceinline__ void set_m(int64_t v, V x) const {
    Ms[v] = (uint8_t)x.s;
    Mp[v] = x.p;
    Mi[v] = x.i;
  }
  __device__ __forceinline__ static V fresh(const PrioCfg& p, uint32_t iter, int64_t v) {
    uint64_t h;
    if (p.variant == MIS2_HASH_XORSHIFT) {
      h = xorshift64(xorshift64((uint64_t)iter) ^ xorshift64((uint64_t)v) ^ p.seed);
    } else {
      const uint64_t it = p.variant == MIS2_HASH_FIXED ? 0ull : (uint64_t)iter;
      h = xorshift_star64(xorshift_star64(it) ^ xorshift_star64((uint64_t)v) ^ p.seed);
    }
    // the 32 - b priority bits of Eq. 1's packed tuple (b = p.b): the same
    // order as the packed form, kept in a field of its own
    const uint32_t prio = p.b >= 32 ? 0u : (uint32_t)(h & ((1ull << (32 - p.b)) - 1ull));
    return V{1u, prio, (uint32_t)v};
  }
  __device__ __forceinline__ static bool undecided(V x) { return x.s == 1u; }
  __device__ __forceinline__ static bool is_in(V x) { return x.s == 0u; }
  __device__ __forceinline__ static bool is_out(V x) { return x.s == 2u; }
  __device__ __forceinline__ static V in() { return V{0u, 0u, 0u}; }
  __device__ __forceinline__ static V out() { return V{2u, 0xFFFFFFFFu, 0xFFFFFFFFu}; }
  __device__ __forceinline__ static bool lt(V a, V b) {
    if (a.s != b.s) return a.s < b.s;
    if (a.p != b.p) return a.p < b.p;
    return a.i < b.i;
  }
  __device__ __forceinline__ static bool eq(V a, V b) { return a.s == b.s && a.p == b.p && a.i == b.i; }
  template <int G>
  __device__ __forceinline__ static V gmin(V x) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const V y{__shfl_xor_sync(kFull, x.s, o), __shfl_xor_sync(kFull, x.p, o), __shfl_xor_sync(kFull, x.i, o)};
      if (lt(y, x)) x = y;
    }
    return x;
  }
};

// Row refresh: T_v = h(iter, v) for v in worklist 1 (list null: every v).
template <class TP>
__global__ void __launch_bounds__(kBlock) k_te_refresh(TP tp, PrioCfg p, uint32_t iter, const int32_t* wl,
                                                       int64_t cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += stride) {
    const int64_t v = wl ? wl[j] : j;
    tp.set_t(v, TP::fresh(p, iter, v));
  }
}

// Column: M_v = the smallest T over N[v], IN turned into OUT, for v in
// worklist 2.  G lanes per row.
template <int G, class TP, typename I>
__global__ void __launch_bounds__(kBlock) k_te_column(GraphView<I> g, TP tp, const int32_t* wl, int64_t cnt) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW; base < cnt; base += nw * RPW) {
    const int64_t j = base + sub;
    typename TP::V m = TP::out();
    int64_t v = -1;
    if (j < cnt) {
      v = wl ? wl[j] : j;
      if (lg == 0) m = tp.t(v);
      int64_t s, e;
      row_range(g, v, s, e);
      for (int64_t k = s + lg; k < e; k += G) {
        const typename TP::V x = tp.t(__ldg(g.colind + k));
        if (TP::lt(x, m)) m = x;
      }
    }
    m = TP::template gmin<G>(m);
    if (j < cnt && lg == 0) tp.set_m(v, TP::is_in(m) ? TP::out() : m);
  }
}

// Decide, for v in worklist 1: OUT if some M over N[v] is OUT, else IN if
// every one equals T_v.
template <int G, class TP, typename I>
__global__ void __launch_bounds__(kBlock) k_te_decide(GraphView<I> g, TP tp, const int32_t* wl, int64_t cnt) {
  constexpr int RPW = 32 / G;
  const int lane = lane_id(), lg = lane & (G - 1), sub = lane / G;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW; base < cnt; base += nw * RPW) {
    const int64_t j = base + sub;
    bool any_out = false, all_eq = true;
    int64_t v = -1;
    if (j < cnt) {
      v = wl ? wl[j] : j;
      const typename TP::V tv = tp.t(v);
      if (lg == 0) {
        const typename TP::V mv = tp.m(v);
        any_out = TP::is_out(mv);
        all_eq = TP::eq(mv, tv);
      }
      int64_t s, e;
      row_range(g, v, s, e);
      for (int64_t k = s + lg; k < e; k += G) {
        const typename TP::V mw = tp.m(__ldg(g.colind + k));
        any_out |= TP::is_out(mw);
        all_eq &= TP::eq(mw, tv);
      }
    }
    any_out = group_any<G>(any_out);
    all_eq = group_all<G>(all_eq);
    if (j < cnt && lg == 0) {
      if (any_out) tp.set_t(v, TP::out());
      else if (all_eq) tp.set_t(v, TP::in());
    }
  }
}

// Worklist flags for the next round: f1 = T undecided, f2 = M not OUT.
template <class TP>
__global__ void __launch_bounds__(kBlock) k_te_flags(int64_t n, TP tp, uint8_t* f1, uint8_t* f2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    f1[v] = TP::undecided(tp.t(v));
    f2[v] = !TP::is_out(tp.m(v));
  }
}

// The final statuses in Eq. 1's form (IN / OUT) in T, for the root list.
__global__ void __launch_bounds__(kBlock) k_te_final(int64_t n, const uint8_t* Ts, uint32_t* T) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    T[v] = Ts[v] == 0 ? kIn : kOut;
}

template <int G, class TP, typename I>
int te_rounds(mis2_ctx* c, const GraphView<I>& gv, const PrioCfg& p, const TP& tp, cudaStream_t st,
              int32_t* rounds) {
  Scratch& s = c->s;
  uint8_t* f1 = reinterpret_cast<uint8_t*>(s.left);
  uint8_t* f2 = reinterpret_cast<uint8_t*>(s.left_heavy);
  int32_t* wl1 = s.roots2;
  int32_t* wl2 = s.qlist;
  const int rb = grid_for(c, gv.n, kBlock);
  const int wb = grid_for(c, gv.n, kBlock / 32 * (32 / G));
  const int32_t* l1 = nullptr;  // round 0: every vertex in both lists
  const int32_t* l2 = nullptr;
  int64_t n1 = gv.n, n2 = gv.n;
  for (int32_t r = 0;; r++) {
    if (r > gv.n) return MIS2_ERR_NO_PROGRESS;
    k_te_refresh<TP><<<rb, kBlock, 0, st>>>(tp, p, (uint32_t)r, l1, n1);
    if (n2 > 0) k_te_column<G, TP, I><<<wb, kBlock, 0, st>>>(gv, tp, l2, n2);
    k_te_decide<G, TP, I><<<wb, kBlock, 0, st>>>(gv, tp, l1, n1);
    k_te_flags<TP><<<rb, kBlock, 0, st>>>(gv.n, tp, f1, f2);
    c->launches += 4;
    MIS2_CUDA(cudaGetLastError());
    MIS2_TRY(compact_flags(c, f1, nullptr, gv.n, wl1, s.ctr + kCtrRoots, st));
    MIS2_TRY(compact_flags(c, f2, nullptr, gv.n, wl2, s.ctr + kCtrM2, st));
    MIS2_CUDA(cudaMemcpyAsync(c->h_ctr, s.ctr, kReadbackWords * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MIS2_CUDA(cudaStreamSynchronize(st));
    n1 = c->h_ctr[kCtrRoots];
    n2 = c->h_ctr[kCtrM2];
    l1 = wl1;
    l2 = wl2;
    if (n1 == 0) {
      *rounds = r + 1;
      return MIS2_OK;
    }
  }
}

template <typename I>
int te_t(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, bool unpacked, cudaStream_t st, int32_t* rounds) {
  GraphView<I> gv;
  gv.rowptr = static_cast<const I*>(g.rowptr);
  gv.colind = g.colind;
  gv.n = g.n;
  gv.nnz = g.nnz;
  gv.vec = g.vec ? 1 : 0;
  gv.pad = 0;
  Scratch& s = c->s;
  const bool narrow = g.n > 0 && (double)g.nnz / (double)g.n < 40.0;
  if (!unpacked) {
    const PackedTuples tp{s.T, s.M};
    return narrow ? te_rounds<4>(c, gv, p, tp, st, rounds) : te_rounds<32>(c, gv, p, tp, st, rounds);
  }
  const UnpackedTuples tp{s.qflag, s.M, reinterpret_cast<uint8_t*>(s.aggsize), reinterpret_cast<uint32_t*>(s.tent),
                          reinterpret_cast<uint32_t*>(s.members)};
  const int rc = narrow ? te_rounds<4>(c, gv, p, tp, st, rounds) : te_rounds<32>(c, gv, p, tp, st, rounds);
  if (rc != MIS2_OK) return rc;
  k_te_final<<<grid_for(c, g.n, kBlock), kBlock, 0, st>>>(g.n, s.qflag, s.T);
  c->launches++;
  MIS2_CUDA(cudaGetLastError());
  return MIS2_OK;
}

}  // namespace

int tuple_engine_impl(mis2_ctx* c, const GraphArgs& g, const PrioCfg& p, bool unpacked, uint8_t* in_set,
                      int32_t* roots, int64_t* n_roots, int32_t* n_rounds, cudaStream_t st) {
  int32_t r = 0;
  if (g.n > 0) MIS2_TRY(g.rp64 ? te_t<int64_t>(c, g, p, unpacked, st, &r) : te_t<int32_t>(c, g, p, unpacked, st, &r));
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
