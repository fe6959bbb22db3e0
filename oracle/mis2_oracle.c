/*
 * mis2_oracle.c -- plain, single-threaded CPU oracle for MIS-2, MIS-2
 * aggregation and the coarse (quotient) graph.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the yardstick the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * and reference legs of the benchmark may load it.  It shares no code with the CUDA path:
 * every constant and helper below is written out here on its own.
 *
 * It follows the paper (Kelley & Rajamanickam, "Parallel, Portable
 * Algorithms for Distance-2 Maximal Independent Set and Graph Coarsening"):
 *
 *   oracle_mis2       Algorithm 1 (Section III-A), with the hashed priority
 *                     h(iter, v) = f(f(iter) xor f(v)) of Section V-A and the
 *                     packed status tuple of Section V-C, Eq. 1.
 *   oracle_aggregate  Algorithm 3 (Section III-B), and Algorithm 2 as the
 *                     BASIC mode.
 *   oracle_coarsen    the coarse graph A_c of Algorithm 4's setup (Section
 *                     III-C): one vertex per aggregate, an edge wherever two
 *                     aggregates are joined by a fine edge.
 *   oracle_coarse_weights, oracle_prolongator
 *                     the off-diagonal of P^T A P and the tentative
 *                     prolongator (Section III-B, the step after coarsening).
 *   oracle_misk       distance-k MIS, Algorithm 1 generalised (Section II).
 *   oracle_mis2_unpacked
 *                     Algorithm 1 with unpacked (status, priority, id)
 *                     tuples (what Section V-C's packing is measured against).
 *   oracle_color_greedy
 *                     the colouring of Algorithm 4's setup: first fit in
 *                     ascending round-0 tuple order.
 *
 * Every function is pinned by tests to something other than itself (the
 * worked example of Fig. 1, brute-force definitions, scipy's sparse
 * products, equality with another function where the paper says they
 * agree); none is parity-unpinned.
 *
 * Readings where the paper is silent (they bind the CUDA path too):
 *   - adj(v) in the column and decide steps is the CLOSED neighbourhood
 *     N[v] = N(v) + {v}: Fig. 1 shows M_1 = T_1 although vertex 1's only
 *     neighbour has a larger tuple.
 *   - decide: "if some M_w = OUT then OUT, else if every M_w = T_v then IN",
 *     both tests on the tuple T_v held before the step (Fig. 1, round 2).
 *   - f is xorshift64* (Vigna 2016: shifts 12, 25, 27, multiplier
 *     0x2545F4914F6CDD1D); Table I's plain "Xor" hash is the same xorshift
 *     stage without the multiply (Section V-A describes xorshift* as
 *     xorshift followed by a linear congruential step).  Eq. 1's
 *     (priority << b) | (id + 1) is evaluated in the 32-bit status word,
 *     so the priority is the hash truncated to 32 bits whose low 32-b bits
 *     survive the shift.  A caller seed is xored into the inner term (seed
 *     0 = the paper's formula).  iter restarts at 0 for every MIS-2.
 *   - phase 2 runs MIS-2 on the subgraph induced by the unaggregated
 *     vertices, in the original numbering (b from the full n); other
 *     vertices are absent from it (neither relay nor block).
 *   - phase-2 roots need >= 2 unaggregated neighbours u != v.
 *   - phase 3 ties: max coupling, then min tentative size, then min id.
 *   - aggregates are numbered phase-1 roots ascending, then qualifying
 *     phase-2 roots ascending.
 *   - coarse rows are ascending, unique, without the diagonal.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_IN 0u
#define ORC_OUT 0xFFFFFFFFu

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = -1,
  ORC_ERR_NOMEM = -2,
  ORC_ERR_NOT_MIS2 = -4,
  ORC_ERR_NO_PROGRESS = -6
};

/* hash variants for the priority ablation of Section V-A, Table I */
enum { ORC_HASH_XORSHIFT_STAR = 0, ORC_HASH_XORSHIFT = 1, ORC_HASH_FIXED = 2 };

/* ------------------------------------------------------------ priorities */

/* Marsaglia's 64-bit xorshift with Vigna's (12, 25, 27) triple, followed by
 * the multiplicative step of xorshift64* (Vigna, ACM TOMS 42(4), 2016). */
static uint64_t orc_xorshift_star(uint64_t x) {
  x ^= x >> 12;
  x ^= x << 25;
  x ^= x >> 27;
  return x * 2685821657736338717ull;
}

/* Plain 64-bit xorshift: the xorshift stage of xorshift64* above without
 * its multiplicative step (Section V-A: xorshift* is xorshift followed by a
 * linear congruential step), the "Xor Hash" column of Table I. */
static uint64_t orc_xorshift(uint64_t x) {
  x ^= x >> 12;
  x ^= x << 25;
  x ^= x >> 27;
  return x;
}

/* h(iter, v) = f(f(iter) xor f(v)) (Section V-A); seed xored in. */
static uint64_t orc_hash(int variant, uint64_t iter, uint64_t v, uint64_t seed) {
  if (variant == ORC_HASH_XORSHIFT)
    return orc_xorshift(orc_xorshift(iter) ^ orc_xorshift(v) ^ seed);
  if (variant == ORC_HASH_FIXED) iter = 0; /* priorities drawn once */
  return orc_xorshift_star(orc_xorshift_star(iter) ^ orc_xorshift_star(v) ^ seed);
}

/* b = ceil(log2(|V| + 2)) id bits (Section V-C). */
int oracle_id_bits(int64_t n) {
  int b = 0;
  while (((uint64_t)1 << b) < (uint64_t)n + 2u) b++;
  return b;
}

/* Eq. 1 packing in the 32-bit status word: (priority << b) | (id + 1) with
 * priority = the hash truncated to 32 bits, so its low 32-b bits remain. */
uint32_t oracle_priority_bits(uint64_t hash, int b) {
  if (b >= 32) return 0u;
  return (uint32_t)(hash & ((((uint64_t)1) << (32 - b)) - 1u));
}

uint32_t oracle_pack(uint64_t hash, int64_t v, int b) {
  uint32_t hi = b >= 32 ? 0u : (oracle_priority_bits(hash, b) << b);
  return hi | (uint32_t)(v + 1);
}

/* The 64-bit hash h(iter, v) itself (exported for the tests that pin f). */
uint64_t oracle_hash(int variant, uint64_t iter, int64_t v, uint64_t seed) {
  return orc_hash(variant, iter, (uint64_t)v, seed);
}

uint32_t oracle_priority_tuple(int variant, uint64_t iter, int64_t v, int64_t n, uint64_t seed) {
  return oracle_pack(orc_hash(variant, iter, (uint64_t)v, seed), v, oracle_id_bits(n));
}

/* ------------------------------------------------------------ Algorithm 1 */

/*
 * MIS-2 of the subgraph induced by {v : member[v]} (all vertices when member
 * is NULL).  rowptr int64[n+1], colind int32[nnz]; self-loops and duplicate
 * entries are allowed.
 *
 * prio_table (test hook for the worked example of Fig. 1): when non-NULL,
 * round r uses priority prio_table[r*n + v] instead of the hash, for
 * r < table_rounds, and the hash after that.
 *
 * trace (optional, int64[4*trace_cap]): per round W1 = |worklist1|,
 * W2 = |worklist2|, D1 = sum of row lengths over worklist1 and D2 over
 * worklist2, taken at the start of the round.
 *
 * snaps (optional, uint32[3*n*snap_cap]): for round r < snap_cap, T after
 * the row refresh, M after the column step and T after the decide step, at
 * snaps[(3r + 0|1|2) * n].  Entries never written hold OUT.
 *
 * Outputs: in_set[v] = 1 iff T_v = IN at the end; *n_rounds = iterations.
 */
int oracle_mis2_snap(int64_t n, const int64_t* rowptr, const int32_t* colind, uint64_t seed,
                     int hash_variant, const uint8_t* member, const uint32_t* prio_table,
                     int64_t table_rounds, uint8_t* in_set, int32_t* n_rounds, int64_t* trace,
                     int64_t trace_cap, uint32_t* snaps, int64_t snap_cap) {
  if (n < 0 || (n > 0 && (!rowptr || !colind || !in_set))) return ORC_ERR_ARG;
  const int b = oracle_id_bits(n);
  uint32_t* T = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
  uint32_t* M = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
  int64_t* worklist1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* worklist2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!T || !M || !worklist1 || !worklist2) {
    free(T); free(M); free(worklist1); free(worklist2);
    return ORC_ERR_NOMEM;
  }
  /* worklist1 <- worklist2 <- 0..|V| (restricted to the subgraph) */
  int64_t w1 = 0, w2 = 0;
  for (int64_t v = 0; v < n; v++) {
    T[v] = ORC_OUT;
    M[v] = ORC_OUT;
    if (member && !member[v]) continue;
    worklist1[w1++] = v;
    worklist2[w2++] = v;
  }
  int64_t iter = 0;
  int rc = ORC_OK;
  while (w1 > 0) {
    if (iter > n) { rc = ORC_ERR_NO_PROGRESS; break; }
    if (trace && iter < trace_cap) {
      int64_t d1 = 0, d2 = 0;
      for (int64_t i = 0; i < w1; i++) d1 += rowptr[worklist1[i] + 1] - rowptr[worklist1[i]];
      for (int64_t i = 0; i < w2; i++) d2 += rowptr[worklist2[i] + 1] - rowptr[worklist2[i]];
      trace[4 * iter + 0] = w1;
      trace[4 * iter + 1] = w2;
      trace[4 * iter + 2] = d1;
      trace[4 * iter + 3] = d2;
    }
    /* Refresh row status: T_v <- h(iter, v) | v+1 */
    for (int64_t i = 0; i < w1; i++) {
      int64_t v = worklist1[i];
      if (prio_table && iter < table_rounds) {
        uint32_t prio = prio_table[iter * n + v];
        T[v] = (b >= 32 ? 0u : (prio << b)) | (uint32_t)(v + 1);
      } else {
        T[v] = oracle_pack(orc_hash(hash_variant, (uint64_t)iter, (uint64_t)v, seed), v, b);
      }
    }
    /* Refresh column status: M_v <- min(T_w : w in adj[v]); IN -> OUT */
    for (int64_t i = 0; i < w2; i++) {
      int64_t v = worklist2[i];
      uint32_t m = T[v];
      for (int64_t k = rowptr[v]; k < rowptr[v + 1]; k++) {
        int64_t w = colind[k];
        if (member && !member[w]) continue;
        if (T[w] < m) m = T[w];
      }
      if (m == ORC_IN) m = ORC_OUT;
      M[v] = m;
    }
    if (snaps && iter < snap_cap) {
      memcpy(snaps + (3 * iter + 0) * n, T, sizeof(uint32_t) * (size_t)n);
      memcpy(snaps + (3 * iter + 1) * n, M, sizeof(uint32_t) * (size_t)n);
    }
    /* Decide IN/OUT of set */
    for (int64_t i = 0; i < w1; i++) {
      int64_t v = worklist1[i];
      const uint32_t t = T[v];
      int any_out = (M[v] == ORC_OUT);
      int all_eq = (M[v] == t);
      for (int64_t k = rowptr[v]; k < rowptr[v + 1]; k++) {
        int64_t w = colind[k];
        if (member && !member[w]) continue;
        if (M[w] == ORC_OUT) any_out = 1;
        if (M[w] != t) all_eq = 0;
      }
      if (any_out)
        T[v] = ORC_OUT;
      else if (all_eq)
        T[v] = ORC_IN;
    }
    if (snaps && iter < snap_cap) memcpy(snaps + (3 * iter + 2) * n, T, sizeof(uint32_t) * (size_t)n);
    /* Compact worklists (order preserved) */
    int64_t nw1 = 0, nw2 = 0;
    for (int64_t i = 0; i < w1; i++)
      if (T[worklist1[i]] != ORC_IN && T[worklist1[i]] != ORC_OUT) worklist1[nw1++] = worklist1[i];
    for (int64_t i = 0; i < w2; i++)
      if (M[worklist2[i]] != ORC_OUT) worklist2[nw2++] = worklist2[i];
    w1 = nw1;
    w2 = nw2;
    iter++;
  }
  for (int64_t v = 0; v < n; v++) in_set[v] = (uint8_t)(T[v] == ORC_IN);
  if (n_rounds) *n_rounds = (int32_t)iter;
  free(T); free(M); free(worklist1); free(worklist2);
  return rc;
}

int oracle_mis2(int64_t n, const int64_t* rowptr, const int32_t* colind, uint64_t seed,
                int hash_variant, const uint8_t* member, const uint32_t* prio_table,
                int64_t table_rounds, uint8_t* in_set, int32_t* n_rounds, int64_t* trace,
                int64_t trace_cap) {
  return oracle_mis2_snap(n, rowptr, colind, seed, hash_variant, member, prio_table, table_rounds,
                          in_set, n_rounds, trace, trace_cap, NULL, 0);
}

/*
 * Algorithm 1 with the status tuple left unpacked (the variant Section V-C's
 * packing is measured against, Fig. 2): T_v = (status, priority, id) with
 * status IN < UNDECIDED < OUT, priority = the same 32-b hash bits that Eq. 1
 * packs (so both forms order undecided vertices alike and reach the same
 * set: the packing changes the representation, not the result), id = v,
 * compared field by field.  The round structure is Algorithm 1's: row
 * refresh of the undecided vertices, column = the smallest tuple of the
 * closed neighbourhood with IN turned into OUT, decide = OUT if some
 * neighbour's column tuple is OUT, else IN if every one equals T_v.  Every
 * vertex is visited each round; a decided vertex keeps its status and a
 * column tuple that is OUT stays OUT, so this is the worklist version's
 * result.  Self-loops and duplicate entries are harmless.
 */
typedef struct {
  int status; /* 0 IN, 1 UNDECIDED, 2 OUT */
  uint32_t prio;
  int64_t id;
} orc_tuple;

static int orc_tuple_lt(orc_tuple a, orc_tuple b) {
  if (a.status != b.status) return a.status < b.status;
  if (a.prio != b.prio) return a.prio < b.prio;
  return a.id < b.id;
}

static int orc_tuple_eq(orc_tuple a, orc_tuple b) {
  return a.status == b.status && a.prio == b.prio && a.id == b.id;
}

int oracle_mis2_unpacked(int64_t n, const int64_t* rowptr, const int32_t* colind, uint64_t seed, int hash_variant,
                         uint8_t* in_set, int32_t* n_rounds) {
  if (n < 0 || (n > 0 && (!rowptr || !colind || !in_set))) return ORC_ERR_ARG;
  orc_tuple* T = (orc_tuple*)malloc(sizeof(orc_tuple) * (size_t)(n + 1));
  orc_tuple* M = (orc_tuple*)malloc(sizeof(orc_tuple) * (size_t)(n + 1));
  orc_tuple* Tn = (orc_tuple*)malloc(sizeof(orc_tuple) * (size_t)(n + 1));
  if (!T || !M || !Tn) { free(T); free(M); free(Tn); return ORC_ERR_NOMEM; }
  const orc_tuple out = {2, 0xFFFFFFFFu, INT64_MAX};
  const int b = oracle_id_bits(n);
  for (int64_t v = 0; v < n; v++) T[v].status = 1;
  int64_t iter = 0, undecided = n;
  int rc = ORC_OK;
  while (undecided > 0) {
    if (iter > n) { rc = ORC_ERR_NO_PROGRESS; break; }
    /* refresh row */
    for (int64_t v = 0; v < n; v++)
      if (T[v].status == 1) {
        T[v].prio = oracle_priority_bits(orc_hash(hash_variant, (uint64_t)iter, (uint64_t)v, seed), b);
        T[v].id = v;
      }
    /* refresh column */
    for (int64_t v = 0; v < n; v++) {
      orc_tuple m = T[v];
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++)
        if (orc_tuple_lt(T[colind[e]], m)) m = T[colind[e]];
      M[v] = m.status == 0 ? out : m;
    }
    /* decide */
    for (int64_t v = 0; v < n; v++) {
      Tn[v] = T[v];
      if (T[v].status != 1) continue;
      int any_out = M[v].status == 2, all_eq = orc_tuple_eq(M[v], T[v]);
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
        const orc_tuple mw = M[colind[e]];
        if (mw.status == 2) any_out = 1;
        if (!orc_tuple_eq(mw, T[v])) all_eq = 0;
      }
      if (any_out) Tn[v] = out;
      else if (all_eq) Tn[v].status = 0;
    }
    undecided = 0;
    for (int64_t v = 0; v < n; v++) {
      T[v] = Tn[v];
      undecided += T[v].status == 1;
    }
    iter++;
  }
  for (int64_t v = 0; v < n; v++) in_set[v] = (uint8_t)(T[v].status == 0);
  if (n_rounds) *n_rounds = (int32_t)iter;
  free(T);
  free(M);
  free(Tn);
  return rc;
}

/* ------------------------------------------------------------ Algorithm 3 */

/*
 * Aggregation.  in_set = the phase-1 MIS-2 (flags).  mode 0 = Algorithm 3
 * (phases 1, 2, 3), mode 1 = Algorithm 2 (phase 1, then each leftover joins
 * a neighbouring aggregate by the phase-3 rule).  labels int32[n] receive
 * aggregate ids in [0, *n_aggs).  The phase-2 MIS-2 uses the same seed and
 * hash; its round count goes to *n_rounds2 and its per-round trace to
 * trace2 when given.  *n_phase1 receives the number of phase-1 aggregates.
 */
int oracle_aggregate(int64_t n, const int64_t* rowptr, const int32_t* colind,
                     const uint8_t* in_set, uint64_t seed, int hash_variant, int mode,
                     int32_t* labels, int64_t* n_aggs, int64_t* n_phase1, int32_t* n_rounds2,
                     int64_t* trace2, int64_t trace_cap) {
  if (n < 0 || (n > 0 && (!rowptr || !colind || !in_set || !labels))) return ORC_ERR_ARG;
  if (n_rounds2) *n_rounds2 = 0;
  for (int64_t v = 0; v < n; v++) labels[v] = -1;
  int64_t k = 0;
  /* Phase 1: each MIS-2 vertex with its neighbours forms an aggregate */
  for (int64_t v = 0; v < n; v++) {
    if (!in_set[v]) continue;
    if (labels[v] != -1) return ORC_ERR_NOT_MIS2;
    labels[v] = (int32_t)k;
    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
      int64_t u = colind[e];
      if (u == v || labels[u] == (int32_t)k) continue; /* self-loop or duplicate entry */
      if (labels[u] != -1) return ORC_ERR_NOT_MIS2;       /* roots closer than 3 */
      labels[u] = (int32_t)k;
    }
    k++;
  }
  if (n_phase1) *n_phase1 = k;
  /* Phase 2: MIS-2 of G minus the aggregated vertices */
  if (mode == 0 && n > 0) {
    uint8_t* unagg = (uint8_t*)malloc((size_t)n);
    uint8_t* m2 = (uint8_t*)malloc((size_t)n);
    if (!unagg || !m2) { free(unagg); free(m2); return ORC_ERR_NOMEM; }
    for (int64_t v = 0; v < n; v++) unagg[v] = (uint8_t)(labels[v] == -1);
    int rc = oracle_mis2(n, rowptr, colind, seed, hash_variant, unagg, NULL, 0, m2, n_rounds2,
                         trace2, trace_cap);
    if (rc != ORC_OK) { free(unagg); free(m2); return rc; }
    for (int64_t v = 0; v < n; v++) {
      if (!m2[v]) continue;
      int64_t cnt = 0;
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
        int64_t u = colind[e];
        if (u != v && unagg[u]) cnt++;
      }
      if (cnt < 2) continue; /* too small: left for phase 3 */
      labels[v] = (int32_t)k;
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
        int64_t u = colind[e];
        if (u != v && unagg[u]) labels[u] = (int32_t)k;
      }
      k++;
    }
    free(unagg);
    free(m2);
  }
  /* Phase 3: leftovers join the most strongly coupled aggregate, using the
   * tentative labels (frozen copy) for coupling and sizes. */
  int32_t* tent = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int64_t* aggsize = (int64_t*)calloc((size_t)(k + 1), sizeof(int64_t));
  int64_t* coupling = (int64_t*)calloc((size_t)(k + 1), sizeof(int64_t));
  if (!tent || !aggsize || !coupling) { free(tent); free(aggsize); free(coupling); return ORC_ERR_NOMEM; }
  for (int64_t v = 0; v < n; v++) tent[v] = labels[v];
  for (int64_t v = 0; v < n; v++)
    if (tent[v] >= 0) aggsize[tent[v]]++;
  int rc = ORC_OK;
  for (int64_t v = 0; v < n; v++) {
    if (tent[v] != -1) continue;
    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
      int64_t u = colind[e];
      if (u != v && tent[u] >= 0) coupling[tent[u]]++;
    }
    int64_t best = -1;
    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
      int64_t u = colind[e];
      if (u == v || tent[u] < 0) continue;
      int64_t a = tent[u];
      if (best < 0 || coupling[a] > coupling[best] ||
          (coupling[a] == coupling[best] &&
           (aggsize[a] < aggsize[best] || (aggsize[a] == aggsize[best] && a < best))))
        best = a;
    }
    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
      int64_t u = colind[e];
      if (u != v && tent[u] >= 0) coupling[tent[u]] = 0;
    }
    if (best < 0) { rc = ORC_ERR_NOT_MIS2; break; } /* not within distance 2 of a root */
    labels[v] = (int32_t)best;
  }
  free(tent);
  free(aggsize);
  free(coupling);
  if (n_aggs) *n_aggs = k;
  return rc;
}

/* ------------------------------------------------------------ coarse graph */

static int orc_cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Coarse graph: row A lists, ascending and once each, every aggregate B != A
 * that holds a fine neighbour of a member of A.  c_rowptr int64[n_aggs+1];
 * c_colind must hold *c_nnz entries: call with c_colind == NULL first to get
 * the size, then again with the buffer.
 */
int oracle_coarsen(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* labels,
                   int64_t n_aggs, int64_t* c_rowptr, int32_t* c_colind, int64_t* c_nnz) {
  if (n < 0 || n_aggs < 0 || !c_rowptr || (n > 0 && (!rowptr || !colind || !labels)))
    return ORC_ERR_ARG;
  for (int64_t v = 0; v < n; v++)
    if (labels[v] < 0 || labels[v] >= n_aggs) return ORC_ERR_ARG;
  /* members of each aggregate */
  int64_t* mptr = (int64_t*)calloc((size_t)(n_aggs + 1), sizeof(int64_t));
  int64_t* members = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* fill = (int64_t*)calloc((size_t)(n_aggs + 1), sizeof(int64_t));
  int64_t* seen = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_aggs + 1));
  int32_t* row = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_aggs + 1));
  if (!mptr || !members || !fill || !seen || !row) {
    free(mptr); free(members); free(fill); free(seen); free(row);
    return ORC_ERR_NOMEM;
  }
  for (int64_t v = 0; v < n; v++) mptr[labels[v] + 1]++;
  for (int64_t a = 0; a < n_aggs; a++) mptr[a + 1] += mptr[a];
  for (int64_t v = 0; v < n; v++) members[mptr[labels[v]] + fill[labels[v]]++] = v;
  for (int64_t a = 0; a < n_aggs; a++) seen[a] = -1;
  int64_t total = 0;
  c_rowptr[0] = 0;
  for (int64_t a = 0; a < n_aggs; a++) {
    int64_t len = 0;
    for (int64_t i = mptr[a]; i < mptr[a + 1]; i++) {
      int64_t u = members[i];
      for (int64_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
        int32_t bagg = labels[colind[e]];
        if (bagg == a || seen[bagg] == a) continue;
        seen[bagg] = a;
        row[len++] = bagg;
      }
    }
    qsort(row, (size_t)len, sizeof(int32_t), orc_cmp_i32);
    if (c_colind)
      for (int64_t i = 0; i < len; i++) c_colind[total + i] = row[i];
    total += len;
    c_rowptr[a + 1] = total;
  }
  if (c_nnz) *c_nnz = total;
  free(mptr); free(members); free(fill); free(seen); free(row);
  return ORC_OK;
}

/* ------------------------------------------------------------ Galerkin pieces */

/*
 * Weights of the coarse graph (the step after coarsen in a multilevel
 * method, Section III-B): for coarse row A and column B, the number of fine
 * entries (u, v) with labels[u] = A and labels[v] = B, u's row listing v.
 * These are the off-diagonal entries of P^T A P for the 0/1 adjacency A and
 * the 0/1 tentative prolongator P.  c_rowptr / c_colind as oracle_coarsen
 * returns them; each entry is located by a linear scan of its coarse row.
 */
int oracle_coarse_weights(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* labels,
                          int64_t n_aggs, const int64_t* c_rowptr, const int32_t* c_colind, int64_t* c_weights) {
  if (n < 0 || n_aggs < 0 || !c_rowptr || (n > 0 && (!rowptr || !colind || !labels))) return ORC_ERR_ARG;
  for (int64_t k = 0; k < c_rowptr[n_aggs]; k++) c_weights[k] = 0;
  for (int64_t u = 0; u < n; u++) {
    const int32_t a = labels[u];
    for (int64_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
      const int32_t b = labels[colind[e]];
      if (b == a) continue;
      int64_t k = c_rowptr[a];
      while (k < c_rowptr[a + 1] && c_colind[k] != b) k++;
      if (k == c_rowptr[a + 1]) return ORC_ERR_ARG; /* not the coarse graph of these labels */
      c_weights[k]++;
    }
  }
  return ORC_OK;
}

/*
 * Tentative prolongator of the aggregation (Section III-B: the coarse system
 * receives restricted residuals and its solution is interpolated back): P is
 * n x n_aggs with one entry per row, P[v, labels[v]] = 1, or
 * 1 / sqrt(|aggregate|) when normalize is set (orthonormal columns: the
 * smoothed-aggregation tentative prolongator for a constant near-null space).
 */
int oracle_prolongator(int64_t n, const int32_t* labels, int64_t n_aggs, int normalize, int32_t* p_colind,
                       double* p_values) {
  if (n < 0 || n_aggs < 0 || (n > 0 && (!labels || !p_colind || !p_values))) return ORC_ERR_ARG;
  int64_t* size = (int64_t*)calloc((size_t)(n_aggs + 1), sizeof(int64_t));
  if (!size) return ORC_ERR_NOMEM;
  for (int64_t v = 0; v < n; v++) {
    if (labels[v] < 0 || labels[v] >= n_aggs) {
      free(size);
      return ORC_ERR_ARG;
    }
    size[labels[v]]++;
  }
  for (int64_t v = 0; v < n; v++) {
    p_colind[v] = labels[v];
    p_values[v] = normalize ? 1.0 / sqrt((double)size[labels[v]]) : 1.0;
  }
  free(size);
  return ORC_OK;
}

/* ------------------------------------------------------------ MIS-k */

/*
 * Distance-k maximal independent set, the generalisation of Algorithm 1
 * (Section II: distance-k independence; Section III-A: the column step
 * spreads statuses one hop and decide reads one more hop, so k - 1 column
 * steps reach distance k).  Each round, on the statuses T of the round
 * (undecided vertices refreshed with h(iter, v) as in Algorithm 1), two
 * quantities spread hop by hop:
 *   B(j)_v = some IN vertex within distance j of v,
 *   P(j)_v = the smallest undecided tuple within distance j of v (OUT when
 *            none; IN and OUT vertices do not compete),
 * with B(0)_v = T_v is IN, P(0)_v = T_v if undecided (else OUT), and B(j),
 * P(j) the OR / min of B(j-1), P(j-1) over N[v].  An undecided v becomes OUT
 * if B(k)_v, else IN if P(k)_v = T_v: the last hop is the decide step, the
 * k - 1 before it the column steps.  All decisions of a round read the
 * statuses from before the round.  For k = 2 this is Algorithm 1 exactly: its
 * M_v = OUT stands for B(1)_v (the only other case, a neighbourhood decided
 * entirely OUT, never reaches an undecided vertex's decide, since that
 * vertex lies in the neighbourhood), and "every M_w equals T_v" is
 * P(2)_v = T_v because each such M_w is at most T_v.  For k >= 3 the two
 * have to stay apart: a neighbourhood decided entirely OUT blocks nothing.
 * Every vertex is visited every round.
 */
int oracle_misk(int64_t n, const int64_t* rowptr, const int32_t* colind, int k, uint64_t seed, int hash_variant,
                uint8_t* in_set, int32_t* n_rounds) {
  if (n < 0 || k < 1 || (n > 0 && (!rowptr || !colind || !in_set))) return ORC_ERR_ARG;
  const int b = oracle_id_bits(n);
  uint32_t* T = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
  uint32_t* Tn = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
  uint32_t* Pa = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
  uint32_t* Pb = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
  uint8_t* Ba = (uint8_t*)malloc((size_t)(n + 1));
  uint8_t* Bb = (uint8_t*)malloc((size_t)(n + 1));
  if (!T || !Tn || !Pa || !Pb || !Ba || !Bb) {
    free(T); free(Tn); free(Pa); free(Pb); free(Ba); free(Bb);
    return ORC_ERR_NOMEM;
  }
  for (int64_t v = 0; v < n; v++) T[v] = 1; /* any undecided value; refreshed below */
  int64_t iter = 0, undecided = n;
  int rc = ORC_OK;
  while (undecided > 0) {
    if (iter > n) { rc = ORC_ERR_NO_PROGRESS; break; }
    for (int64_t v = 0; v < n; v++)
      if (T[v] != ORC_IN && T[v] != ORC_OUT)
        T[v] = oracle_pack(orc_hash(hash_variant, (uint64_t)iter, (uint64_t)v, seed), v, b);
    /* hop 0: B(0)_v = T_v is IN, P(0)_v = T_v if undecided, else OUT */
    for (int64_t v = 0; v < n; v++) {
      Ba[v] = (uint8_t)(T[v] == ORC_IN);
      Pa[v] = (T[v] == ORC_IN || T[v] == ORC_OUT) ? ORC_OUT : T[v];
    }
    for (int j = 1; j <= k - 1; j++) {
      for (int64_t v = 0; v < n; v++) {
        uint8_t bl = Ba[v];
        uint32_t m = Pa[v];
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
          bl |= Ba[colind[e]];
          if (Pa[colind[e]] < m) m = Pa[colind[e]];
        }
        Bb[v] = bl;
        Pb[v] = m;
      }
      uint8_t* tb = Ba; Ba = Bb; Bb = tb;
      uint32_t* tp = Pa; Pa = Pb; Pb = tp;
    }
    for (int64_t v = 0; v < n; v++) {
      Tn[v] = T[v];
      if (T[v] == ORC_IN || T[v] == ORC_OUT) continue;
      int blocked = Ba[v];
      uint32_t m = Pa[v];
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
        if (Ba[colind[e]]) blocked = 1;
        if (Pa[colind[e]] < m) m = Pa[colind[e]];
      }
      if (blocked) Tn[v] = ORC_OUT;
      else if (m == T[v]) Tn[v] = ORC_IN;
    }
    undecided = 0;
    for (int64_t v = 0; v < n; v++) {
      T[v] = Tn[v];
      undecided += (T[v] != ORC_IN && T[v] != ORC_OUT);
    }
    iter++;
  }
  for (int64_t v = 0; v < n; v++) in_set[v] = (uint8_t)(T[v] == ORC_IN);
  if (n_rounds) *n_rounds = (int32_t)iter;
  free(T); free(Tn); free(Pa); free(Pb); free(Ba); free(Bb);
  return rc;
}

/* ------------------------------------------------------------ coloring */

/*
 * Greedy (first-fit) distance-1 coloring of a graph in ascending order of
 * the vertices' round-0 tuples (Eq. 1 packing of h(0, v), so the order is
 * the one a parallel Jones-Plassmann pass with those priorities
 * reproduces): each vertex takes the smallest color no neighbour earlier in
 * the order holds.  Used on the coarse graph for the colour sets of cluster
 * multicolor Gauss-Seidel (Algorithm 4's setup).  Self-loops are ignored.
 * colors int32[n]; *n_colors = 1 + the largest color (0 when n = 0).
 */
static const uint32_t* orc_sort_key;
static int orc_cmp_by_key(const void* a, const void* b) {
  const uint32_t x = orc_sort_key[*(const int64_t*)a], y = orc_sort_key[*(const int64_t*)b];
  return x < y ? -1 : (x > y ? 1 : 0);
}

int oracle_color_greedy(int64_t n, const int64_t* rowptr, const int32_t* colind, uint64_t seed, int hash_variant,
                        int32_t* colors, int32_t* n_colors) {
  if (n < 0 || (n > 0 && (!rowptr || !colind || !colors))) return ORC_ERR_ARG;
  const int b = oracle_id_bits(n);
  uint32_t* prio = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n + 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  uint8_t* used = (uint8_t*)calloc((size_t)(n + 2), 1);
  if (!prio || !order || !used) {
    free(prio); free(order); free(used);
    return ORC_ERR_NOMEM;
  }
  for (int64_t v = 0; v < n; v++) {
    prio[v] = oracle_pack(orc_hash(hash_variant, 0, (uint64_t)v, seed), v, b);
    order[v] = v;
    colors[v] = -1;
  }
  orc_sort_key = prio;
  qsort(order, (size_t)n, sizeof(int64_t), orc_cmp_by_key);
  int32_t nc = 0;
  for (int64_t i = 0; i < n; i++) {
    const int64_t v = order[i];
    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++)
      if (colind[e] != v && colors[colind[e]] >= 0) used[colors[colind[e]]] = 1;
    int32_t c = 0;
    while (used[c]) c++;
    colors[v] = c;
    if (c + 1 > nc) nc = c + 1;
    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++)
      if (colind[e] != v && colors[colind[e]] >= 0) used[colors[colind[e]]] = 0;
  }
  if (n_colors) *n_colors = nc;
  free(prio); free(order); free(used);
  return ORC_OK;
}
