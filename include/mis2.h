/*
 * mis2.h -- C ABI of the GB300 (sm_103a) MIS-2 / aggregation / coarsening
 * library.
 *
 * The three calls follow the problem statement of Kelley & Rajamanickam,
 * "Parallel, Portable Algorithms for Distance-2 Maximal Independent Set and
 * Graph Coarsening" (arXiv 2204.02934):
 *
 *   mis2_run        Algorithm 1 (Section III-A): a distance-2 maximal
 *                   independent set of an undirected graph G = (V, E)
 *                   (Section I).  Returns the in-set flags and root list.
 *   mis2_aggregate  Algorithm 3 (Section III-B), or Algorithm 2 in BASIC
 *                   mode: one aggregate id per vertex.
 *   mis2_coarsen    the coarsened graph A_c with the vertex -> cluster map
 *                   (Section III-C, the setup of Algorithm 4).
 *
 * Conventions shared by every call
 *   - Graph input is CSR: rowptr (int32 or int64, n+1 entries) and colind
 *     (int32, nnz entries), both in DEVICE memory owned by the caller.  The
 *     graph must be symmetric (undirected, Section I); this is not checked
 *     unless debug_checks is set.  Self-loops are allowed everywhere.
 *     Duplicate entries are allowed in mis2_run (they change no minimum,
 *     "any" or "all" of Algorithm 1), but aggregation counts neighbours over
 *     the edge set (the ">= 2" test of phase 2, the coupling of phase 3), so
 *     rows passed to mis2_aggregate / mis2_coarsen_level must list each
 *     neighbour once.
 *   - Every output pointer is DEVICE memory owned by the caller unless
 *     marked "host".  The library owns only the scratch memory inside its
 *     context, sized at creation.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *     return a count through a host pointer synchronise that stream before
 *     returning; no other host synchronisation is performed.
 *   - Results are bit-identical run to run and independent of launch
 *     configuration (every phase is a per-vertex map over arrays written in
 *     earlier phases; counts use integer atomics).
 *   - A context is not thread-safe: use one context per host thread/stream.
 *   - Return value: MIS2_OK (0) or a negative mis2_status.  After
 *     MIS2_ERR_CUDA the CUDA error string is available through
 *     mis2_last_error().
 */
#ifndef MIS2_GB300_H
#define MIS2_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MIS2_OK = 0,
  MIS2_ERR_INVALID_ARG = -1,   /* NULL pointer, negative size, n >= 2^32 - 2, size above capacity */
  MIS2_ERR_OUT_OF_MEMORY = -2, /* context scratch too small, or cudaMalloc failed */
  MIS2_ERR_CUDA = -3,          /* a CUDA runtime call failed; see mis2_last_error() */
  MIS2_ERR_BAD_GRAPH = -4,     /* debug_checks: malformed CSR, or roots not an MIS-2 */
  MIS2_ERR_TIMEOUT = -5,       /* a device-side barrier gave up after spin_limit polls */
  MIS2_ERR_NO_PROGRESS = -6,   /* round cap (n + 1 rounds) reached */
  MIS2_ERR_CANCELLED = -7      /* serving: the request was cancelled before it started */
} mis2_status;

/* Aggregation modes. */
enum { MIS2_AGG_ALG3 = 0, MIS2_AGG_BASIC = 1 };

/* Priority hash variants (Section V-A, Table I): h(iter, v) = f(f(iter) ^
 * f(v) ^ seed).  XORSHIFT_STAR (the paper's choice and the default): f =
 * xorshift64*, shifts 12/25/27 then a multiply by 0x2545F4914F6CDD1D.
 * XORSHIFT: the same shifts without the multiply.  FIXED: xorshift64* with
 * iter held at 0 (priorities drawn once).  The priority of Eq. 1 is the
 * hash truncated to the 32-bit status word, shifted left by b: its low
 * 32 - b bits. */
enum { MIS2_HASH_XORSHIFT_STAR = 0, MIS2_HASH_XORSHIFT = 1, MIS2_HASH_FIXED = 2 };

/* Round-loop drivers: HOST reads the worklist size back after every round
 * (one stream synchronisation per round); DEVICE runs the whole round loop
 * inside one persistent cooperative kernel with grid-wide barriers. */
enum { MIS2_LOOP_HOST = 0, MIS2_LOOP_DEVICE = 1 };

typedef struct {
  int64_t n;            /* number of vertices, 0 <= n < 2^31 */
  int64_t nnz;          /* number of colind entries, 0 <= nnz < 2^31 */
  int32_t rowptr_is_64; /* 0: rowptr is int32_t[n+1]; 1: int64_t[n+1] */
  int32_t reserved;
  const void* rowptr;   /* device */
  const int32_t* colind;/* device, 4-byte aligned (16-byte alignment enables vector loads) */
} mis2_csr;

typedef struct {
  int32_t hash_variant;   /* MIS2_HASH_*; default XORSHIFT_STAR */
  int32_t agg_mode;       /* MIS2_AGG_*; default ALG3 */
  int32_t group_lanes;    /* lanes per low-degree row: 0 = pick from average degree, else 1,2,4,8,16,32 */
  int32_t warp_degree;    /* rows with degree >= this get a full warp; 0 (default) = 32 below an
                             average degree of 40, else 256 (capped by block_degree) */
  int32_t block_degree;   /* rows with degree >= this get a full block (default 2048) */
  int32_t block_size;     /* threads per block for row kernels (default 256) */
  int32_t loop;           /* MIS2_LOOP_*; default HOST (DEVICE: one persistent launch per MIS-2 or
                             colouring) */
  int32_t debug_checks;   /* MIS2_DEBUG_* bits (extra passes, synchronising); default 0 */
  int32_t timing;         /* MIS2_TIMING_*: CUDA-event times per kernel class into mis2_stats; default 0 */
  int32_t loop_blocks_per_sm; /* blocks per SM of the device-loop kernel: 0 = default (2) */
  int32_t ablation;       /* MIS2_ABLATE_* bits (the Fig. 2 variants); default 0 */
  int32_t serial_launches; /* 1: every kernel around the MIS-2 loops is scheduled only after the
                              previous one has finished; 0 (default): programmatic dependent
                              launch lets it be scheduled while that one finishes (same results) */
  int64_t spin_limit;     /* polls before a device barrier reports MIS2_ERR_TIMEOUT */
} mis2_config;

/* Per-call statistics of the last mis2_run / mis2_aggregate / mis2_coarsen /
 * mis2_coarsen_level on a context.  trace[r] = {W1, W2, D1, D2}: worklist
 * sizes and summed row lengths at the start of MIS-2 round r (phase-1 MIS-2
 * in trace, phase-2 MIS-2 in trace2), up to MIS2_TRACE_CAP rounds. */
/* debug_checks bits.
 * MIS2_DEBUG_VALIDATE: before computing, every entry point taking a graph
 *   checks rowptr (0 first, nnz last, non-decreasing), colind in [0, n) and
 *   symmetry (two order-independent 64-bit hash sums over the entries and
 *   over their mirrors must agree); mis2_aggregate also checks that the roots
 *   are ascending, in range and pairwise more than two hops apart, and
 *   mis2_coarsen that every label is in [0, n_aggs).  A failed check returns
 *   MIS2_ERR_BAD_GRAPH before any kernel indexes memory with the bad value.
 * MIS2_DEBUG_FORCE_TIMEOUT: test hook for the bounded waits: the grid
 *   barriers of the device loops (MIS-2 rounds, colouring rounds) wait for
 *   one arrival more than the grid makes, so every block gives up after
 *   spin_limit polls and the call returns MIS2_ERR_TIMEOUT; the context
 *   stays usable. */
/* ablation bits (Section VI-A, Fig. 2: the optimisations one at a time).
 * MIS2_ABLATE_NO_WORKLISTS: every round visits every vertex of the
 *   (sub)graph in both steps instead of the compacted worklists (decide skips
 *   vertices already IN or OUT); the result is the same MIS-2.  The fixed
 *   priorities and the xorshift hash of Fig. 2 / Table I are hash_variant
 *   values.  Per-round statistics then count the vertices visited. */
#define MIS2_ABLATE_NO_WORKLISTS 0x1
/* MIS2_ABLATE_TUPLE_ENGINE: mis2_run computes Algorithm 1 through a plain
 *   engine (host-driven rounds, worklists rebuilt by ordered compaction each
 *   round, G lanes per row) with the packed tuple of Eq. 1: the same MIS-2.
 * MIS2_ABLATE_UNPACKED_TUPLES: the same engine with the status tuple left
 *   unpacked (Section V-C's packing measured against, Fig. 2): status,
 *   priority and vertex id in separate arrays, compared field by field, the
 *   priority being the 32 - b bits Eq. 1 packs: the same order, so the same
 *   MIS-2 as the packed engine and mis2_run.
 * Both apply to mis2_run alone: mis2_run_with_priorities, mis2_aggregate,
 * mis2_coarsen_level(_host) and mis2_batch_create refuse a configuration
 * with either set (MIS2_ERR_INVALID_ARG). */
#define MIS2_ABLATE_TUPLE_ENGINE 0x2
#define MIS2_ABLATE_UNPACKED_TUPLES 0x4

/* timing values.
 * MIS2_TIMING_ALL: every kernel class is bracketed by CUDA events, the
 *   device loop stamps every grid barrier (loop_ns), and the kernels are
 *   launched one after another (serial_launches implied), so that each
 *   class's time is its own.
 * MIS2_TIMING_LOOP: only the device-loop MIS-2 launches (class 6) are
 *   bracketed by events; everything else runs as with timing off. */
#define MIS2_TIMING_OFF 0
#define MIS2_TIMING_ALL 1
#define MIS2_TIMING_LOOP 2

#define MIS2_DEBUG_VALIDATE 0x1
#define MIS2_DEBUG_FORCE_TIMEOUT 0x100

#define MIS2_TRACE_CAP 64
#define MIS2_LOOP_TS_WORDS (4 + 4 * MIS2_TRACE_CAP)
#define MIS2_NUM_KERNEL_CLASSES 8
typedef struct {
  int32_t rounds;           /* rounds of the phase-1 MIS-2 (Algorithm 1 loop count) */
  int32_t rounds2;          /* rounds of the phase-2 MIS-2 (0 in BASIC mode) */
  int64_t n_roots;          /* |MIS-2| */
  int64_t n_phase1;         /* phase-1 aggregates */
  int64_t n_aggs;           /* all aggregates */
  int64_t c_nnz;            /* coarse graph entries */
  int64_t trace[MIS2_TRACE_CAP][4];
  int64_t trace2[MIS2_TRACE_CAP][4];
  /* timing (config.timing != 0; MIS2_TIMING_LOOP: class 6 only): total ms
   * and launches per kernel class:
   * 0 init, 1 column, 2 decide, 3 roots/compaction, 4 aggregation,
   * 5 coarse graph, 6 device-loop MIS-2 kernel, 7 other */
  double kernel_ms[MIS2_NUM_KERNEL_CLASSES];
  int64_t kernel_launches[MIS2_NUM_KERNEL_CLASSES];
  int64_t launches;         /* CUDA kernels launched by the last call (always counted) */
  /* device loop with MIS2_TIMING_ALL: globaltimer ns of [0] block 0's start and [1]
   * the end of its round-0 set-up, then per
   * grid barrier b (b = 0 after set-up, 2r+1 after round r's column step,
   * 2r+2 after its decide step) the last block's arrival [2+2b] and block 0's
   * departure [3+2b]; one row per MIS-2 (phase-1, phase-2) */
  int64_t loop_ns[2][MIS2_LOOP_TS_WORDS];
} mis2_stats;

typedef struct mis2_ctx mis2_ctx;

/* Fill *cfg with the defaults listed above. */
void mis2_config_default(mis2_config* cfg);

/* Create a context whose scratch holds graphs of up to max_n vertices and
 * max_nnz entries (allocated now with cudaMalloc on the current device).
 * cfg may be NULL (defaults).  *ctx receives the handle; on failure *ctx is
 * NULL and nothing stays allocated. */
int mis2_ctx_create(mis2_ctx** ctx, int64_t max_n, int64_t max_nnz, const mis2_config* cfg);

/* Free a context and its scratch; NULL is ignored.  Synchronises the device. */
int mis2_ctx_destroy(mis2_ctx* ctx);

/* Replace the context's configuration (same validation as create). */
int mis2_ctx_set_config(mis2_ctx* ctx, const mis2_config* cfg);

/* Copy the statistics of the last call into *out (host). */
int mis2_get_stats(const mis2_ctx* ctx, mis2_stats* out);

/*
 * MIS-2 of `g` (Algorithm 1 with the hashed priority of Section V-A and the
 * packed tuples of Section V-C, Eq. 1).
 *   seed      xored into the hash; 0 gives the paper's h(iter, v).
 *   in_set    uint8[n], device: 1 for vertices in the MIS-2, else 0.  May be NULL.
 *   roots     int32[n] capacity, device: MIS-2 vertices ascending.  May be NULL.
 *   n_roots   host: |MIS-2|.  n_rounds: host, may be NULL.
 * Synchronises `stream`.
 */
int mis2_run(mis2_ctx* ctx, const mis2_csr* g, uint64_t seed, uint8_t* in_set, int32_t* roots,
             int64_t* n_roots, int32_t* n_rounds, void* stream);

/*
 * Test hook for the worked example of Fig. 1: like mis2_run, but round r
 * uses priority prio_table[r*n + v] (host, uint32, table_rounds * n
 * entries) instead of the hash for r < table_rounds.  Priorities must be
 * below 2^(32-b), b = ceil(log2(n+2)).
 */
int mis2_run_with_priorities(mis2_ctx* ctx, const mis2_csr* g, const uint32_t* prio_table,
                             int32_t table_rounds, uint8_t* in_set, int32_t* roots,
                             int64_t* n_roots, int32_t* n_rounds, void* stream);

/*
 * Test hook for the round-by-round values of Fig. 1 (Section III-A):
 * mis2_run_with_priorities, recording for every round r < snap_rounds three
 * copies of the status arrays into snaps (DEVICE, uint32, snap_rounds * 3 * n
 * entries, written by the call): [r][0] = T after round r's row refresh,
 * [r][1] = the column tuples M after its column step, [r][2] = T after its
 * decide step.  The row refresh of round r + 1 is fused into round r's
 * decide, so in [r][2] a vertex still undecided holds its next round's tuple:
 * there only IN (0), OUT (0xFFFFFFFF) and "undecided" are the step's result.
 * Rounds that did not run, and M of vertices the column step no longer
 * visits (their M stays OUT), read OUT.  Works with both round-loop drivers.
 */
int mis2_run_snapshots(mis2_ctx* ctx, const mis2_csr* g, const uint32_t* prio_table, int32_t table_rounds,
                       uint32_t* snaps, int32_t snap_rounds, uint8_t* in_set, int32_t* roots, int64_t* n_roots,
                       int32_t* n_rounds, void* stream);

/*
 * Aggregation (Algorithm 3, or Algorithm 2 when mode = MIS2_AGG_BASIC).
 *   roots     int32[n_roots], device, ascending: an MIS-2 of g (e.g. from mis2_run).
 *   labels    int32[n], device: aggregate id of each vertex, in [0, *n_aggs).
 *             Phase-1 aggregates are numbered by ascending root, then
 *             phase-2 aggregates by ascending root.
 *   n_aggs    host.
 * The phase-2 MIS-2 uses the same seed and restarts its round counter at 0.
 * Synchronises `stream`.
 */
int mis2_aggregate(mis2_ctx* ctx, const mis2_csr* g, const int32_t* roots, int64_t n_roots,
                   uint64_t seed, int32_t mode, int32_t* labels, int64_t* n_aggs, void* stream);

/*
 * Coarse graph of an aggregation: row A lists, ascending and once each,
 * every aggregate B != A holding a fine neighbour of a member of A.
 *   labels      int32[n], device, values in [0, n_aggs).
 *   c_rowptr    int32[n_aggs + 1], device.
 *   c_colind    int32[c_colind_cap], device; c_colind_cap >= nnz always suffices.
 *   c_nnz       host.
 * Synchronises `stream`.
 */
int mis2_coarsen(mis2_ctx* ctx, const mis2_csr* g, const int32_t* labels, int64_t n_aggs,
                 int32_t* c_rowptr, int32_t* c_colind, int64_t c_colind_cap, int64_t* c_nnz,
                 void* stream);

/*
 * One full coarsening level: mis2_run, then mis2_aggregate in the
 * context's agg_mode, then mis2_coarsen.  Device outputs as above
 * (in_set and roots may be NULL).  Host outputs n_roots, n_aggs, c_nnz may
 * be NULL.  Synchronises `stream`.
 */
int mis2_coarsen_level(mis2_ctx* ctx, const mis2_csr* g, uint64_t seed, uint8_t* in_set,
                       int32_t* roots, int32_t* labels, int32_t* c_rowptr, int32_t* c_colind,
                       int64_t c_colind_cap, int64_t* n_roots, int64_t* n_aggs, int64_t* c_nnz,
                       void* stream);

/*
 * Same as mis2_coarsen_level, with every buffer in HOST memory (pinned
 * memory gives asynchronous copies): the graph is copied into context
 * scratch, processed, and the outputs copied back.  rowptr is int32 or
 * int64 as g->rowptr_is_64 says; g->rowptr and g->colind are host pointers
 * here.  The context needs max_nnz >= nnz for the copy of colind.
 */
int mis2_coarsen_level_host(mis2_ctx* ctx, const mis2_csr* g_host, uint64_t seed,
                            uint8_t* in_set, int32_t* roots, int32_t* labels, int32_t* c_rowptr,
                            int32_t* c_colind, int64_t c_colind_cap, int64_t* n_roots,
                            int64_t* n_aggs, int64_t* c_nnz, void* stream);

/* Distance-k maximal independent set (Section II: no two members within k
 * hops, every vertex within k hops of one), the generalisation of
 * Algorithm 1: each round spreads, over k hops of closed neighbourhoods,
 * "some IN vertex within reach" and "the smallest undecided tuple within
 * reach" (tuples of Section V); an undecided vertex becomes OUT if an IN
 * vertex is within k hops, IN if its tuple is the smallest within k hops.
 * k = 2 gives exactly mis2_run's set and round count, k = 1 a maximal
 * independent set.  1 <= k <= 16.  Outputs as mis2_run; host-driven rounds
 * over every vertex; synchronises once per round. */
int mis2_run_k(mis2_ctx* ctx, const mis2_csr* g, int32_t k, uint64_t seed, uint8_t* in_set, int32_t* roots,
               int64_t* n_roots, int32_t* n_rounds, void* stream);

/* Colour sets for cluster multicolor Gauss-Seidel (Algorithm 4's setup:
 * colorsets = color(A_c), meant for the coarse graph of mis2_coarsen): a
 * distance-1 colouring, the first-fit greedy colouring in ascending order of
 * the round-0 tuples h(0, v) (Eq. 1; seed as in mis2_run), computed by
 * Jones-Plassmann rounds that reproduce that order exactly.  Outputs
 * (DEVICE): colors [n]; color_ptr (capacity n + 1) and color_list [n]: the
 * vertices of colour k, ascending, are color_list[color_ptr[k] ..
 * color_ptr[k+1]); *n_colors and *n_rounds (host).  Self-loops are ignored.
 * Synchronises. */
int mis2_color(mis2_ctx* ctx, const mis2_csr* g, uint64_t seed, int32_t* colors, int32_t* color_ptr,
               int32_t* color_list, int32_t* n_colors, int32_t* n_rounds, void* stream);

/* Cluster lists of cluster multicolor Gauss-Seidel (Algorithm 4 relaxes the
 * fine rows of one cluster in order): the fine vertices of each aggregate,
 * ascending.  labels (DEVICE, [n]) as written by mis2_aggregate, values in
 * [0, n_aggs); outputs (DEVICE): c_ptr [n_aggs + 1] and members [n], the
 * vertices of aggregate a being members[c_ptr[a] .. c_ptr[a+1]).
 * MIS2_ERR_INVALID_ARG for n > max_n, n_aggs > n, or n > 0 with n_aggs == 0;
 * MIS2_ERR_BAD_GRAPH when a label lies outside [0, n_aggs) (the outputs are
 * then unspecified, but nothing is written outside them).  Synchronises. */
int mis2_cluster_lists(mis2_ctx* ctx, const int32_t* labels, int64_t n, int64_t n_aggs, int32_t* c_ptr,
                       int32_t* members, void* stream);

/* Coarse edge weights (Section III-B: the coarse system of a multilevel
 * method): c_weights[k] = the number of fine entries (u, v) of g with
 * labels[u] = A and labels[v] = c_colind[k], for k in coarse row A; i.e. the
 * off-diagonal of P^T A P for the 0/1 adjacency A and the 0/1 tentative
 * prolongator P.  labels / n_aggs as mis2_aggregate returns them,
 * c_rowptr / c_colind / c_nnz as mis2_coarsen returns them (each row
 * ascending); c_weights (DEVICE, c_nnz int32) is written.  Synchronises;
 * MIS2_ERR_BAD_GRAPH if an entry has no coarse counterpart. */
int mis2_coarse_weights(mis2_ctx* ctx, const mis2_csr* g, const int32_t* labels, int64_t n_aggs,
                        const int32_t* c_rowptr, const int32_t* c_colind, int64_t c_nnz, int32_t* c_weights,
                        void* stream);

/* Tentative prolongator of an aggregation (Section III-B: residuals are
 * restricted to the coarse system, its solution interpolated back): P is
 * n x n_aggs in CSR with one entry per row, P[v, labels[v]] = 1, or
 * 1/sqrt(|aggregate of v|) with normalize != 0 (orthonormal columns: the
 * smoothed-aggregation tentative prolongator for a constant near-null
 * space; IEEE double sqrt and division).  Outputs (DEVICE): p_rowptr
 * [n+1] = 0..n, p_colind [n] = labels, p_values [n].  Asynchronous. */
int mis2_tentative_prolongator(mis2_ctx* ctx, const int32_t* labels, int64_t n, int64_t n_aggs,
                               int32_t normalize, int32_t* p_rowptr, int32_t* p_colind, double* p_values,
                               void* stream);

/* ------------------------------------------------------------------------
 * Batched hierarchies: many graphs, every level of their recursive
 * coarsening (Section I: multilevel methods coarsen recursively until the
 * graph is below a threshold), processed together.  Each level of all live
 * graphs runs as one block-diagonal union: one persistent launch per MIS-2
 * for every graph's rounds, aggregation and coarse graph on the union.  Every
 * graph's results are bit-identical to coarsening it alone with
 * mis2_coarsen_level, level after level.
 * ------------------------------------------------------------------------ */
typedef struct mis2_batch mis2_batch;

/* Scratch for up to max_graphs graphs totalling max_total_n vertices and
 * max_total_nnz entries at level 0 (allocated now; per-level outputs are
 * allocated on first use and reused by later runs of the same sizes). */
int mis2_batch_create(mis2_batch** b, int32_t max_graphs, int64_t max_total_n, int64_t max_total_nnz,
                      const mis2_config* cfg);
int mis2_batch_destroy(mis2_batch* b);

/*
 * Coarsen each graph (graphs: HOST array of n_graphs mis2_csr whose rowptr /
 * colind are device pointers; rows must list each neighbour once) level
 * after level while it has >= min_n vertices and keeps shrinking, for at most
 * max_levels levels.  *n_levels (host) receives the number of levels built.
 * Synchronises `stream`.
 */
int mis2_batch_coarsen(mis2_batch* b, int32_t n_graphs, const mis2_csr* graphs, uint64_t seed, int64_t min_n,
                       int32_t max_levels, int32_t* n_levels, void* stream);

/* Sizes at `level`: n[g] vertices, n_aggs[g] aggregates and c_nnz[g] coarse
 * entries of graph g (host arrays of n_graphs, each may be NULL; 0 for
 * graphs not coarsened at that level). */
int mis2_batch_level_sizes(const mis2_batch* b, int32_t level, int64_t* n, int64_t* n_aggs, int64_t* c_nnz);

/* Aggregate labels of graph `graph` at `level` (device int32[n], values in
 * [0, n_aggs)); MIS2_ERR_INVALID_ARG if the graph was not coarsened there. */
int mis2_batch_labels(const mis2_batch* b, int32_t level, int32_t graph, int32_t* labels, void* stream);

/* Coarse graph of graph `graph` built at `level` (device int32[n_aggs+1]
 * and int32[c_colind_cap >= c_nnz]); the same graph is the input of
 * level + 1.  Synchronises `stream`. */
int mis2_batch_coarse(const mis2_batch* b, int32_t level, int32_t graph, int32_t* c_rowptr, int32_t* c_colind,
                      int64_t c_colind_cap, void* stream);

/* Statistics of the last mis2_batch_coarsen (launch count, kernel times). */
int mis2_batch_stats(const mis2_batch* b, mis2_stats* out);

/* ------------------------------------------------------------------------
 * Serving: a request loop with continuous batching.  Each request is one
 * coarsening level (mis2_coarsen_level_host) of a graph in HOST memory.
 * Requests queue in arrival order and are admitted while an execution slot
 * is free and the device-memory budget holds their buffers; each slot owns a
 * resident context (status arrays, worklists, staging buffers), a stream and
 * a host thread, so requests admitted while others run overlap on the GPU.
 * Results are independent of the mix (every slot has its own scratch).
 * ------------------------------------------------------------------------ */
typedef struct mis2_server mis2_server;

typedef struct {
  int32_t slots;          /* concurrent launches (default 4) */
  int32_t batch_max;      /* requests merged into one launch by a slot: 0 or 1 = one request per slot
                             (its own context); >= 2 = the queued requests that fit (same seed, at most
                             batch_max of them, slot_max_n / slot_max_nnz in total) run together as one
                             block-diagonal union through the batched engine (mis2_batch_coarsen, one
                             level) */
  int64_t mem_budget;     /* bytes of request buffers admitted at once (default 8 GiB) */
  int64_t slot_max_n;     /* largest request (batch_max >= 2: largest union) per slot (vertices, entries) */
  int64_t slot_max_nnz;
  mis2_config cfg;        /* per-slot configuration.  Default loop: MIS2_LOOP_HOST, whose
                             per-round kernels of different requests interleave on the GPU;
                             with MIS2_LOOP_DEVICE the slots share a lock so that one
                             device-loop kernel runs at a time (the other steps of their
                             requests overlap freely), which suits a single slot best */
} mis2_server_config;

typedef struct {
  int64_t ticket;
  int64_t n, nnz;
  int64_t n_roots, n_aggs, c_nnz;
  /* Fingerprint of the outputs, computed on the device: with
   * mix(z) = the SplitMix64 finaliser (z ^= z>>30; z *= 0xBF58476D1CE4E5B9;
   * z ^= z>>27; z *= 0x94D049BB133111EB; z ^= z>>31), arrays A_0..A_3 =
   * roots[n_roots], labels[n], c_rowptr[n_aggs+1], c_colind[c_nnz] and
   * counts (n_roots, n_aggs, c_nnz), it is the sum mod 2^64 of
   * mix(mix((k << 40) + i) ^ (uint32)A_k[i]) over every k, i, plus
   * mix(((uint64)(5 + j) << 40) ^ count_j) for j = 0..2. */
  uint64_t checksum;
  double t_arrive, t_start, t_done;  /* seconds since the server was created */
  int32_t status;           /* mis2_status of the request */
  int32_t slot;
} mis2_result;

/* Host buffers that receive a request's results (any may be NULL: not
 * returned).  in_set[n], roots[n], labels[n], c_rowptr[n+1], c_colind
 * [c_colind_cap]: the outputs of mis2_coarsen_level_host for the request's
 * graph; a coarse graph larger than c_colind_cap fails the request with
 * MIS2_ERR_INVALID_ARG.  They must stay valid until the request completes. */
typedef struct {
  uint8_t* in_set;
  int32_t* roots;
  int32_t* labels;
  int32_t* c_rowptr;
  int32_t* c_colind;
  int64_t c_colind_cap;
} mis2_request_out;

void mis2_server_config_default(mis2_server_config* cfg);
/* Creates cfg->slots contexts (cudaMalloc now) and their worker threads. */
int mis2_server_create(mis2_server** s, const mis2_server_config* cfg);
/* Stops the workers after the queue drains, frees everything. */
int mis2_server_destroy(mis2_server* s);
/* Queue one request; g_host points to HOST memory that must stay valid until
 * the request completes.  *ticket (host) identifies it.  Does not block. */
int mis2_server_submit(mis2_server* s, const mis2_csr* g_host, uint64_t seed, int64_t* ticket);
/* mis2_server_submit, with the request's results also written to *out's
 * host buffers (out may be NULL: results as fingerprint only). */
int mis2_server_submit_out(mis2_server* s, const mis2_csr* g_host, uint64_t seed, const mis2_request_out* out,
                           int64_t* ticket);
/* Block until request `ticket` completes; *out (host) receives its result. */
int mis2_server_wait(mis2_server* s, int64_t ticket, mis2_result* out);
/* Withdraw request `ticket` if it is still queued: *cancelled (host) = 1 and
 * its result (mis2_server_wait) has status MIS2_ERR_CANCELLED; a request
 * already running or finished is left alone (*cancelled = 0).  Does not
 * block on the GPU.  MIS2_ERR_INVALID_ARG for an unknown ticket. */
int mis2_server_cancel(mis2_server* s, int64_t ticket, int32_t* cancelled);
/* Replay an arrival trace: request i (graph pool_host[pool_index[i]])
 * arrives arrival_s[i] seconds after the call starts; results[i] (host)
 * receive the outcomes, *max_in_flight the peak number of concurrent
 * requests.  Blocks until all complete. */
int mis2_server_replay(mis2_server* s, int32_t n_pool, const mis2_csr* pool_host, int64_t n_req,
                       const double* arrival_s, const int32_t* pool_index, uint64_t seed, mis2_result* results,
                       int64_t* max_in_flight);

/*
 * MIS-2 without allocating: the same result as mis2_run (and the same
 * arguments, minus the context), for callers that cannot call cudaMalloc --
 * processes whose device memory is fully budgeted up front, or whose
 * allocator owns the whole device, and latency-critical code that must not
 * block on cudaMalloc / cudaFree.  The paper has no counterpart.
 *
 * Scratch comes from a fixed array of about 14.7 MB compiled into the
 * library.  The array is committed when the library's device code is loaded
 * into a context: with CUDA's default lazy module loading that is usually
 * the first call of this function on a device, so a process that budgets
 * device memory up front must make one (small) warm-up call before its
 * allocator reserves the rest of the device; the array then stays committed
 * until the context ends.  Graphs with more than MIS2_NOALLOC_MAX_N vertices
 * are rejected with MIS2_ERR_INVALID_ARG (message in mis2_last_error());
 * nnz is not limited, since colind stays in caller memory.  The call itself
 * makes no cudaMalloc, cudaFree or other allocating call: host-side counters
 * use stack memory.
 *
 * The array's device address is looked up (cudaGetSymbolAddress) the first
 * time a context calls this function -- once per device, or again after
 * cudaDeviceReset or when the caller made another context current; make that
 * first call before any CUDA stream capture.  All calls share the array and
 * it keeps the last call's contents (the counters are cleared at the start of
 * each call), so calls that overlap on the GPU (concurrent streams or
 * threads) race and give wrong results; serialise them.  The round loop runs
 * on the device (MIS2_LOOP_DEVICE) with the default configuration.
 * Synchronises `stream`.
 */
#define MIS2_NOALLOC_MAX_N 262144
int mis2_run_noalloc(const mis2_csr* g, uint64_t seed, uint8_t* in_set, int32_t* roots,
                     int64_t* n_roots, int32_t* n_rounds, void* stream);

/* Human-readable name of a status code (static storage). */
const char* mis2_status_string(int status);

/* Text of the last CUDA error seen by the library in this thread ("" if none). */
const char* mis2_last_error(void);

/* Library version, e.g. "0.1.0". */
const char* mis2_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MIS2_GB300_H */
