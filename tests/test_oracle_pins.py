"""Pins for the CPU oracle: every check compares it with something other than
itself (the paper's worked example, definitions, an independent ball-form
restatement of Algorithm 1, closed forms, the paper's tables)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2204_02934_gb300 import graphgen as gg
from _pins import (adjacency_sets, ball_mis2, check_aggregation, check_distance2_mis,
                   check_lemma1, csr_pairs, quotient_pairs)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
OUT = 0xFFFFFFFF


def _unpack(x, b):
    if x == 0:
        return "IN"
    if x == OUT:
        return "OUT"
    return [x >> b, x & ((1 << b) - 1)]


# ------------------------------------------------------------------ Fig. 1
def test_fig1_worked_example():
    """Section III-A, Fig. 1: priorities, column tuples, decisions, result."""
    fx = json.load(open(os.path.join(GOLDEN, "fig1.json")))
    n = fx["n"]
    g = gg.graph_from_edges(n, [(a - 1, b - 1) for a, b in fx["edges"]])
    tab = np.zeros((len(fx["rounds"]), n), dtype=np.uint32)
    for r, rd in enumerate(fx["rounds"]):
        for vid, p in rd["priorities"].items():
            tab[r, int(vid) - 1] = p
    in_set, roots, rounds, _, snaps = oracle.mis2(g, prio_table=tab, snap_cap=4)
    b = oracle.id_bits(n)
    assert b == 3
    assert rounds == fx["n_rounds"]
    assert (roots + 1).tolist() == fx["result"]
    for r, rd in enumerate(fx["rounds"]):
        T0, M, T1 = snaps[r]
        for vid, p in rd["priorities"].items():
            assert _unpack(int(T0[int(vid) - 1]), b) == [p, int(vid)]
        for vid, m in rd["column"].items():
            assert _unpack(int(M[int(vid) - 1]), b) == m
        for vid, d in rd["decide"].items():
            got = _unpack(int(T1[int(vid) - 1]), b)
            assert (got if isinstance(got, str) else "U") == d


# ------------------------------------------------------------------ Eq. 1
@pytest.mark.parametrize("n", list(range(0, 70)) + [254, 255, 256, 1022, 1023, 1024, 65533, 65534,
                                                     65535, 65536, 2**20 - 2, 2**20, 2**31 - 3])
def test_packing_never_collides(n):
    """Section V-C, Eq. 1: 2^b >= |V| + 2, so a packed undecided tuple is
    never IN (0) nor OUT (UINT_MAX), and it orders like (priority, id)."""
    b = oracle.id_bits(n)
    assert 2 ** b >= n + 2 and (b == 0 or 2 ** (b - 1) < n + 2)
    top = (1 << 64) - 1
    ids = sorted(set([0, max(n - 1, 0), n // 2, max(n - 2, 0)]))
    for v in ids:
        if v >= n:
            continue
        lo = oracle.pack(0, v, b)
        hi = oracle.pack(top, v, b)
        assert lo not in (0, OUT) and hi not in (0, OUT)
        assert lo & ((1 << b) - 1) == v + 1 and hi & ((1 << b) - 1) == v + 1
    # lexicographic order of (priority, id) = integer order of packed tuples
    if n >= 2:
        hs = [0, 1 << 40, 1 << 63, top]
        keys = [(h >> (32 + b), v, oracle.pack(h, v, b)) for h in hs for v in (0, n - 1)]
        keys.sort()
        assert [k[2] for k in keys] == sorted(k[2] for k in keys)


def test_xorshift_star_zero_fixed_point():
    """xorshift maps 0 to 0, so h(0, 0) = f(0) = 0: vertex 0 has the smallest
    possible tuple (priority 0, id 1) in round 0 with seed 0."""
    assert oracle.priority_tuple(0, 0, 100, 0) == 1


# ------------------------------------------------------------------ ball form
def _random_table(n, rounds, seed):
    b = oracle.id_bits(n)
    hi = 1 << (32 - b)
    u = gg.splitmix64(np.arange(rounds * n, dtype=np.uint64), seed)
    return (u % np.uint64(hi)).astype(np.uint32).reshape(rounds, n)


def _edges_of(n, mask):
    pairs = list(itertools.combinations(range(n), 2))
    return [p for k, p in enumerate(pairs) if (mask >> k) & 1]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_exhaustive_small_graphs_ball_form(n):
    """Every labelled graph on n <= 5 vertices, 3 random priority tables each:
    same per-round decisions as the ball form, and a valid MIS-2."""
    m = n * (n - 1) // 2
    for mask in range(1 << m):
        edges = _edges_of(n, mask)
        g = gg.graph_from_edges(n, edges)
        adj = adjacency_sets(g)
        for s in range(3):
            tab = _random_table(n, n + 2, 1000 * mask + s)
            in_set, roots, rounds, _, snaps = oracle.mis2(g, prio_table=tab, snap_cap=n + 2)
            IN, r_ball, hist = ball_mis2(adj, lambda r, v: (int(tab[r, v]), v))
            assert set(roots.tolist()) == IN
            assert rounds == r_ball
            check_lemma1(n, edges, roots)


def test_exhaustive_n6_definitions():
    """All 2^15 labelled graphs on 6 vertices (hash priorities, seed 0):
    the oracle's output is distance-2 independent and maximal (Lemma 1)."""
    n = 6
    for mask in range(1 << 15):
        edges = _edges_of(n, mask)
        g = gg.graph_from_edges(n, edges)
        _, roots, rounds, _ = oracle.mis2(g)
        check_lemma1(n, edges, roots)
        assert 1 <= rounds <= n


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n,p", [(40, 0.08), (120, 0.03), (200, 0.015)])
def test_random_graphs_ball_form_hash(n, p, seed):
    """Random G(n,p): per-round agreement with the ball form under the hashed
    priorities, and the Section I definitions."""
    g = gg.random_graph(n, p, seed)
    adj = adjacency_sets(g)
    _, roots, rounds, _ = oracle.mis2(g, seed=seed)
    IN, r_ball, _ = ball_mis2(adj, lambda r, v: oracle.priority_tuple(r, v, n, seed))
    assert set(roots.tolist()) == IN and rounds == r_ball
    check_distance2_mis(adj, roots)
    assert rounds <= n  # progress: the minimum undecided tuple is decided


@pytest.mark.parametrize("seed", range(4))
def test_masked_mis2_is_mis2_of_induced_subgraph(seed):
    """Phase 2 reading: MIS-2 of G minus a vertex set = MIS-2 of the induced
    subgraph, same ids; removed vertices neither relay nor block."""
    g = gg.random_graph(150, 0.03, 50 + seed)
    u = gg.uniform01(np.arange(150, dtype=np.uint64), 77 + seed)
    member = (u < 0.6).astype(np.uint8)
    adj_sub = adjacency_sets(g, member)
    in_set, roots, rounds, _ = oracle.mis2(g, seed=seed, member=member)
    assert set(roots.tolist()) <= set(np.flatnonzero(member).tolist())
    IN, r_ball, _ = ball_mis2(adj_sub, lambda r, v: oracle.priority_tuple(r, v, 150, seed),
                              member=member)
    assert set(roots.tolist()) == IN and rounds == r_ball
    check_distance2_mis(adj_sub, roots, member)


# ------------------------------------------------------------------ edge cases
def test_degenerate_graphs():
    g0 = gg.graph_from_edges(0, [])
    in_set, roots, rounds, _ = oracle.mis2(g0)
    assert len(roots) == 0 and rounds == 0
    g1 = gg.graph_from_edges(1, [])
    _, roots, rounds, _ = oracle.mis2(g1)
    assert roots.tolist() == [0] and rounds == 1
    # isolated vertices are all IN in round 0
    giso = gg.graph_from_edges(5, [])
    _, roots, rounds, _ = oracle.mis2(giso)
    assert roots.tolist() == [0, 1, 2, 3, 4] and rounds == 1
    # a clique has exactly one root; a star's root set is one vertex
    k = gg.graph_from_edges(7, list(itertools.combinations(range(7), 2)))
    _, roots, _, _ = oracle.mis2(k)
    assert len(roots) == 1
    star = gg.graph_from_edges(9, [(0, i) for i in range(1, 9)])
    _, roots, _, _ = oracle.mis2(star)
    assert len(roots) == 1


def _with_extra_entries(g, self_loops=True, duplicates=True):
    rp = g.rowptr.astype(np.int64)
    rows, cols = [], []
    for v in range(g.n):
        row = list(g.colind[rp[v]:rp[v + 1]])
        cs = row + ([v] if self_loops else []) + (row[:1] if duplicates else [])
        rows.append(len(cs))
        cols.extend(cs)
    rp2 = np.concatenate([[0], np.cumsum(rows)]).astype(np.int64)
    return gg.CSRGraph(g.n, rp2, np.asarray(cols, dtype=np.int32))


def test_self_loops_and_duplicates_are_harmless():
    """Closed neighbourhoods: a stored diagonal or a duplicate entry changes
    no min / any / all of Algorithm 1.  Aggregation counts neighbours (the
    >= 2 test of phase 2, coupling in phase 3) over the edge set, so there a
    row may hold a self-loop but must list each neighbour once."""
    g = gg.random_graph(80, 0.05, 3)
    g2 = _with_extra_entries(g)
    a = oracle.mis2(g, seed=5)
    b = oracle.mis2(g2, seed=5)
    assert (a[0] == b[0]).all() and a[2] == b[2]
    g3 = _with_extra_entries(g, duplicates=False)
    for mode in (0, 1):
        la = oracle.coarsen_level(g, seed=5, mode=mode)
        lb = oracle.coarsen_level(g3, seed=5, mode=mode)
        assert (la.labels == lb.labels).all() and la.n_aggs == lb.n_aggs
        assert (la.c_rowptr == lb.c_rowptr).all() and (la.c_colind == lb.c_colind).all()


def test_path_graph_closed_form():
    """A path is decided from the hashed minima; every root set must leave no
    gap longer than 2 and keep roots >= 3 apart (definition on a path)."""
    for n in (2, 3, 10, 101):
        g = gg.graph_from_edges(n, [(i, i + 1) for i in range(n - 1)])
        _, roots, _, _ = oracle.mis2(g, seed=n)
        r = roots.tolist()
        assert all(b - a >= 3 for a, b in zip(r, r[1:]))
        assert r[0] <= 2 and r[-1] >= n - 3
        assert all(b - a <= 5 for a, b in zip(r, r[1:]))


# ------------------------------------------------------------------ aggregation
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("seed", range(5))
def test_aggregation_properties(mode, seed):
    for g in (gg.random_graph(120, 0.04, 300 + seed), gg.grid2d_5pt(13, 11, np.int64),
              gg.rgg2d(300, 6.0, 900 + seed, np.int64)):
        in_set, roots, _, _ = oracle.mis2(g, seed=seed)
        labels, n_aggs, n1, _, _ = oracle.aggregate(g, in_set, seed=seed, mode=mode)
        m2 = None
        if mode == 0:
            # independent phase-2 MIS-2: ball form on the leftover subgraph
            adj = adjacency_sets(g)
            agg1 = np.zeros(g.n, dtype=bool)
            for r in roots.tolist():
                agg1[r] = True
                agg1[list(adj[r])] = True
            member = (~agg1).astype(np.uint8)
            IN, _, _ = ball_mis2(adjacency_sets(g, member),
                                 lambda r, v: oracle.priority_tuple(r, v, g.n, seed), member=member)
            m2 = IN
        check_aggregation(g, in_set, labels, n_aggs, n1, mode, m2)


def test_aggregation_exhaustive_small():
    """All graphs on 5 vertices: both modes give a valid aggregation."""
    n = 5
    for mask in range(1 << 10):
        g = gg.graph_from_edges(n, _edges_of(n, mask))
        in_set, roots, _, _ = oracle.mis2(g)
        for mode in (0, 1):
            labels, n_aggs, n1, _, _ = oracle.aggregate(g, in_set, mode=mode)
            m2 = None
            if mode == 0:
                adj = adjacency_sets(g)
                agg1 = np.zeros(n, dtype=bool)
                for r in roots.tolist():
                    agg1[r] = True
                    agg1[list(adj[r])] = True
                member = (~agg1).astype(np.uint8)
                m2, _, _ = ball_mis2(adjacency_sets(g, member),
                                     lambda r, v: oracle.priority_tuple(r, v, n, 0), member=member)
            check_aggregation(g, in_set, labels, n_aggs, n1, mode, m2)


def test_aggregation_rejects_non_mis2():
    g = gg.graph_from_edges(3, [(0, 1), (1, 2)])
    with pytest.raises(oracle.OracleError):
        oracle.aggregate(g, np.array([1, 0, 1], dtype=np.uint8))


# ------------------------------------------------------------------ coarse graph
@pytest.mark.parametrize("seed", range(4))
def test_coarse_graph_is_quotient(seed):
    for g in (gg.random_graph(150, 0.04, 10 + seed), gg.grid3d_7pt(6, 5, 4, np.int64),
              gg.rmat(9, 8, seed=seed)):
        lv = oracle.coarsen_level(g, seed=seed)
        pairs = csr_pairs(lv.c_rowptr, lv.c_colind)
        assert pairs == quotient_pairs(g, lv.labels)
        assert pairs == {(b, a) for a, b in pairs}  # symmetric
        rp = lv.c_rowptr
        for a in range(lv.n_aggs):
            row = lv.c_colind[rp[a]:rp[a + 1]]
            assert (np.diff(row) > 0).all() and a not in row.tolist()


def test_hierarchy_shrinks_and_stops():
    g = gg.grid2d_5pt(80, 70, np.int64)
    levels = oracle.hierarchy(g, min_n=100)
    sizes = [g.n] + [lv.n_aggs for lv in levels]
    assert all(b < a for a, b in zip(sizes, sizes[1:]))
    assert sizes[-1] < 100 and sizes[-2] >= 100


def test_determinism():
    g = gg.rmat(12, 8, seed=1)
    a = oracle.coarsen_level(g, seed=3)
    for _ in range(3):
        b = oracle.coarsen_level(g, seed=3)
        assert (a.labels == b.labels).all() and (a.c_colind == b.c_colind).all()


# ------------------------------------------------------------------ paper tables
def _band(tab, got_size, got_iters, ref):
    assert abs(got_size - ref["mis2"]) <= tab["bands"]["size_rel"] * ref["mis2"]
    assert abs(got_iters - ref["iters"]) <= tab["bands"]["iters_abs"]


def test_table3_laplace_small():
    """Section VI-B, Table III (soft band: the hash bits are a reading)."""
    tab = json.load(open(os.path.join(GOLDEN, "tables.json")))
    ref = tab["table3"][0]
    g = gg.grid3d_7pt(*ref["dims"])
    _, roots, rounds, _ = oracle.mis2(g)
    _band(tab, len(roots), rounds, ref)


@pytest.mark.slow
def test_table3_and_table1_full():
    """Table III rows, and the Table I ordering on Laplace3D_100 (xorshift*
    needs fewer rounds than fixed priorities)."""
    tab = json.load(open(os.path.join(GOLDEN, "tables.json")))
    for ref in tab["table3"]:
        if ref["problem"] == "laplace":
            g = gg.grid3d_7pt(*ref["dims"])
        else:
            g = gg.elasticity3d(*ref["dims"])
        _, roots, rounds, _ = oracle.mis2(g)
        _band(tab, len(roots), rounds, ref)
    g = gg.grid3d_7pt(100, 100, 100)
    r_star = oracle.mis2(g, hash_variant=oracle.HASH_XORSHIFT_STAR)[2]
    r_fixed = oracle.mis2(g, hash_variant=oracle.HASH_FIXED)[2]
    t1 = tab["table1_laplace3d_100"]
    assert abs(r_fixed - t1["fixed"]) <= tab["bands"]["iters_abs"]
    assert r_star < r_fixed


# ------------------------------------------------------------ Galerkin pieces
def _pt_a_p(g, labels, n_aggs):
    """P^T A P with scipy.sparse: A the 0/1 adjacency, P[v, labels[v]] = 1."""
    sp = pytest.importorskip("scipy.sparse")
    n = g.n
    rows = np.repeat(np.arange(n), np.diff(np.asarray(g.rowptr, dtype=np.int64)))
    A = sp.csr_matrix((np.ones(len(g.colind)), (rows, np.asarray(g.colind))), shape=(n, n))
    P = sp.csr_matrix((np.ones(n), (np.arange(n), np.asarray(labels))), shape=(n, n_aggs))
    return (P.T @ A @ P).tocsr()


@pytest.mark.parametrize("name,g", [("grid2d", gg.grid2d_5pt(23, 17)), ("grid3d27", gg.grid3d_27pt(9, 8, 7)),
                                    ("rmat", gg.rmat(10, 8, seed=9)), ("gnp", gg.random_graph(300, 0.02, 5))])
def test_coarse_weights_are_the_offdiagonal_of_galerkin_product(name, g):
    lv = oracle.coarsen_level(g, seed=1)
    w = oracle.coarse_weights(g, lv.labels, lv.n_aggs, lv.c_rowptr, lv.c_colind)
    G = _pt_a_p(g, lv.labels, lv.n_aggs)
    G.setdiag(0)
    G.eliminate_zeros()
    G.sort_indices()
    assert np.array_equal(G.indptr.astype(np.int64), lv.c_rowptr)  # the coarse graph is the product's pattern
    assert np.array_equal(G.indices, lv.c_colind)
    assert np.array_equal(G.data.astype(np.int64), w)
    crossing = int(np.sum(lv.labels[np.repeat(np.arange(g.n), np.diff(g.rowptr))] != lv.labels[g.colind]))
    assert int(w.sum()) == crossing and (w >= 1).all()
    # symmetric graph -> symmetric weights
    assert (abs(G - G.T)).nnz == 0


def test_prolongator_columns_and_rows():
    g = gg.grid3d_7pt(11, 10, 9)
    lv = oracle.coarsen_level(g, seed=4)
    sizes = np.bincount(lv.labels, minlength=lv.n_aggs)
    pc, pv = oracle.prolongator(lv.labels, lv.n_aggs, normalize=False)
    assert np.array_equal(pc, lv.labels) and (pv == 1.0).all()  # piecewise constant: row sums 1
    pc, pv = oracle.prolongator(lv.labels, lv.n_aggs, normalize=True)
    sp = pytest.importorskip("scipy.sparse")
    P = sp.csr_matrix((pv, (np.arange(g.n), pc)), shape=(g.n, lv.n_aggs))
    PtP = (P.T @ P).toarray()
    assert np.allclose(PtP, np.eye(lv.n_aggs), rtol=0, atol=4e-16 * sizes.max())  # orthonormal columns
    assert np.array_equal(pv, 1.0 / np.sqrt(sizes[lv.labels].astype(np.float64)))


# ------------------------------------------------------------ MIS-k
def _dist_le(g, src, k):
    """Vertices within k hops of src (BFS)."""
    seen = {src}
    frontier = [src]
    for _ in range(k):
        nxt = []
        for u in frontier:
            for w in g.colind[g.rowptr[u]:g.rowptr[u + 1]]:
                if int(w) not in seen:
                    seen.add(int(w))
                    nxt.append(int(w))
        frontier = nxt
    return seen


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("seed", [0, 3])
def test_misk_is_a_maximal_distance_k_independent_set(k, seed):
    for g in (gg.random_graph(80, 0.05, seed + 1), gg.grid2d_5pt(9, 8), gg.rmat(7, 4, seed=seed + 2)):
        in_set, roots, rounds = oracle.misk(g, k, seed)
        roots = [int(r) for r in roots]
        covered = set()
        for r in roots:
            ball = _dist_le(g, r, k)
            assert not (ball - {r}) & set(roots), "two roots within distance k"
            covered |= ball
        assert covered == set(range(g.n)), "not maximal: a vertex is farther than k from every root"
        assert rounds <= g.n


def test_misk_with_k_2_is_algorithm_1():
    for seed in range(4):
        for g in (gg.random_graph(150, 0.03, seed), gg.grid3d_27pt(6, 5, 4), gg.rmat(9, 8, seed=seed)):
            a = oracle.misk(g, 2, seed)
            b = oracle.mis2(g, seed)
            assert np.array_equal(a[0], b[0]) and a[2] == b[2]


# ------------------------------------------------------------ coloring
@pytest.mark.parametrize("seed", [0, 5])
def test_greedy_coloring_is_proper_first_fit_in_priority_order(seed):
    for g in (gg.random_graph(120, 0.05, seed + 1), gg.grid3d_27pt(5, 5, 4), gg.rmat(8, 8, seed=seed)):
        colors, nc = oracle.color_greedy(g, seed)
        prio = np.array([oracle.priority_tuple(0, v, g.n, seed) for v in range(g.n)], dtype=np.int64)
        maxdeg = int(np.max(np.diff(g.rowptr))) if g.n else 0
        assert nc == int(colors.max()) + 1 and nc <= maxdeg + 1
        for v in range(g.n):
            nb = [int(w) for w in g.colind[g.rowptr[v]:g.rowptr[v + 1]] if int(w) != v]
            assert all(colors[w] != colors[v] for w in nb), "improper"
            earlier = {int(colors[w]) for w in nb if prio[w] < prio[v]}
            assert colors[v] == min(set(range(len(earlier) + 1)) - earlier), "not first fit in priority order"


def test_color_sets_group_ascending():
    colors = np.array([2, 0, 2, 1, 0, 2], dtype=np.int32)
    ptr, lst = oracle.color_sets(colors, 3)
    assert list(ptr) == [0, 2, 3, 6] and list(lst) == [1, 4, 3, 0, 2, 5]


@pytest.mark.parametrize("n,n_keys", [(0, 0), (1, 1), (50, 7), (400, 400), (300, 1000)])
def test_cluster_lists_are_the_brute_force_grouping(n, n_keys):
    keys = gg.splitmix64(np.arange(n, dtype=np.uint64), 17) % np.uint64(max(n_keys, 1))
    keys = keys.astype(np.int32)
    ptr, lst = oracle.cluster_lists(keys, n_keys)
    assert len(ptr) == n_keys + 1 and ptr[0] == 0 and ptr[-1] == n
    for k in range(n_keys):
        assert list(lst[ptr[k]:ptr[k + 1]]) == [v for v in range(n) if keys[v] == k]


# ------------------------------------------------------------ unpacked tuples
def _unpacked_graphs():
    yield gg.grid2d_5pt(9, 7)
    yield gg.grid3d_27pt(4, 4, 3)
    for seed in range(6):
        yield gg.random_graph(40, 0.08 + 0.02 * seed, seed)
    yield gg.rmat(7, 6, seed=3)


@pytest.mark.parametrize("seed", [0, 3])
def test_unpacked_mis2_is_a_maximal_distance2_independent_set(seed):
    for g in _unpacked_graphs():
        in_set, roots, rounds = oracle.mis2_unpacked(g, seed)
        assert rounds >= 1
        check_distance2_mis(adjacency_sets(g), roots)
        again = oracle.mis2_unpacked(g, seed)
        assert np.array_equal(again[0], in_set) and again[2] == rounds  # deterministic


def test_unpacked_equals_packed_when_truncated_priorities_are_distinct():
    # Eq. 1 keeps the top 32-b hash bits; the unpacked tuple keeps 32.  The
    # truncation is monotone, so when the truncated priorities of every round
    # are pairwise distinct both orders agree and Algorithm 1 takes the same
    # steps: the two results must coincide.
    checked = 0
    for seed in range(4):
        for g in _unpacked_graphs():
            pk = oracle.mis2(g, seed)
            up = oracle.mis2_unpacked(g, seed)
            b = oracle.id_bits(g.n)
            distinct = True
            for r in range(max(pk[2], up[2])):
                trunc = {oracle.priority_tuple(r, v, g.n, seed) >> b for v in range(g.n)}
                distinct &= len(trunc) == g.n
            if not distinct:
                continue
            checked += 1
            assert np.array_equal(pk[0], up[0]) and pk[2] == up[2]
    assert checked >= 20


def test_unpacked_tuples_break_truncated_ties_by_the_full_priority():
    # Two adjacent vertices 0 and 1 among 2^20 - 2 isolated ones (b = 20, so
    # Eq. 1 keeps 12 priority bits).  For a seed where both draw the same 12
    # top bits but vertex 0 the larger 30 top bits, the packed tuple breaks
    # the tie by id (vertex 0 joins) and the unpacked one by priority
    # (vertex 1 joins).
    n = (1 << 20) - 2
    assert oracle.id_bits(n) == 20
    for seed in range(200000):
        t12 = [oracle.priority_tuple(0, v, n, seed) >> 20 for v in (0, 1)]
        if t12[0] != t12[1]:
            continue
        t30 = [oracle.priority_tuple(0, v, 1, seed) >> 2 for v in (0, 1)]
        if t30[0] > t30[1]:
            break
    else:
        pytest.fail("no seed with a 12-bit tie")
    g = gg.graph_from_edges(n, [(0, 1)])
    pk = oracle.mis2(g, seed)
    up = oracle.mis2_unpacked(g, seed)
    assert (pk[0][0], pk[0][1]) == (1, 0)
    assert (up[0][0], up[0][1]) == (0, 1)
    assert pk[0][2:].all() and up[0][2:].all()  # isolated vertices join
