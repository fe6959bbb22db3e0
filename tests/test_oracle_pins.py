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
        hs = [0, 1, 1 << 40, (1 << 32) - 1, 1 << 63, top]
        keys = [((h & 0xFFFFFFFF) % (1 << (32 - b)), v, oracle.pack(h, v, b)) for h in hs for v in (0, n - 1)]
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


def _table_graph(ref):
    return gg.grid3d_7pt(*ref["dims"]) if ref["problem"] == "laplace" else gg.elasticity3d(*ref["dims"])


def test_table3_laplace_small():
    """Section VI-B, Table III (soft band: the hash constants are a reading)."""
    tab = json.load(open(os.path.join(GOLDEN, "tables.json")))
    for ref in tab["table3"]:
        if ref["n"] <= 125000:
            _, roots, rounds, _ = oracle.mis2(_table_graph(ref))
            _band(tab, len(roots), rounds, ref)


@pytest.mark.slow
def test_table3_full():
    """Every row of Table III: |MIS-2| within 5 % and the iteration count
    within 3 of the printed ones (xorshift* priorities)."""
    tab = json.load(open(os.path.join(GOLDEN, "tables.json")))
    for ref in tab["table3"]:
        _, roots, rounds, _ = oracle.mis2(_table_graph(ref))
        _band(tab, len(roots), rounds, ref)


def test_table1_priority_schemes_laplace3d_100():
    """Section V-A, Table I on Laplace3D_100: the iteration count of each
    priority scheme within 3 of the printed one (Fixed 14, Xor 20, Xor* 10),
    so plain xorshift needs markedly more rounds than fixed priorities and
    xorshift* fewer."""
    tab = json.load(open(os.path.join(GOLDEN, "tables.json")))
    ref = tab["table1"][0]
    assert ref["matrix"] == "Laplace3D_100"
    g = _table_graph(ref)
    got = {k: oracle.mis2(g, hash_variant=v)[2] for k, v in
           (("fixed", oracle.HASH_FIXED), ("xor", oracle.HASH_XORSHIFT), ("xor_star", oracle.HASH_XORSHIFT_STAR))}
    for k, r in got.items():
        assert abs(r - ref[k]) <= tab["bands"]["iters_abs"], (k, r, ref[k])
    assert got["xor"] > got["fixed"] > got["xor_star"]


@pytest.mark.slow
def test_table1_priority_schemes_elasticity3d_60():
    """Table I on Elasticity3D_60: Fixed and Xor* within 3 of the printed 13
    and 10, and the same order of the three schemes as printed (Xor > Fixed >
    Xor*).  Plain xorshift takes 16 rounds here against the printed 23: the
    order holds, the count does not (the only Table I entry outside the band
    among the two regenerable matrices)."""
    tab = json.load(open(os.path.join(GOLDEN, "tables.json")))
    ref = tab["table1"][1]
    assert ref["matrix"] == "Elasticity3D_60"
    g = _table_graph(ref)
    got = {k: oracle.mis2(g, hash_variant=v)[2] for k, v in
           (("fixed", oracle.HASH_FIXED), ("xor", oracle.HASH_XORSHIFT), ("xor_star", oracle.HASH_XORSHIFT_STAR))}
    for k in ("fixed", "xor_star"):
        assert abs(got[k] - ref[k]) <= tab["bands"]["iters_abs"], (k, got[k], ref[k])
    assert got["xor"] > got["fixed"] > got["xor_star"]


# ------------------------------------------------------------ the hash f
_ORDER = (1 << 64) - 1
_ORDER_PRIMES = (3, 5, 17, 257, 641, 65537, 6700417)  # 2^64 - 1 = their product


def _gf2_columns(f):
    """The 64 x 64 matrix over GF(2) of a linear map f on 64-bit words, as
    the images of the unit vectors (column j = f(1 << j))."""
    return [f(1 << j) for j in range(64)]


def _gf2_apply(cols, x):
    y = 0
    j = 0
    while x:
        if x & 1:
            y ^= cols[j]
        x >>= 1
        j += 1
    return y


def _gf2_mul(a, b):
    """Columns of A.B (apply B, then A)."""
    return [_gf2_apply(a, c) for c in b]


def _gf2_pow(cols, e):
    result = [1 << j for j in range(64)]
    base = cols
    while e:
        if e & 1:
            result = _gf2_mul(base, result)
        base = _gf2_mul(base, base)
        e >>= 1
    return result


def test_plain_xorshift_is_a_full_period_xorshift():
    """f of the Xor Hash (Section V-A) read through the seed argument
    (h(0, 0) with seed s is f(s), since f(0) = 0): it must be linear over
    GF(2) and, as a generator x -> f(x), have the full period 2^64 - 1 over
    the non-zero words, Marsaglia's condition for a usable xorshift triple
    (J. Stat. Softw. 8(14), 2003): T^(2^64-1) = I and T^((2^64-1)/p) != I
    for every prime p dividing 2^64 - 1.  A wrong shift amount or direction
    makes the period short (or the map singular)."""
    f = lambda s: oracle.hash64(0, 0, s, oracle.HASH_XORSHIFT)
    assert f(0) == 0
    rng = np.random.default_rng(5)
    for _ in range(50):
        a, b = (int(x) for x in rng.integers(0, 1 << 63, 2, dtype=np.uint64))
        assert f(a ^ b) == f(a) ^ f(b)
    cols = _gf2_columns(f)
    identity = [1 << j for j in range(64)]
    assert _gf2_pow(cols, _ORDER) == identity
    for p in _ORDER_PRIMES:
        assert _gf2_pow(cols, _ORDER // p) != identity, p
    # h(iter, v) = f(f(iter) ^ f(v)): linear, so h(i, v) ^ h(j, v) does not
    # depend on v -- the correlation between rounds that Section V-A blames
    # for the plain hash's extra iterations
    d = {oracle.hash64(3, v, 0, oracle.HASH_XORSHIFT) ^ oracle.hash64(4, v, 0, oracle.HASH_XORSHIFT)
         for v in range(100)}
    assert len(d) == 1


def test_xorshift_star_is_the_xorshift_stage_then_one_multiply():
    """Section V-A: xorshift* is xorshift followed by a multiplicative
    (linear congruential) step.  f*(s) / f(s) mod 2^64 must be one odd
    constant over every s whose f(s) is odd (f = the plain variant), and f*
    must not be linear over GF(2)."""
    f = lambda s: oracle.hash64(0, 0, s, oracle.HASH_XORSHIFT)
    fs = lambda s: oracle.hash64(0, 0, s, oracle.HASH_XORSHIFT_STAR)
    mult = set()
    for s in range(1, 400):
        x = f(s)
        if x & 1:
            mult.add(fs(s) * pow(x, -1, 1 << 64) % (1 << 64))
    assert len(mult) == 1 and next(iter(mult)) & 1
    assert any(fs(a ^ b) != fs(a) ^ fs(b) for a, b in ((1, 2), (3, 12), (5, 1 << 40)))
    # FIXED is xorshift* with the round held at 0
    for v in (0, 1, 77, 1 << 20):
        assert oracle.hash64(9, v, 0, oracle.HASH_FIXED) == oracle.hash64(0, v, 0, oracle.HASH_XORSHIFT_STAR)


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


def test_unpacked_equals_packed():
    # The unpacked tuple holds the same 32-b priority bits as Eq. 1's packed
    # word, compared as (status, priority, id): the order of undecided
    # vertices is the packed integer order, so Algorithm 1 takes the same
    # steps and the two results coincide on every graph, seed and hash.
    for seed in range(3):
        for variant in (oracle.HASH_XORSHIFT_STAR, oracle.HASH_XORSHIFT, oracle.HASH_FIXED):
            for g in _unpacked_graphs():
                pk = oracle.mis2(g, seed, hash_variant=variant)
                up = oracle.mis2_unpacked(g, seed, hash_variant=variant)
                assert np.array_equal(pk[0], up[0]) and pk[2] == up[2]


def test_unpacked_tuples_break_priority_ties_by_id():
    # Two adjacent vertices 0 and w among 2^20 - 2 otherwise isolated ones
    # (b = 20, so 12 priority bits), w chosen so that both draw the same 12
    # bits in round 0: the tie goes to the smaller id in both forms, so
    # vertex 0 joins and w does not.
    n = (1 << 20) - 2
    assert oracle.id_bits(n) == 20
    p0 = oracle.priority_tuple(0, 0, n, 0) >> 20
    w = next((v for v in range(1, n) if oracle.priority_tuple(0, v, n, 0) >> 20 == p0), None)
    assert w is not None
    g = gg.graph_from_edges(n, [(0, w)])
    pk = oracle.mis2(g, 0)
    up = oracle.mis2_unpacked(g, 0)
    for res in (pk, up):
        assert res[0][0] == 1 and res[0][w] == 0
        assert res[0].sum() == n - 1  # every other vertex is isolated and joins
