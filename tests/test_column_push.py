"""The column step of Algorithm 1 in push form gives the same column tuples
as the pull form it restates.

Pull (Algorithm 1): for v in worklist 2, M_v = min over N[v] of T_w, with IN
turned into OUT.  Push: reset M_v = OUT for v in worklist 2; every undecided
u lowers M_w to T_u for w in N[u] and in worklist 2; every vertex that
became IN in the previous round lowers them to IN, read as OUT.  A vertex
next to an older IN vertex already left worklist 2 (its M went OUT the round
after), and decided OUT vertices cannot lower a minimum, so both forms agree
round by round.  A push-form column kernel for the narrow middle rounds
would rely on this; here both run in plain Python over the oracle's tuples
and the final sets are checked against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2204_02934_gb300 import graphgen as gg

IN, OUT = oracle.IN, oracle.OUT


def _rows(g):
    rp = g.rowptr.astype(np.int64)
    return [g.colind[rp[v]:rp[v + 1]].tolist() for v in range(g.n)]


def _run(g, seed, push):
    n = g.n
    rows = _rows(g)
    T = [0] * n
    M = [OUT] * n
    undecided = set(range(n))
    wl2 = set(range(n))
    newly_in = set()
    history = []
    for it in range(n + 1):
        if not undecided:
            break
        for v in undecided:
            T[v] = oracle.priority_tuple(it, v, n, seed)
        if push:
            for v in wl2:
                M[v] = OUT
            for u in undecided | newly_in:
                val = T[u]  # IN (0) for a newly IN vertex
                for w in [u] + rows[u]:
                    if w in wl2 and val < M[w]:
                        M[w] = val
            for v in wl2:
                if M[v] == IN:
                    M[v] = OUT
        else:
            for v in wl2:
                m = T[v]
                for w in rows[v]:
                    m = min(m, T[w])
                M[v] = OUT if m == IN else m
        history.append(list(M))
        newly_in = set()
        decided = {}
        for v in undecided:
            ms = [M[v]] + [M[w] for w in rows[v]]
            if any(x == OUT for x in ms):
                decided[v] = OUT
            elif all(x == T[v] for x in ms):
                decided[v] = IN
        for v, t in decided.items():
            T[v] = t
            undecided.discard(v)
            if t == IN:
                newly_in.add(v)
        wl2 = {v for v in wl2 if M[v] != OUT}
    in_set = np.array([1 if T[v] == IN else 0 for v in range(n)], dtype=np.uint8)
    return in_set, len(history), history


def _graphs():
    yield gg.grid2d_5pt(9, 8)
    yield gg.grid3d_27pt(4, 4, 3)
    yield gg.rmat(7, 6, seed=5)
    for s in range(4):
        yield gg.random_graph(45, 0.06 + 0.03 * s, 10 + s)
    yield gg.graph_from_edges(30, [(0, i) for i in range(1, 20)] + [(20, 21), (21, 22)])


@pytest.mark.parametrize("seed", [0, 2])
def test_push_column_equals_pull_column(seed):
    for g in _graphs():
        a_in, a_rounds, a_hist = _run(g, seed, push=False)
        b_in, b_rounds, b_hist = _run(g, seed, push=True)
        assert a_hist == b_hist, "column tuples differ in some round"
        assert np.array_equal(a_in, b_in) and a_rounds == b_rounds
        ref = oracle.mis2(g, seed)
        assert np.array_equal(a_in, ref[0]) and a_rounds == ref[2]
