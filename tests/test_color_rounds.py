"""The round structure the colouring kernels rely on, replayed on CPU: Jones-
Plassmann rounds with the round-0 tuples as fixed priorities, where an
uncoloured vertex resumes its scan at the chunk of its last blocker and
collects the colours of the neighbours it finds coloured into a mask kept
across rounds, and takes the first free colour of that mask once nothing
smaller blocks it.  This must give the oracle's first-fit colouring in tuple
order, on every graph and for any scan chunk: a neighbour coloured before v
has the smaller tuple (a larger one waits for v), so the mask sees every
colour v has to avoid."""
import numpy as np
import pytest

import oracle
from paper_2204_02934_gb300 import graphgen as gg

UNCOLORED = 1 << 30


def _rounds(g, seed, chunk):
    n = g.n
    rp = g.rowptr.astype(np.int64)
    rows = [g.colind[rp[v]:rp[v + 1]].tolist() for v in range(n)]
    prio = [oracle.priority_tuple(0, v, n, seed) for v in range(n)]
    col = [-1] * n
    when = [UNCOLORED] * n
    resume = [0] * n
    mask = [set() for _ in range(n)]
    r = 0
    while any(w == UNCOLORED for w in when):
        assert r <= n
        coloured_now = []
        for v in range(n):
            if when[v] != UNCOLORED:
                continue
            row = rows[v]
            blocked_at = None
            for off in range(resume[v], len(row), chunk):
                hit = False
                for w in row[off:off + chunk]:
                    if w == v:
                        continue
                    if when[w] < r:
                        mask[v].add(col[w])  # coloured before this round: final
                    elif prio[w] < prio[v]:
                        hit = True  # smaller and uncoloured at the start of the round
                if hit:
                    blocked_at = off
                    break
            if blocked_at is not None:
                resume[v] = blocked_at
                continue
            c = 0
            while c in mask[v]:
                c += 1
            coloured_now.append((v, c))
        for v, c in coloured_now:  # a vertex coloured this round counts as uncoloured until it ends
            col[v] = c
            when[v] = r
        r += 1
    return np.array(col, dtype=np.int32), r


def _graphs():
    yield gg.grid2d_5pt(8, 7)
    yield gg.grid3d_27pt(4, 3, 3)
    yield gg.rmat(7, 6, seed=9)
    yield gg.random_graph(40, 0.5, 4)  # dense: many colours
    yield gg.graph_from_edges(25, [(0, i) for i in range(1, 25)])  # star


@pytest.mark.parametrize("chunk", [1, 3, 16])
@pytest.mark.parametrize("seed", [0, 5])
def test_resumed_masked_rounds_give_first_fit_in_tuple_order(seed, chunk):
    for g in _graphs():
        colors, rounds = _rounds(g, seed, chunk)
        ref, nc = oracle.color_greedy(g, seed)
        assert np.array_equal(colors, ref)
        assert 1 <= rounds <= g.n
