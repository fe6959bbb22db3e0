"""Independent checks that pin the oracle to the paper's definitions.

Nothing here calls the oracle's decision logic.  It restates what MIS-2,
aggregation and the coarse graph must satisfy:

- distance-k independence and maximality (Section I), via BFS balls and via
  the matrix-power criterion of Lemma 1 (Section IV);
- the "ball" form of one round of Algorithm 1 (Section III-A, the radius-2
  minimum argument): an undecided v becomes OUT iff a vertex that was IN
  before the round lies within distance 2, else IN iff its tuple is the
  strict minimum over the undecided vertices within distance 2.  It compares
  (priority, id) tuples lexicographically and never builds the column array;
- the aggregation rules of Algorithms 2 and 3 (Section III-B) as properties
  of the output labels;
- the coarse graph as the set of aggregate pairs joined by a fine edge.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def adjacency_sets(g, member=None):
    rp = np.asarray(g.rowptr, dtype=np.int64)
    ci = np.asarray(g.colind, dtype=np.int64)
    adj = []
    for v in range(g.n):
        s = set(int(w) for w in ci[rp[v]:rp[v + 1]] if w != v)
        if member is not None:
            s = {w for w in s if member[w]} if member[v] else set()
        adj.append(s)
    return adj


def ball(adj, v, radius):
    seen = {v: 0}
    q = deque([v])
    while q:
        u = q.popleft()
        if seen[u] == radius:
            continue
        for w in adj[u]:
            if w not in seen:
                seen[w] = seen[u] + 1
                q.append(w)
    return set(seen)


def check_distance2_mis(adj, roots, member=None):
    """Distance-2 independence and maximality (Section I definitions)."""
    n = len(adj)
    verts = [v for v in range(n) if member is None or member[v]]
    rs = set(int(r) for r in roots)
    for r in rs:
        b = ball(adj, r, 2)
        assert not (b & rs) - {r}, f"roots within distance 2 of {r}"
    for v in verts:
        if v in rs:
            continue
        assert ball(adj, v, 2) & rs, f"vertex {v} has no root within distance 2"


def check_lemma1(n, edges, roots):
    """Independence/maximality through G^2 with self-loops (Lemma 1, Lemma 2):
    roots form an independent, maximal set of (I + A)^2."""
    B = np.eye(n, dtype=np.int64)
    for u, v in edges:
        B[u, v] = B[v, u] = 1
    B2 = (B @ B) > 0
    r = np.zeros(n, dtype=bool)
    r[list(roots)] = True
    sub = B2[np.ix_(r, r)]
    assert (sub == np.eye(int(r.sum()), dtype=bool)).all()
    assert B2[:, r].any(axis=1).all() if n else True


def ball_mis2(adj, tuple_of, member=None, max_rounds=10_000):
    """Rounds of Algorithm 1 in ball form.  tuple_of(round, v) returns any
    totally ordered key (e.g. (priority, id)).  Returns (IN set, rounds,
    per-round list of (new_in, new_out))."""
    n = len(adj)
    verts = [v for v in range(n) if member is None or member[v]]
    balls = {v: ball(adj, v, 2) for v in verts}
    undecided = set(verts)
    IN = set()
    hist = []
    r = 0
    while undecided:
        assert r < max_rounds
        key = {v: tuple_of(r, v) for v in undecided}
        new_in, new_out = [], []
        for v in undecided:
            if balls[v] & IN:
                new_out.append(v)
            elif all(key[v] < key[u] for u in balls[v] if u != v and u in undecided):
                new_in.append(v)
        IN.update(new_in)
        undecided.difference_update(new_in)
        undecided.difference_update(new_out)
        hist.append((sorted(new_in), sorted(new_out)))
        r += 1
    return IN, r, hist


def check_aggregation(g, in_set, labels, n_aggs, n_phase1, mode, m2_roots=None):
    """Algorithm 3 (mode 0) / Algorithm 2 (mode 1) as properties of labels.

    m2_roots: the MIS-2 of the subgraph induced by the vertices left
    unaggregated after phase 1 (mode 0 only), computed independently.
    """
    n = g.n
    adj = adjacency_sets(g)
    labels = np.asarray(labels)
    assert labels.shape == (n,)
    assert (labels >= 0).all() and (labels < n_aggs).all(), "every vertex in exactly one aggregate"
    roots1 = np.flatnonzero(np.asarray(in_set)).tolist()
    assert n_phase1 == len(roots1)
    tent = np.full(n, -1, dtype=np.int64)
    root_of = {}
    # phase 1: root i (ascending) and its neighbours form aggregate i
    for i, r in enumerate(roots1):
        for u in [r] + sorted(adj[r]):
            assert tent[u] == -1, "phase-1 aggregates overlap: roots not distance-2 independent"
            tent[u] = i
            assert labels[u] == i, "phase-1 aggregate is not root + neighbours"
        root_of[i] = r
    k = len(roots1)
    if mode == 0:
        unagg = tent == -1
        for v in sorted(m2_roots):
            nb = [u for u in adj[v] if unagg[u]]
            if len(nb) < 2:
                continue
            for u in [v] + nb:
                assert tent[u] == -1
                tent[u] = k
                assert labels[u] == k, "phase-2 aggregate is not root + unaggregated neighbours"
            root_of[k] = v
            k += 1
    assert k == n_aggs, "aggregate count = phase-1 roots + qualifying phase-2 roots"
    size = np.bincount(tent[tent >= 0], minlength=n_aggs)
    # phase 3: each leftover joins the adjacent aggregate of max coupling,
    # ties to min tentative size, then min id
    for v in np.flatnonzero(tent == -1).tolist():
        coup = {}
        for u in adj[v]:
            if tent[u] >= 0:
                coup[int(tent[u])] = coup.get(int(tent[u]), 0) + 1
        assert coup, f"leftover {v} has no aggregated neighbour"
        a = int(labels[v])
        assert a in coup, "leftover joined a non-adjacent aggregate"
        for b, c in coup.items():
            assert (coup[a], -size[a], -a) >= (c, -size[b], -b), "phase-3 choice is not the max"
    # one root per aggregate; aggregates connected
    assert len(root_of) == n_aggs
    members = [[] for _ in range(n_aggs)]
    for v in range(n):
        members[labels[v]].append(v)
    for a in range(n_aggs):
        ms = set(members[a])
        r = root_of[a]
        assert r in ms
        seen = {r}
        q = deque([r])
        while q:
            u = q.popleft()
            for w in adj[u]:
                if w in ms and w not in seen:
                    seen.add(w)
                    q.append(w)
        assert seen == ms, f"aggregate {a} is not connected"


def quotient_pairs(g, labels):
    """Coarse graph as the set of (label u, label v) over fine edges, u, v in
    different aggregates."""
    rp = np.asarray(g.rowptr, dtype=np.int64)
    ci = np.asarray(g.colind, dtype=np.int64)
    lab = np.asarray(labels, dtype=np.int64)
    rows = np.repeat(np.arange(g.n), rp[1:] - rp[:-1])
    a, b = lab[rows], lab[ci]
    keep = a != b
    return set(zip(a[keep].tolist(), b[keep].tolist()))


def csr_pairs(rowptr, colind):
    rp = np.asarray(rowptr, dtype=np.int64)
    out = set()
    for a in range(len(rp) - 1):
        for b in np.asarray(colind[rp[a]:rp[a + 1]]).tolist():
            out.add((a, int(b)))
    return out
