"""The GPU aggregation computes each pass with the suitor algorithm (Manne &
Halappanavar 2014): every cluster keeps the smallest key proposed to it, a
displaced suitor proposes again, and a proposal made on a stale view of the
keys fails and is retried.  This module runs that algorithm as a sequential
model under random interleavings of the proposing threads, with stale reads,
and checks that every interleaving yields the oracle's greedy matching (the
equivalence the GPU relies on, Sec. 3.2.2 reading).  No GPU code is involved.
"""
import random

import numpy as np

INF = (float("inf"), 1 << 40)


def suitor_pass(n, adj, key, ends, rng, stale_prob=0.3):
    """One pass of the suitor algorithm; adj[v] = [(w, e)], key[e] unique."""
    ws = [INF] * n
    seen = [[INF] for _ in range(n)]  # every value ws[v] has held (a stale read returns one)

    def thread(start):
        cur = start
        while cur is not None:
            best, bb = INF, None
            for b, e in adj[cur]:
                k = key[e]
                if k >= best:
                    continue
                w = rng.choice(seen[b]) if rng.random() < stale_prob else ws[b]
                if k < w:
                    best, bb = k, b
                yield
            if bb is None:
                return
            old = ws[bb]  # the atomic minimum
            if old > best:
                ws[bb] = best
                seen[bb].append(best)
                if old == INF:
                    cur = None
                else:
                    p, q = ends[old[1]]
                    cur = q if p == bb else p
            yield

    threads = [thread(v) for v in range(n)]
    live = list(range(n))
    while live:
        i = rng.randrange(len(live))
        try:
            next(threads[live[i]])
        except StopIteration:
            live.pop(i)
    pairs = []
    for b in range(n):
        if ws[b] == INF:
            continue
        p, q = ends[ws[b][1]]
        a = q if p == b else p
        assert ws[a] == ws[b], "one-sided suitor at termination"
        if b < a:
            pairs.append((b, a))
    return sorted(pairs)


def test_suitor_equals_greedy_under_random_interleavings(oracle_mod):
    rng = random.Random(5)
    for _ in range(200):
        n = rng.randint(2, 14)
        edges = sorted({(min(u, v), max(u, v)) for u, v in
                        ((rng.randrange(n), rng.randrange(n)) for _ in range(rng.randint(1, 3 * n))) if u != v})
        if not edges:
            continue
        m = len(edges)
        u = np.array([e[0] for e in edges], np.int32)
        v = np.array([e[1] for e in edges], np.int32)
        d = np.round(np.array([rng.random() for _ in range(m)]), 1)  # many ties: the edge id decides
        key = [(float(d[e]), e) for e in range(m)]
        adj = [[] for _ in range(n)]
        for e, (a, b) in enumerate(edges):
            adj[a].append((b, e))
            adj[b].append((a, e))
        pairs = suitor_pass(n, adj, key, edges, rng)
        agg, _ = oracle_mod.aggregate(n, u, v, d, 1, 1)  # one pass, target 1: no truncation
        groups = {}
        for i, a in enumerate(agg):
            groups.setdefault(int(a), []).append(i)
        assert pairs == sorted(tuple(g) for g in groups.values() if len(g) == 2)
