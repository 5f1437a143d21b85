"""Second, independent aggregation implementation used only to pin the oracle.

The oracle aggregates by sequential greedy matching in (d, edge id) order.  This
module computes the same aggregates a different way: rounds of the parallel
"handshake" (every free cluster points at its best free neighbour, mutual pairs
merge; repeat until no free cluster has a free neighbour), which yields the
unique locally-dominant matching (Preis 1999; Manne & Bisseling 2007), followed
by truncation to the smallest allowed keys.  Plain Python, small graphs only.
"""


def handshake_aggregate(n, u, v, d, target_nc, passes):
    rep = list(range(n))
    n_cur = n
    for _ in range(passes):
        if n_cur <= target_nc:
            break
        # cluster pair -> smallest fine key
        key = {}
        for e in range(len(u)):
            A, B = rep[u[e]], rep[v[e]]
            if A == B:
                continue
            pair = (min(A, B), max(A, B))
            k = (float(d[e]), e)
            if pair not in key or k < key[pair]:
                key[pair] = k
        nbrs = {}
        for (A, B), k in key.items():
            nbrs.setdefault(A, []).append((k, B))
            nbrs.setdefault(B, []).append((k, A))
        free = set(nbrs.keys())
        matched = []
        while True:
            best = {}
            for A in free:
                cands = [(k, B) for (k, B) in nbrs[A] if B in free]
                if cands:
                    best[A] = min(cands)
            if not best:
                break
            progress = False
            for A, (k, B) in best.items():
                if A < B and B in best and best[B][1] == A:
                    matched.append((k, A, B))
                    progress = True
            for _, A, B in matched:
                free.discard(A)
                free.discard(B)
            assert progress, "handshake made no progress"
        allowed = n_cur - max(target_nc, 0)
        matched.sort()
        matched = matched[:allowed]
        newrep = {}
        for _, A, B in matched:
            newrep[A] = min(A, B)
            newrep[B] = min(A, B)
        rep = [newrep.get(r, r) for r in rep]
        n_cur -= len(matched)
        if not matched:
            break
    reps = sorted(set(rep))
    label = {r: i for i, r in enumerate(reps)}
    return [label[r] for r in rep], len(reps)
