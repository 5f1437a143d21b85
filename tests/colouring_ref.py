"""Independent reference for the oracle's greedy colouring: Jones-Plassmann
rounds (every uncoloured node whose priority beats all its uncoloured
neighbours takes the smallest colour its coloured neighbours leave free).
With distinct priorities this colours exactly like the greedy scan in
descending priority.  Test infrastructure only."""
import numpy as np


def jones_plassmann(n, u, v, prio):
    nbrs = [[] for _ in range(n)]
    for a, b in zip(np.asarray(u).tolist(), np.asarray(v).tolist()):
        nbrs[a].append(b)
        nbrs[b].append(a)
    key = [(int(prio[i]), i) for i in range(n)]
    colour = [-1] * n
    left = set(range(n))
    while left:
        ready = [i for i in left if all(colour[j] >= 0 or key[j] < key[i] for j in nbrs[i])]
        assert ready
        for i in ready:
            taken = {colour[j] for j in nbrs[i] if colour[j] >= 0}
            c = 0
            while c in taken:
                c += 1
            colour[i] = c
        left.difference_update(ready)
    return np.array(colour, np.int32)
