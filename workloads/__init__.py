"""Seeded synthetic graphs shaped like the paper's workloads (Sec. 5, Table 1).

This module builds inputs only: canonical undirected edge lists
``(u < v, sorted by (u, v), unique, w > 0)`` plus the node count.  It holds none
of the reduction method's arithmetic, so both the CUDA library's tests and the
oracle consume the same bytes from it.  All randomness comes from numpy's
PCG64 with an explicit seed.

Named workloads (sizes of the paper's graphs; the datasets themselves are not
used):
  grid2d_64      64 x 64 grid, unit weights (4,096 nodes, 8,064 edges)
  knn_200k       kNN (k=10) graph of 200,000 GMM points in 10-D, Gaussian weights
  chunglu_434k   Chung-Lu power-law graph, 434,000 nodes, ~16M unit edges,
                 mean degree ~73.5, max expected degree 1,200, exponent 2.5
                 (shaped like coPapersCiteseer, Table 1)
  mesh3d_128     128^3 7-point mesh, log-normal weights (2,097,152 nodes)
  knn_1m         kNN (k=15) graph of 1,000,000 GMM points in 16-D
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Graph:
    n: int
    u: np.ndarray  # int32[m], u < v
    v: np.ndarray  # int32[m]
    w: np.ndarray  # float64[m], > 0
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.u.shape[0])


def sorted_unique(k):
    """Sorted distinct values of an int64 array (np.sort + run heads; much
    faster than np.unique on large inputs)."""
    s = np.sort(np.asarray(k, np.int64), kind="stable")
    if s.shape[0] == 0:
        return s
    head = np.empty(s.shape[0], bool)
    head[0] = True
    np.not_equal(s[1:], s[:-1], out=head[1:])
    return s[head]


def canonicalize(n, a, b, w=None, combine="first"):
    """Turn an arbitrary undirected pair list into the canonical form: drop
    self-loops, orient u < v, sort by (u, v), merge duplicates.  ``combine``
    decides the weight of a merged pair: 'first' keeps the first occurrence's
    weight, 'sum' adds them."""
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    if w is None:
        w = np.ones(a.shape[0], np.float64)
    w = np.asarray(w, np.float64)
    keep = a != b
    a, b, w = a[keep], b[keep], w[keep]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = lo * np.int64(n) + hi
    order = np.argsort(key, kind="stable")
    key = key[order]
    w = w[order]
    first = np.ones(key.shape[0], bool)
    first[1:] = key[1:] != key[:-1]
    if combine == "sum":
        idx = np.cumsum(first) - 1
        ws = np.zeros(int(first.sum()), np.float64)
        np.add.at(ws, idx, w)
        w = ws
    else:
        w = w[first]
    key = key[first]
    u = (key // n).astype(np.int32)
    v = (key % n).astype(np.int32)
    return u, v, w


# ---------------------------------------------------------------------------
# Regular meshes
# ---------------------------------------------------------------------------
def grid2d(a: int, b: int, weights=None) -> Graph:
    """a x b grid, node id i + a*j, edges to the right and up."""
    ids = np.arange(a * b, dtype=np.int64).reshape(b, a)  # ids[j, i]
    h0, h1 = ids[:, :-1].ravel(), ids[:, 1:].ravel()
    v0, v1 = ids[:-1, :].ravel(), ids[1:, :].ravel()
    u, v, _ = canonicalize(a * b, np.concatenate([h0, v0]), np.concatenate([h1, v1]))
    w = np.ones(u.shape[0]) if weights is None else weights(u.shape[0])
    return Graph(a * b, u, v, w, "grid2d_%dx%d" % (a, b))


def mesh3d(a: int, b: int, c: int, sigma: float = 1.0, seed: int = 12349) -> Graph:
    """a x b x c 7-point mesh, id i + a*j + a*b*k; weights exp(N(0, sigma^2))
    drawn in canonical edge order (circuit-grid-like, log-normal)."""
    n = a * b * c
    ids = np.arange(n, dtype=np.int64).reshape(c, b, a)
    pairs = [
        (ids[:, :, :-1].ravel(), ids[:, :, 1:].ravel()),
        (ids[:, :-1, :].ravel(), ids[:, 1:, :].ravel()),
        (ids[:-1, :, :].ravel(), ids[1:, :, :].ravel()),
    ]
    u, v, _ = canonicalize(n, np.concatenate([p[0] for p in pairs]), np.concatenate([p[1] for p in pairs]))
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.exp(rng.normal(0.0, sigma, size=u.shape[0]))
    return Graph(n, u, v, w, "mesh3d_%dx%dx%d" % (a, b, c))


def path(n: int, w=None) -> Graph:
    u = np.arange(n - 1, dtype=np.int32)
    v = u + 1
    return Graph(n, u, v.astype(np.int32), np.ones(n - 1) if w is None else np.asarray(w, np.float64), "path%d" % n)


def cycle(n: int, weight: float = 1.0) -> Graph:
    u, v, w = canonicalize(n, np.arange(n), (np.arange(n) + 1) % n, np.full(n, weight))
    return Graph(n, u, v, w, "cycle%d" % n)


def circulant(n: int, offsets_weights) -> Graph:
    """Weighted circulant graph: i ~ i+s (mod n) with weight w_s."""
    a, b, w = [], [], []
    for s, ws in offsets_weights:
        a.append(np.arange(n))
        b.append((np.arange(n) + s) % n)
        w.append(np.full(n, float(ws)))
    u, v, ww = canonicalize(n, np.concatenate(a), np.concatenate(b), np.concatenate(w))
    return Graph(n, u, v, ww, "circulant%d" % n)


def torus2d(a: int, b: int) -> Graph:
    ids = np.arange(a * b, dtype=np.int64).reshape(b, a)
    right = np.roll(ids, -1, axis=1)
    up = np.roll(ids, -1, axis=0)
    u, v, w = canonicalize(a * b, np.concatenate([ids.ravel(), ids.ravel()]),
                           np.concatenate([right.ravel(), up.ravel()]))
    return Graph(a * b, u, v, w, "torus%dx%d" % (a, b))


def complete(n: int, weight: float = 1.0) -> Graph:
    iu = np.triu_indices(n, 1)
    return Graph(n, iu[0].astype(np.int32), iu[1].astype(np.int32), np.full(len(iu[0]), weight), "K%d" % n)


def star(n: int) -> Graph:
    u = np.zeros(n - 1, np.int32)
    v = np.arange(1, n, dtype=np.int32)
    return Graph(n, u, v, np.ones(n - 1), "star%d" % n)


def random_sparse(n: int, m: int, seed: int, weighted=True, connected=True) -> Graph:
    """Erdos-Renyi-like multigraph sample, canonicalised; a random spanning
    path is added first when ``connected``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.integers(0, n, size=m)
    b = rng.integers(0, n, size=m)
    if connected and n > 1:
        perm = rng.permutation(n)
        a = np.concatenate([perm[:-1], a])
        b = np.concatenate([perm[1:], b])
    w = rng.uniform(0.1, 2.0, size=a.shape[0]) if weighted else None
    u, v, ww = canonicalize(n, a, b, w)
    return Graph(n, u, v, ww, "rand%d_%d" % (n, m))


# ---------------------------------------------------------------------------
# Chung-Lu power-law graph
# ---------------------------------------------------------------------------
def chung_lu_weights(n: int, mean_deg: float, max_deg: float, exponent: float = 2.5):
    """Expected degrees w_i = c (1 + i/i0)^(-1/(exponent-1)), c = max_deg, with
    i0 solved so the mean is mean_deg."""
    g = 1.0 / (exponent - 1.0)
    i = np.arange(n, dtype=np.float64)

    def mean_for(i0):
        return float(np.mean(max_deg * (1.0 + i / i0) ** (-g)))

    lo, hi = 1e-3, float(n) * 1e3
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        if mean_for(mid) < mean_deg:
            lo = mid
        else:
            hi = mid
    i0 = np.sqrt(lo * hi)
    return max_deg * (1.0 + i / i0) ** (-g)


def chung_lu(n: int = 434_000, m_target: int = 16_000_000, mean_deg: float = 73.5,
             max_deg: float = 1200.0, exponent: float = 2.5, seed: int = 12348) -> Graph:
    """Sample endpoints proportional to the expected degrees, drop self-loops
    and duplicates, and top up until m_target unique unit-weight edges."""
    wts = chung_lu_weights(n, mean_deg, max_deg, exponent)
    cdf = np.cumsum(wts)
    cdf /= cdf[-1]
    rng = np.random.Generator(np.random.PCG64(seed))
    keys = np.empty(0, np.int64)
    need = m_target
    margin = 1.12
    while need > 0:
        batch = int(need * margin) + 1024
        a = np.searchsorted(cdf, rng.random(batch), side="right").astype(np.int64)
        b = np.searchsorted(cdf, rng.random(batch), side="right").astype(np.int64)
        np.minimum(a, n - 1, out=a)
        np.minimum(b, n - 1, out=b)
        keep = a != b
        a, b = a[keep], b[keep]
        k = np.minimum(a, b) * np.int64(n) + np.maximum(a, b)
        keys = sorted_unique(np.concatenate([keys, k]))
        need = m_target - keys.shape[0]
        margin = 2.0
    if keys.shape[0] > m_target:
        # drop a uniformly random surplus (keeps the degree profile unbiased)
        drop = rng.choice(keys.shape[0], keys.shape[0] - m_target, replace=False)
        mask = np.ones(keys.shape[0], bool)
        mask[drop] = False
        keys = keys[mask]
    # keys stay sorted and unique: the list is canonical
    u = (keys // n).astype(np.int32)
    v = (keys % n).astype(np.int32)
    return Graph(n, u, v, np.ones(u.shape[0]), "chunglu_%d" % n)


# ---------------------------------------------------------------------------
# kNN graphs of Gaussian-mixture points
# ---------------------------------------------------------------------------
def gmm_points(npts: int, dim: int, ncomp: int, seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(-10.0, 10.0, size=(ncomp, dim))
    comp = rng.integers(0, ncomp, size=npts)
    return centres[comp] + rng.normal(0.0, 1.0, size=(npts, dim))


def knn_indices(P: np.ndarray, k: int, device=None, chunk=4096):
    """Exact k nearest neighbours (excluding self), distance ties broken by
    index.  Candidates come from torch (on ``device`` if given, FP32), then
    the final choice and distances are recomputed in FP64 on the host."""
    import torch

    n = P.shape[0]
    extra = 4
    kk = min(k + 1 + extra, n)
    dev = torch.device(device) if device is not None else torch.device("cpu")
    Pt = torch.from_numpy(P.astype(np.float32)).to(dev)
    sq = (Pt * Pt).sum(1)
    cand = np.empty((n, kk), np.int64)
    for s in range(0, n, chunk):
        e = min(s + chunk, n)
        d2 = sq[s:e, None] - 2.0 * (Pt[s:e] @ Pt.T) + sq[None, :]
        cand[s:e] = torch.topk(d2, kk, dim=1, largest=False).indices.cpu().numpy()
    # exact FP64 refinement over the candidates (chunked)
    idx = np.empty((n, k), np.int64)
    dd = np.empty((n, k), np.float64)
    for s in range(0, n, 65536):
        e = min(s + 65536, n)
        c = cand[s:e]
        diff = P[c] - P[s:e, None, :]
        dist2 = np.einsum("ijk,ijk->ij", diff, diff)
        dist2[c == np.arange(s, e)[:, None]] = np.inf
        order = np.lexsort((c, dist2), axis=1)[:, :k]
        idx[s:e] = np.take_along_axis(c, order, 1)
        dd[s:e] = np.sqrt(np.take_along_axis(dist2, order, 1))
    return idx, dd


def knn_gmm(npts: int = 200_000, dim: int = 10, ncomp: int = 10, k: int = 10,
            seed: int = 12347, device=None) -> Graph:
    """kNN graph (union-symmetrised) of GMM points; w = exp(-d^2/sigma^2) with
    sigma the median kNN distance."""
    P = gmm_points(npts, dim, ncomp, seed)
    idx, dd = knn_indices(P, k, device=device)
    sigma = float(np.median(dd))
    a = np.repeat(np.arange(npts), k)
    b = idx.ravel()
    w = np.exp(-(dd.ravel() ** 2) / sigma ** 2)
    u, v, ww = canonicalize(npts, a, b, w, combine="first")
    ww = np.maximum(ww, np.finfo(np.float64).tiny)
    return Graph(npts, u, v, ww, "knn_%d_%dd_k%d" % (npts, dim, k))


# ---------------------------------------------------------------------------
# Named configurations (reduction parameters ride along)
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    K: int
    sweeps: int
    omega: float
    precision: str          # "f64", "f32", "bf16"
    final_target: int
    make: object            # callable(device) -> Graph


WORKLOADS = {
    "grid2d_64": Workload("grid2d_64", 8, 5, 0.7, "f64", 1024, lambda device=None: grid2d(64, 64)),
    "knn_200k": Workload("knn_200k", 16, 5, 0.7, "f32", 6250,
                         lambda device=None: knn_gmm(200_000, 10, 10, 10, 12347, device)),
    "chunglu_434k": Workload("chunglu_434k", 16, 5, 0.7, "f32", 13000, lambda device=None: chung_lu()),
    "mesh3d_128": Workload("mesh3d_128", 24, 8, 0.7, "f32", 32768, lambda device=None: mesh3d(128, 128, 128)),
    "knn_1m": Workload("knn_1m", 16, 5, 0.7, "f32", 31250,
                       lambda device=None: knn_gmm(1_000_000, 16, 20, 15, 12350, device)),
}
