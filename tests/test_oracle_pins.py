"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check reaches the expected value by a route other than the oracle's own
code: closed-form spectra, FFT diagonalisation of circulant operators, published
generator outputs, dense brute force, an independent handshake matching, finite
differences.  A dropped term, a wrong sign or index, or a transposed operand in
the oracle fails at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import workloads as W
from handshake_ref import handshake_aggregate

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------------------
# Laplacian (Sec. 2.1): L = D - A, zero row sums, closed-form spectra
# ---------------------------------------------------------------------------
def test_laplacian_zero_row_sums_and_structure(oracle_mod):
    g = W.random_sparse(40, 120, seed=1)
    L = oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w)
    assert np.allclose(L.sum(1), 0.0, rtol=0, atol=1e-13)
    assert np.allclose(L, L.T, rtol=0, atol=0)
    off = L - np.diag(np.diag(L))
    assert (off <= 0).all()
    # diagonal is the weighted degree: every weight counted at both endpoints
    assert np.isclose(np.trace(L), 2.0 * g.w.sum())


def test_laplacian_quadratic_form(oracle_mod):
    g = W.random_sparse(50, 200, seed=2)
    rng = np.random.default_rng(3)
    x = rng.normal(size=g.n)
    Lx = oracle_mod.laplacian_apply(g.n, g.u, g.v, g.w, x)
    q = float(np.sum(g.w * (x[g.u] - x[g.v]) ** 2))
    assert np.isclose(x @ Lx, q, rtol=1e-13)


@pytest.mark.parametrize("n", [7, 16])
def test_spectrum_path_cycle_complete_star(oracle_mod, n):
    j = np.arange(n)
    g = W.path(n)
    ev = np.linalg.eigvalsh(oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w))
    assert np.allclose(ev, np.sort(4 * np.sin(np.pi * j / (2 * n)) ** 2), rtol=0, atol=1e-12)
    g = W.cycle(n)
    ev = np.linalg.eigvalsh(oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w))
    assert np.allclose(ev, np.sort(4 * np.sin(np.pi * j / n) ** 2), rtol=0, atol=1e-12)
    g = W.complete(n, weight=1.5)
    ev = np.linalg.eigvalsh(oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w))
    assert np.allclose(ev, [0.0] + [1.5 * n] * (n - 1), rtol=0, atol=1e-12)
    g = W.star(n)
    ev = np.linalg.eigvalsh(oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w))
    assert np.allclose(ev, [0.0] + [1.0] * (n - 2) + [float(n)], rtol=0, atol=1e-12)


def test_spectrum_grid(oracle_mod):
    a, b = 6, 5
    g = W.grid2d(a, b)
    ev = np.linalg.eigvalsh(oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w))
    i, j = np.meshgrid(np.arange(a), np.arange(b))
    ref = np.sort((4 * np.sin(np.pi * i / (2 * a)) ** 2 + 4 * np.sin(np.pi * j / (2 * b)) ** 2).ravel())
    assert np.allclose(ev, ref, rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------
# Test vectors (Sec. 3.2.1): SplitMix64 known answers, uniform on [-1, 1)
# ---------------------------------------------------------------------------
def test_splitmix64_known_answers(oracle_mod):
    with open(os.path.join(GOLDEN, "splitmix64_seed0.json")) as f:
        ref = json.load(f)
    for c, hexval in enumerate(ref["outputs"]):
        assert oracle_mod.splitmix64(0, c) == int(hexval, 16)


def test_test_vectors_distribution(oracle_mod):
    X = oracle_mod.test_vectors_raw(20000, 4, seed=0, level=0)
    assert X.min() >= -1.0 and X.max() < 1.0
    assert abs(X.mean()) < 5 * np.sqrt(1 / 3 / X.size)
    assert abs(X.var() - 1 / 3) < 0.01
    from scipy.stats import kstest
    assert kstest(X.ravel(), "uniform", args=(-1, 2)).pvalue > 1e-4
    # levels and seeds give different streams
    assert not np.array_equal(X[:10], oracle_mod.test_vectors_raw(20000, 4, 0, 1)[:10])
    assert not np.array_equal(X[:10], oracle_mod.test_vectors_raw(20000, 4, 1, 0)[:10])


def test_center_normalize(oracle_mod):
    X = oracle_mod.center_normalize(oracle_mod.test_vectors_raw(1000, 5, 7, 0))
    assert np.all(np.abs(X.sum(0)) <= 1e-13 * np.sqrt(1000))
    assert np.allclose((X * X).sum(0), 1.0, rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# Smoothing (Alg. 3): FFT-diagonalised circulant graphs, complete graph,
# dense brute force, isolated nodes, invariants
# ---------------------------------------------------------------------------
def _normalize_center(Y):
    Y = Y - Y.mean(0)
    return Y / np.linalg.norm(Y, axis=0)


@pytest.mark.parametrize("omega,S", [(0.7, 5), (0.5, 8), (0.9, 3)])
def test_smooth_cycle_fft(oracle_mod, omega, S):
    n, K = 64, 6
    g = W.cycle(n, weight=2.5)
    X0 = oracle_mod.center_normalize(oracle_mod.test_vectors_raw(n, K, 0, 0))
    theta = 2 * np.pi * np.arange(n) / n
    mu = (1 - omega) + omega * np.cos(theta)  # eigenvalues of J on the cycle
    ref = np.real(np.fft.ifft(np.fft.fft(X0, axis=0) * (mu ** S)[:, None], axis=0))
    ref = _normalize_center(ref)
    X = oracle_mod.smooth(n, g.u, g.v, g.w, K, S, omega, 0, 0)
    assert np.max(np.abs(X - ref)) < 1e-13


def test_smooth_weighted_circulant_fft(oracle_mod):
    n, K, omega, S = 40, 4, 0.7, 6
    a, b = 0.3, 2.0
    g = W.circulant(n, [(1, a), (2, b)])
    X0 = oracle_mod.center_normalize(oracle_mod.test_vectors_raw(n, K, 5, 2))
    th = 2 * np.pi * np.arange(n) / n
    mu = (1 - omega) + omega * (2 * a * np.cos(th) + 2 * b * np.cos(2 * th)) / (2 * a + 2 * b)
    ref = _normalize_center(np.real(np.fft.ifft(np.fft.fft(X0, axis=0) * (mu ** S)[:, None], axis=0)))
    X = oracle_mod.smooth(n, g.u, g.v, g.w, K, S, omega, 5, 2)
    assert np.max(np.abs(X - ref)) < 1e-13


def test_smooth_torus_fft2(oracle_mod):
    a, b, K, omega, S = 8, 6, 3, 0.7, 4
    g = W.torus2d(a, b)
    X0 = oracle_mod.center_normalize(oracle_mod.test_vectors_raw(a * b, K, 3, 0))
    ti = 2 * np.pi * np.arange(a) / a
    tj = 2 * np.pi * np.arange(b) / b
    mu = (1 - omega) + omega * (np.cos(ti)[None, :] + np.cos(tj)[:, None]) / 2  # [j, i]
    Xg = X0.reshape(b, a, K)
    ref = np.real(np.fft.ifft2(np.fft.fft2(Xg, axes=(0, 1)) * (mu ** S)[:, :, None], axes=(0, 1)))
    ref = _normalize_center(ref.reshape(a * b, K))
    X = oracle_mod.smooth(a * b, g.u, g.v, g.w, K, S, omega, 3, 0)
    assert np.max(np.abs(X - ref)) < 1e-13


@pytest.mark.parametrize("n,omega,S", [(5, 0.7, 5), (3, 0.9, 3), (3, 0.9, 4)])
def test_smooth_complete_graph(oracle_mod, n, omega, S):
    # Sec. 3.2.3: on a complete graph smoothing cannot separate nodes.  For a
    # centred x, D^-1 A x = -x/(n-1), so each sweep only rescales x.
    g = W.complete(n)
    K = 4
    X0 = oracle_mod.center_normalize(oracle_mod.test_vectors_raw(n, K, 0, 0))
    sign = np.sign(1 - omega - omega / (n - 1)) ** S
    X = oracle_mod.smooth(n, g.u, g.v, g.w, K, S, omega, 0, 0)
    assert np.max(np.abs(X - sign * X0)) < 1e-14


def test_smooth_dense_bruteforce(oracle_mod):
    g = W.random_sparse(30, 80, seed=11)
    n, K, omega, S = g.n, 5, 0.65, 7
    A = np.zeros((n, n))
    A[g.u, g.v] = g.w
    A[g.v, g.u] = g.w
    J = (1 - omega) * np.eye(n) + omega * A / A.sum(1)[:, None]
    X0 = oracle_mod.center_normalize(oracle_mod.test_vectors_raw(n, K, 9, 1))
    ref = _normalize_center(np.linalg.matrix_power(J, S) @ X0)
    X = oracle_mod.smooth(n, g.u, g.v, g.w, K, S, omega, 9, 1)
    assert np.max(np.abs(X - ref)) < 1e-13


def test_sweep_isolated_node_unchanged(oracle_mod):
    # node 5 has no edges: the reading (D^-1 A x)_i := x_i keeps its row
    u = np.array([0, 1, 2, 3], np.int32)
    v = np.array([1, 2, 3, 4], np.int32)
    w = np.ones(4)
    X = np.arange(12, dtype=np.float64).reshape(6, 2) - 5.0
    Y = oracle_mod.jacobi_sweep(6, u, v, w, X, 0.7)
    assert np.array_equal(Y[5], X[5])
    # an interior path node: (1-w) x_i + w (x_{i-1} + x_{i+1}) / 2
    assert np.allclose(Y[2], 0.3 * X[2] + 0.7 * (X[1] + X[3]) / 2, rtol=0, atol=1e-15)


def test_smooth_invariants_and_lowpass(oracle_mod):
    g = W.grid2d(20, 20)
    K = 8
    Xprev = oracle_mod.center_normalize(oracle_mod.test_vectors_raw(g.n, K, 0, 0))
    rq = []
    for S in range(1, 6):
        X = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, S, 0.7, 0, 0)
        assert np.all(np.abs(X.sum(0)) <= 1e-13 * np.sqrt(g.n))
        assert np.allclose((X * X).sum(0), 1.0, rtol=0, atol=1e-14)
        LX = oracle_mod.laplacian_apply(g.n, g.u, g.v, g.w, X)
        rq.append(float(np.mean((X * LX).sum(0))))
    # low-pass filter (Sec. 3.5): the Rayleigh quotient falls with every sweep
    assert all(b < a for a, b in zip(rq, rq[1:]))


# ---------------------------------------------------------------------------
# Affinity and algebraic distance (Eq. eqn:agg, Sec. 3.2.2)
# ---------------------------------------------------------------------------
def test_affinity_hand_examples(oracle_mod):
    X = np.array([[1.0, 0.0, 0.0],
                  [1.0, 1.0, 0.0],    # cos^2 with row 0 = 1/2
                  [2.0, 1.0, -2.0],   # orthogonal to row 3
                  [1.0, 2.0, 2.0],
                  [-3.0, -6.0, -6.0],  # parallel (opposite) to row 3
                  [0.0, 0.0, 0.0]])   # zero row
    u = np.array([0, 2, 3, 0], np.int32)
    v = np.array([1, 3, 4, 5], np.int32)
    d, a = oracle_mod.affinity(6, u, v, X, want_a=True)
    assert np.allclose(a, [0.5, 0.0, 1.0, 0.0], rtol=0, atol=1e-15)
    assert np.allclose(d, [0.5, 1.0, 0.0, 1.0], rtol=0, atol=1e-15)
    assert d[2] == 0.0


def test_affinity_identities(oracle_mod):
    rng = np.random.default_rng(4)
    n, K = 200, 8
    X = rng.normal(size=(n, K))
    g = W.random_sparse(n, 800, seed=5)
    d, a = oracle_mod.affinity(n, g.u, g.v, X, want_a=True)
    assert (a >= 0).all() and (a <= 1 + 1e-15).all()
    assert (d >= 0).all() and (d <= 1 + 1e-15).all()
    lo = a < 0.5
    assert np.max(np.abs(d[lo] - (1 - a[lo]))) < 1e-15
    assert np.max(np.abs(d - (1 - a))) < 1e-14
    # symmetric in its two endpoints, bit for bit
    d2 = oracle_mod.affinity(n, g.v, g.u, X)
    assert np.array_equal(d, d2)
    # scale invariant per row
    d3 = oracle_mod.affinity(n, g.u, g.v, X * rng.uniform(0.5, 3.0, size=(n, 1)))
    assert np.max(np.abs(d3 - d)) < 1e-14


def test_affinity_path_distance_scaling(oracle_mod):
    # Sec. 3.2.2: on a path graph d_{p,q} grows like (p - q)^2
    n = 2000
    g = W.path(n)
    X = oracle_mod.smooth(n, g.u, g.v, g.w, 8, 100)
    p = np.arange(800, 1200)
    med = [np.median(oracle_mod.affinity(n, p, p + s, X)) for s in (1, 2, 3)]
    assert 3.8 < med[1] / med[0] < 4.2
    assert 8.0 < med[2] / med[0] < 9.5


# ---------------------------------------------------------------------------
# Aggregation (Sec. 3.2.2, reading: greedy matching in (d, edge id) order)
# ---------------------------------------------------------------------------
def test_aggregate_hand_examples(oracle_mod):
    u = np.array([0, 1, 2], np.int32)
    v = np.array([1, 2, 3], np.int32)
    d = np.array([0.1, 0.3, 0.2])
    # pass 1 merges {0,1} and {2,3}; pass 2 merges the two pairs through edge 1
    agg, nc = oracle_mod.aggregate(4, u, v, d, 1, 2)
    assert nc == 1 and list(agg) == [0, 0, 0, 0]
    agg, nc = oracle_mod.aggregate(4, u, v, d, 2, 2)
    assert nc == 2 and list(agg) == [0, 0, 1, 1]
    # target 3 allows one merge: the smallest key, edge 0
    agg, nc = oracle_mod.aggregate(4, u, v, d, 3, 2)
    assert nc == 3 and list(agg) == [0, 0, 1, 2]
    # equal distances: the smaller edge id wins
    agg, nc = oracle_mod.aggregate(3, u[:2], v[:2], np.array([0.5, 0.5]), 1, 1)
    assert list(agg) == [0, 0, 1]
    # labels are ranks of the smallest member: {0,3} then {1,2}
    u2 = np.array([0, 1, 1, 2], np.int32)
    v2 = np.array([3, 2, 3, 3], np.int32)
    agg, nc = oracle_mod.aggregate(4, u2, v2, np.array([0.1, 0.2, 0.9, 0.9]), 1, 1)
    assert nc == 2 and list(agg) == [0, 1, 1, 0]


def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        es = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        yield es


def test_aggregate_equals_handshake_exhaustive(oracle_mod):
    rng = np.random.default_rng(6)
    count = 0
    for n in (2, 3, 4, 5):
        for es in _all_graphs(n):
            if not es:
                continue
            u = np.array([e[0] for e in es], np.int32)
            v = np.array([e[1] for e in es], np.int32)
            d = rng.permutation(len(es)).astype(np.float64) / len(es)
            for passes, target in ((1, 1), (2, 1), (2, n - 1), (3, 2)):
                agg, nc = oracle_mod.aggregate(n, u, v, d, target, passes)
                ref, rnc = handshake_aggregate(n, u, v, d, target, passes)
                assert nc == rnc and list(agg) == ref, (n, es, passes, target)
                count += 1
    assert count > 4000


@pytest.mark.parametrize("seed", range(6))
def test_aggregate_equals_handshake_random(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 150))
    g = W.random_sparse(n, 3 * n, seed=seed)
    # coarse distance values force many exact ties, broken by edge id
    d = np.round(rng.uniform(0, 1, size=g.m), 1)
    for passes, target in ((1, 1), (2, n // 4), (3, 1), (2, n - 5)):
        agg, nc = oracle_mod.aggregate(n, g.u, g.v, d, target, passes)
        ref, rnc = handshake_aggregate(n, g.u, g.v, d, target, passes)
        assert nc == rnc and list(agg) == ref


def test_aggregate_matching_properties(oracle_mod):
    g = W.random_sparse(300, 1200, seed=7)
    rng = np.random.default_rng(8)
    d = rng.uniform(size=g.m)
    agg, nc = oracle_mod.aggregate(g.n, g.u, g.v, d, 1, 1)
    sizes = np.bincount(agg, minlength=nc)
    assert sizes.max() <= 2
    inner = agg[g.u] == agg[g.v]
    # every pair is joined by an edge
    assert inner.sum() == (sizes == 2).sum()
    # maximal: no edge joins two singletons
    single = sizes[agg] == 1
    assert not np.any(single[g.u] & single[g.v])
    # greedy certificate: every unmatched edge has an end matched by a smaller
    # (d, id) edge -- together with validity this characterises the greedy
    # matching uniquely
    INF = (np.inf, g.m)
    mkey = [INF] * g.n
    for e in np.nonzero(inner)[0]:
        mkey[g.u[e]] = mkey[g.v[e]] = (d[e], e)
    for f in np.nonzero(~inner)[0]:
        assert min(mkey[g.u[f]], mkey[g.v[f]]) < (d[f], f)
    # labels contiguous, smallest member increasing with the label
    first = np.array([np.min(np.nonzero(agg == c)[0]) for c in range(nc)])
    assert np.all(np.diff(first) > 0)


def test_aggregate_passes_and_target(oracle_mod):
    g = W.grid2d(32, 32)
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, 8, 5)
    d = oracle_mod.affinity(g.n, g.u, g.v, X)
    agg1, nc1 = oracle_mod.aggregate(g.n, g.u, g.v, d, 1, 1)
    agg2, nc2 = oracle_mod.aggregate(g.n, g.u, g.v, d, 1, 2)
    assert np.bincount(agg1).max() <= 2 and np.bincount(agg2).max() <= 4
    assert nc2 < nc1 < g.n
    # pass 2 only merges whole pass-1 aggregates
    for c in range(nc1):
        assert len(set(agg2[agg1 == c])) == 1
    # the target is met exactly when truncation is needed
    agg3, nc3 = oracle_mod.aggregate(g.n, g.u, g.v, d, 600, 2)
    assert nc3 == 600


# ---------------------------------------------------------------------------
# Galerkin coarsening L_R = H_G^R L_G H_R^G (Sec. 3.2.2), P 0/1 aggregation
# ---------------------------------------------------------------------------
def _lap_from_edges(n, u, v, w):
    L = np.zeros((n, n))
    for a, b, x in zip(u, v, w):
        L[a, b] -= x
        L[b, a] -= x
        L[a, a] += x
        L[b, b] += x
    return L


def test_galerkin_dense_bruteforce(oracle_mod):
    g = W.random_sparse(60, 200, seed=9)
    rng = np.random.default_rng(10)
    agg = rng.integers(0, 17, size=g.n).astype(np.int32)
    agg[:17] = np.arange(17)  # every label used
    uc, vc, wc = oracle_mod.coarsen(g.n, g.u, g.v, g.w, agg, 17)
    P = np.zeros((g.n, 17))
    P[np.arange(g.n), agg] = 1.0
    ref = P.T @ oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w) @ P
    Lc = _lap_from_edges(17, uc, vc, wc)
    assert np.max(np.abs(Lc - ref)) <= 1e-13 * np.abs(ref).max()
    # canonical, same sparsity pattern as P^T L P
    assert np.all(uc < vc)
    keys = uc.astype(np.int64) * 17 + vc
    assert np.all(np.diff(keys) > 0)
    pattern = {(a, b) for a in range(17) for b in range(a + 1, 17) if abs(ref[a, b]) > 0}
    assert pattern == set(zip(uc.tolist(), vc.tolist()))


def test_galerkin_invariants(oracle_mod):
    g = W.grid2d(30, 30)
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, 8, 5)
    d = oracle_mod.affinity(g.n, g.u, g.v, X)
    agg, nc = oracle_mod.aggregate(g.n, g.u, g.v, d, 225, 2)
    uc, vc, wc = oracle_mod.coarsen(g.n, g.u, g.v, g.w, agg, nc)
    # constant null space kept: L_c 1 = 0
    Lc1 = oracle_mod.laplacian_apply(nc, uc, vc, wc, np.ones(nc))
    assert np.max(np.abs(Lc1)) < 1e-12
    # total weight = fine weight minus the weight inside aggregates
    internal = g.w[agg[g.u] == agg[g.v]].sum()
    assert np.isclose(wc.sum(), g.w.sum() - internal, rtol=1e-14)
    # quadratic form of piecewise-constant vectors is preserved
    rng = np.random.default_rng(12)
    for _ in range(3):
        y = rng.normal(size=nc)
        Py = y[agg]
        lhs = y @ oracle_mod.laplacian_apply(nc, uc, vc, wc, y)
        rhs = Py @ oracle_mod.laplacian_apply(g.n, g.u, g.v, g.w, Py)
        assert np.isclose(lhs, rhs, rtol=1e-12)


def test_galerkin_hand_example(oracle_mod):
    u = np.array([0, 1, 2], np.int32)
    v = np.array([1, 2, 3], np.int32)
    w = np.array([1.0, 2.0, 3.0])
    uc, vc, wc = oracle_mod.coarsen(4, u, v, w, np.array([0, 0, 1, 1], np.int32), 2)
    assert list(uc) == [0] and list(vc) == [1] and list(wc) == [2.0]
    # a square 0-1-2-3-0 with aggregates {0,2} {1,3}: four crossing edges
    u = np.array([0, 0, 1, 2], np.int32)
    v = np.array([1, 3, 2, 3], np.int32)
    w = np.array([1.0, 2.0, 4.0, 8.0])
    uc, vc, wc = oracle_mod.coarsen(4, u, v, w, np.array([0, 1, 0, 1], np.int32), 2)
    assert list(wc) == [15.0]


# ---------------------------------------------------------------------------
# Eigenvalue check solvers (method of the fe_tooth eigenvalue figure)
# ---------------------------------------------------------------------------
def test_eig_solver_closed_forms(oracle_mod):
    g = W.grid2d(40, 30)
    i, j = np.meshgrid(np.arange(40), np.arange(30))
    ref = np.sort((4 * np.sin(np.pi * i / 80) ** 2 + 4 * np.sin(np.pi * j / 60) ** 2).ravel())[1:11]
    for dense_max in (100000, 0):  # dense eigh and shift-invert eigsh
        ev = oracle_mod.smallest_nontrivial_eigs(g.n, g.u, g.v, g.w, 10, dense_max=dense_max)
        assert np.allclose(ev, ref, rtol=1e-9, atol=1e-12)
    g = W.cycle(50)
    ev = oracle_mod.smallest_nontrivial_eigs(g.n, g.u, g.v, g.w, 6)
    ref = np.sort(4 * np.sin(np.pi * np.arange(50) / 50) ** 2)[1:7]
    assert np.allclose(ev, ref, rtol=0, atol=1e-12)
    # two components: two zeros skipped
    u = np.concatenate([W.path(10).u, W.path(10).u + 10]).astype(np.int32)
    v = np.concatenate([W.path(10).v, W.path(10).v + 10]).astype(np.int32)
    ev = oracle_mod.smallest_nontrivial_eigs(20, u, v, np.ones(18), 4)
    jj = np.arange(1, 10)
    ref = np.sort(np.repeat(4 * np.sin(np.pi * jj / 20) ** 2, 2))[:4]
    assert np.allclose(ev, ref, rtol=0, atol=1e-12)
    # 3-D mesh: sums of three 4 sin^2 terms
    g = W.mesh3d(5, 4, 3)
    g.w[:] = 1.0
    ev = oracle_mod.smallest_nontrivial_eigs(g.n, g.u, g.v, g.w, 5)
    t = [4 * np.sin(np.pi * np.arange(k) / (2 * k)) ** 2 for k in (5, 4, 3)]
    ref = np.sort((t[0][None, None, :] + t[1][None, :, None] + t[2][:, None, None]).ravel())[1:6]
    assert np.allclose(ev, ref, rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------
# Spectral-mismatch loss and its hand-derived adjoint
# ---------------------------------------------------------------------------
def _small_reduction(oracle_mod, seed=13, n=60):
    g = W.random_sparse(n, 3 * n, seed=seed)
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, 4, 3)
    d = oracle_mod.affinity(g.n, g.u, g.v, X)
    agg, nc = oracle_mod.aggregate(g.n, g.u, g.v, d, max(n // 4, 2), 2)
    uc, vc, wc = oracle_mod.coarsen(g.n, g.u, g.v, g.w, agg, nc)
    return g, X, agg, nc, uc, vc, wc


def _fd_check(oracle_mod, g, X, agg, nc, uc, vc, wc, S, h=1e-4):
    L0, grad, _, _ = oracle_mod.loss(g.n, g.u, g.v, g.w, nc, uc, vc, wc, agg, X, S)
    fd = np.empty_like(wc)
    for e in range(len(wc)):
        wp = wc.copy()
        wp[e] += h
        wm = wc.copy()
        wm[e] -= h
        lp = oracle_mod.loss(g.n, g.u, g.v, g.w, nc, uc, vc, wp, agg, X, S, want_grad=False)[0]
        lm = oracle_mod.loss(g.n, g.u, g.v, g.w, nc, uc, vc, wm, agg, X, S, want_grad=False)[0]
        fd[e] = (lp - lm) / (2 * h)
    floor = 1e-10 * np.abs(grad).max()
    rel = np.abs(grad - fd) / np.maximum(np.abs(fd), floor)
    return L0, grad, fd, rel


@pytest.mark.parametrize("S", [0, 1, 3, 5])
def test_loss_gradient_finite_differences(oracle_mod, S):
    g, X, agg, nc, uc, vc, wc = _small_reduction(oracle_mod)
    L0, grad, fd, rel = _fd_check(oracle_mod, g, X, agg, nc, uc, vc, wc, S)
    assert L0 > 0
    assert np.all((rel <= 1e-5) | (np.abs(grad - fd) <= 1e-10 * np.abs(grad).max())), rel.max()


def test_loss_zero_for_piecewise_constant_vectors(oracle_mod):
    # x_k = P z_k with M-weighted mean zero: y0 = z, R_c(y0) = R_f(x), loss 0
    g, _, agg, nc, uc, vc, wc = _small_reduction(oracle_mod, seed=21)
    rng = np.random.default_rng(22)
    Z = rng.normal(size=(nc, 3))
    M = np.bincount(agg, minlength=nc).astype(float)
    Z -= (M @ Z) / M.sum()
    X = Z[agg]
    L0, _, Rf, Rc = oracle_mod.loss(g.n, g.u, g.v, g.w, nc, uc, vc, wc, agg, X, 0)
    assert np.allclose(Rc, Rf, rtol=1e-12)
    assert L0 < 1e-24


def test_loss_scale_invariance(oracle_mod):
    g, X, agg, nc, uc, vc, wc = _small_reduction(oracle_mod, seed=31)
    for S in (0, 4):
        l1 = oracle_mod.loss(g.n, g.u, g.v, g.w, nc, uc, vc, wc, agg, X, S, want_grad=False)[0]
        l2 = oracle_mod.loss(g.n, g.u, g.v, g.w, nc, uc, vc, wc, agg, 3.0 * X, S, want_grad=False)[0]
        assert np.isclose(l1, l2, rtol=1e-12)


# ---------------------------------------------------------------------------
# Level loop and stored oracle results
# ---------------------------------------------------------------------------
def test_multilevel_grid(oracle_mod):
    g = W.grid2d(64, 64)
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, 8, 5, final_target=64)
    ns = [lv.n for lv in levels] + [levels[-1].nc]
    assert ns[0] == 4096 and ns[-1] <= 64
    assert all(b < a for a, b in zip(ns, ns[1:]))
    comp = oracle_mod.compose_maps(levels)
    assert comp.min() == 0 and comp.max() == levels[-1].nc - 1


def test_golden_grid64(oracle_mod):
    """The committed script tests/golden/make_golden.py wrote this file by
    calling the oracle; it also guards the oracle's bit-stability across
    machines (x86 here, Arm on the GPU host)."""
    import hashlib
    with open(os.path.join(GOLDEN, "grid64_oracle.json")) as f:
        ref = json.load(f)
    g = W.grid2d(64, 64)
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, 8, 5, 0.7, 0, 0)
    d = oracle_mod.affinity(g.n, g.u, g.v, X)
    agg, nc = oracle_mod.aggregate(g.n, g.u, g.v, d, 1024, 2)
    uc, vc, wc = oracle_mod.coarsen(g.n, g.u, g.v, g.w, agg, nc)
    assert hashlib.sha256(X.tobytes()).hexdigest() == ref["X_sha256"]
    assert hashlib.sha256(d.tobytes()).hexdigest() == ref["d_sha256"]
    assert nc == ref["nc"] and len(uc) == ref["mc"]
    assert hashlib.sha256(agg.tobytes()).hexdigest() == ref["agg_sha256"]
    assert float(wc.sum()) == ref["wc_sum"]


# ---------------------------------------------------------------------------
# Multilevel eigensolver (Alg. 5): shifted Jacobi, coarsest eigenpairs,
# Gram-Schmidt, the level loop
# ---------------------------------------------------------------------------
def _cycle_weighted(n, wt):
    u = np.arange(n - 1, dtype=np.int32)
    v = np.arange(1, n, dtype=np.int32)
    u = np.concatenate([np.array([0], np.int32), u])
    v = np.concatenate([np.array([n - 1], np.int32), v])
    order = np.lexsort((v, u))
    return W.Graph(n, u[order], v[order], np.full(n, wt))


@pytest.mark.parametrize("normalized", [False, True])
def test_shifted_jacobi_fixed_point_on_cycle_eigenvectors(oracle_mod, normalized):
    # unit-free closed form: on a cycle of weight c, L cos(2 pi j i / n) =
    # 2c (1 - cos(2 pi j / n)) cos(...), D = 2c I; an exact eigenpair of
    # (L, B) is a fixed point of every shifted Jacobi iteration
    n, c = 24, 1.5
    g = _cycle_weighted(n, c)
    i = np.arange(n)
    js = [1, 2, 5]
    Y = np.stack([np.cos(2 * np.pi * j * i / n) for j in js], 1)
    lam = np.array([2 * c * (1 - np.cos(2 * np.pi * j / n)) for j in js])
    if normalized:
        lam = lam / (2 * c)
    out = oracle_mod.shifted_jacobi(n, g.u, g.v, g.w, Y, lam, normalized, 0.7, 5)
    assert np.max(np.abs(out - Y)) <= 1e-12
    # a wrong shift moves the vector (the check above is not vacuous)
    moved = oracle_mod.shifted_jacobi(n, g.u, g.v, g.w, Y, lam * 0.5, normalized, 0.7, 1)
    assert np.max(np.abs(moved - Y)) > 1e-3


@pytest.mark.parametrize("normalized", [False, True])
def test_shifted_jacobi_fixed_point_generalized(oracle_mod, normalized):
    from scipy.linalg import eigh
    g = W.random_sparse(40, 150, seed=11)
    L = oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w)
    B = np.diag(np.diag(L)) if normalized else np.eye(g.n)
    lam, U = eigh(L, B)  # LAPACK's generalized solver, not the oracle's reduction
    k = [1, 2, 3, 7]
    out = oracle_mod.shifted_jacobi(g.n, g.u, g.v, g.w, U[:, k], lam[k], normalized, 0.7, 4)
    assert np.max(np.abs(out - U[:, k])) <= 1e-10


def test_shifted_jacobi_keeps_rows_with_nonpositive_diagonal(oracle_mod):
    # node 5 is isolated; node 0 has degree 0.2 < shift 0.5 (ratio cut)
    u = np.array([0, 1, 2, 3], np.int32)
    v = np.array([1, 2, 3, 4], np.int32)
    w = np.array([0.2, 1.0, 1.0, 1.0])
    Y = np.arange(12, dtype=np.float64).reshape(6, 2) + 1.0
    out = oracle_mod.shifted_jacobi(6, u, v, w, Y, np.array([0.5, 0.0]), False, 0.7, 1)
    assert out[5, 0] == Y[5, 0] and out[5, 1] == Y[5, 1]
    assert out[0, 0] == Y[0, 0]  # 0.2 - 0.5 <= 0
    # node 0, column 1 (shift 0): the plain Alg. 3 update toward its neighbour
    assert np.isclose(out[0, 1], 0.3 * Y[0, 1] + 0.7 * Y[1, 1])


def test_coarsest_eigenpairs_closed_forms(oracle_mod):
    n = 30
    p = W.path(n)
    lam, U = oracle_mod.coarsest_eigenpairs(p.n, p.u, p.v, p.w, 6, False)
    assert np.allclose(lam, 4 * np.sin(np.pi * np.arange(6) / (2 * n)) ** 2, rtol=0, atol=1e-12)
    assert np.allclose(U.T @ U, np.eye(6), rtol=0, atol=1e-12)
    # normalised cut on a regular graph: the spectrum divides by the degree
    c = _cycle_weighted(20, 2.0)
    lam_n, Un = oracle_mod.coarsest_eigenpairs(c.n, c.u, c.v, c.w, 5, True)
    lam_r, _ = oracle_mod.coarsest_eigenpairs(c.n, c.u, c.v, c.w, 5, False)
    assert np.allclose(lam_n, lam_r / 4.0, rtol=0, atol=1e-12)


def test_coarsest_eigenpairs_generalized_against_lapack(oracle_mod):
    from scipy.linalg import eigh
    g = W.random_sparse(35, 120, seed=12)
    L = oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w)
    D = np.diag(np.diag(L))
    lam, U = oracle_mod.coarsest_eigenpairs(g.n, g.u, g.v, g.w, 8, True)
    ref = eigh(L, D, eigvals_only=True)[:8]
    assert np.allclose(lam, ref, rtol=0, atol=1e-11)
    assert np.max(np.abs(L @ U - (D @ U) * lam)) <= 1e-10
    assert np.allclose(U.T @ D @ U, np.eye(8), rtol=0, atol=1e-10)  # B-orthonormal


def test_gram_schmidt_properties(oracle_mod):
    rng = np.random.default_rng(13)
    A = rng.normal(size=(50, 6))
    Q = oracle_mod.gram_schmidt(A)
    assert np.allclose(Q.T @ Q, np.eye(6), rtol=0, atol=1e-12)
    # column order: span(Q[:, :j]) = span(A[:, :j]) for every j, and the
    # first column is the first input column normalised
    for j in range(1, 7):
        P = Q[:, :j] @ Q[:, :j].T
        assert np.allclose(P @ A[:, :j], A[:, :j], rtol=0, atol=1e-10)
    assert np.allclose(Q[:, 0], A[:, 0] / np.linalg.norm(A[:, 0]), rtol=0, atol=1e-15)
    # numpy's QR gives the same factor up to column signs
    Qr, _ = np.linalg.qr(A)
    assert np.allclose(np.abs(np.sum(Qr * Q, 0)), 1.0, rtol=0, atol=1e-10)


def test_multilevel_eigensolve_single_level_is_exact(oracle_mod):
    n = 40
    p = W.path(n)
    U, lam = oracle_mod.multilevel_eigensolve([(p.n, p.u, p.v, p.w)], [], 5)
    L = oracle_mod.dense_laplacian(p.n, p.u, p.v, p.w)
    rq = np.sum(U * (L @ U), 0)
    assert np.allclose(rq, 4 * np.sin(np.pi * np.arange(5) / (2 * n)) ** 2, rtol=0, atol=1e-12)


def test_multilevel_eigensolve_prolongation_and_refinement(oracle_mod):
    # two levels of a path: pairs (2i, 2i+1) aggregated; with no smoothing the
    # result is constant on every pair, and smoothing lowers the Rayleigh
    # quotients of the low modes toward the true eigenvalues
    n = 64
    p = W.path(n)
    agg = (np.arange(n) // 2).astype(np.int32)
    uc, vc, wc = oracle_mod.coarsen(p.n, p.u, p.v, p.w, agg, n // 2)
    graphs = [(p.n, p.u, p.v, p.w), (n // 2, uc, vc, wc)]
    U0, lam = oracle_mod.multilevel_eigensolve(graphs, [agg], 4, iters=0)
    assert np.allclose(U0[0::2], U0[1::2], rtol=0, atol=0)
    assert np.allclose(U0.T @ U0, np.eye(4), rtol=0, atol=1e-12)
    L = oracle_mod.dense_laplacian(p.n, p.u, p.v, p.w)
    U1, _ = oracle_mod.multilevel_eigensolve(graphs, [agg], 4, iters=20)
    exact = 4 * np.sin(np.pi * np.arange(4) / (2 * n)) ** 2
    rq0 = np.sum(U0 * (L @ U0), 0)
    rq1 = np.sum(U1 * (L @ U1), 0)
    # the first column stays the constant vector (shift 0 fixes it), so every
    # later column is orthogonal to it and, by Courant-Fischer, its Rayleigh
    # quotient is at least the second eigenvalue
    assert np.allclose(U1[:, 0], U1[0, 0], rtol=0, atol=1e-12)
    assert np.all(rq0[1:] >= exact[1] - 1e-12) and np.all(rq1[1:] >= exact[1] - 1e-12)
    assert np.all(np.abs(rq1[1:] - exact[1:]) < np.abs(rq0[1:] - exact[1:]))


def _two_level_random(oracle_mod, seed, n=90, m=260):
    g = W.random_sparse(n, m, seed=seed)
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, 8, 4, final_target=14)
    assert len(levels) >= 2
    graphs = [(g.n, g.u, g.v, g.w)] + [(lv.nc, lv.uc, lv.vc, lv.wc) for lv in levels]
    maps = [lv.agg for lv in levels]
    return g, graphs, maps


@pytest.mark.parametrize("normalized", [False, True])
def test_galerkin_mass_is_rayleigh_ritz(oracle_mod, normalized):
    # With B_l = P^T B_(l-1) P the coarsest problem is the projection of the
    # finest (L, B) onto the piecewise-constant vectors Q (Q = P_1 P_2 ...):
    # its eigenvalues are those of (Q^T L Q, Q^T B Q), computed here by a dense
    # generalised solver, independently of the level-by-level Galerkin
    # products and mass sums.  The level's own mass fails the identity.
    import scipy.linalg
    g, graphs, maps = _two_level_random(oracle_mod, 41 + int(normalized))
    n, nc = g.n, graphs[-1][0]
    Q = np.zeros((n, nc))
    Q[np.arange(n), _compose(maps)] = 1.0
    L = oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w)
    b0 = oracle_mod.degrees(g.n, g.u, g.v, g.w) if normalized else np.ones(n)
    ref = scipy.linalg.eigh(Q.T @ L @ Q, Q.T @ np.diag(b0) @ Q, eigvals_only=True)[:6]
    _, lam = oracle_mod.multilevel_eigensolve(graphs, maps, 6, normalized, iters=0, mass="galerkin")
    assert np.allclose(lam, ref, rtol=1e-10, atol=1e-12)
    _, lam_level = oracle_mod.multilevel_eigensolve(graphs, maps, 6, normalized, iters=0, mass="level")
    assert not np.allclose(lam_level, ref, rtol=1e-3, atol=1e-6)
    # Courant-Fischer: each is an upper bound of the finest generalised eigenvalue
    fine = scipy.linalg.eigh(L, np.diag(b0), eigvals_only=True)[:6]
    assert np.all(lam >= fine - 1e-10)


def _compose(maps):
    out = np.asarray(maps[0], np.int64)
    for mp in maps[1:]:
        out = np.asarray(mp, np.int64)[out]
    return out


def test_galerkin_mass_path_pairs_closed_form(oracle_mod):
    # path of 64 unit edges, pairs (2i, 2i+1) aggregated: the coarse graph is
    # the path of 32 unit edges with mass 2 on every node, so its eigenvalues
    # are 4 sin^2(pi j / 64) / 2
    n = 64
    p = W.path(n)
    agg = (np.arange(n) // 2).astype(np.int32)
    uc, vc, wc = oracle_mod.coarsen(p.n, p.u, p.v, p.w, agg, n // 2)
    graphs = [(p.n, p.u, p.v, p.w), (n // 2, uc, vc, wc)]
    B = oracle_mod.galerkin_masses(graphs, [agg])
    assert np.array_equal(B[1], np.full(n // 2, 2.0))
    _, lam = oracle_mod.multilevel_eigensolve(graphs, [agg], 6, iters=0, mass="galerkin")
    j = np.arange(6)
    assert np.allclose(lam, 2.0 * np.sin(np.pi * j / n) ** 2, rtol=0, atol=1e-12)


def test_galerkin_masses_are_member_sums(oracle_mod):
    g, graphs, maps = _two_level_random(oracle_mod, 43)
    for normalized in (False, True):
        B = oracle_mod.galerkin_masses(graphs, maps, normalized)
        b0 = oracle_mod.degrees(g.n, g.u, g.v, g.w) if normalized else np.ones(g.n)
        comp = _compose(maps)
        direct = np.zeros(graphs[-1][0])
        np.add.at(direct, comp, b0)
        assert np.allclose(B[-1], direct, rtol=1e-14, atol=0)
        assert abs(B[-1].sum() - b0.sum()) <= 1e-12 * b0.sum()


def test_shifted_jacobi_mass_fixed_point(oracle_mod):
    # eigenpairs of (L, diag(b)) for a random positive b are fixed points of the
    # explicit-mass iteration; with the wrong mass (b = 1) they move
    import scipy.linalg
    g = W.random_sparse(50, 140, seed=44)
    rng = np.random.default_rng(5)
    b = rng.uniform(0.5, 3.0, g.n)
    L = oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w)
    lam, U = scipy.linalg.eigh(L, np.diag(b))
    lam, U = lam[:4], U[:, :4]
    Y = oracle_mod.shifted_jacobi_mass(g.n, g.u, g.v, g.w, U, lam, b, 0.7, 5)
    deg = oracle_mod.degrees(g.n, g.u, g.v, g.w)
    keep = np.all(deg[:, None] - lam[None, :] * b[:, None] > 0, axis=1)
    assert np.allclose(Y[keep], U[keep], rtol=0, atol=1e-10)
    Yw = oracle_mod.shifted_jacobi_mass(g.n, g.u, g.v, g.w, U, lam, np.ones(g.n), 0.7, 5)
    assert not np.allclose(Yw[:, 1:], U[:, 1:], rtol=0, atol=1e-6)


# ---------------------------------------------------------------------------
# Reduced data set (Alg. 6, step 4): F_R = P^T F
# ---------------------------------------------------------------------------
def test_reduce_features_against_dense_product(oracle_mod):
    rng = np.random.default_rng(31)
    n, nc, d = 200, 37, 5
    agg = np.concatenate([np.arange(nc), rng.integers(0, nc, n - nc)]).astype(np.int32)
    F = rng.normal(size=(n, d))
    P = np.zeros((n, nc))
    P[np.arange(n), agg] = 1.0
    assert np.allclose(oracle_mod.reduce_features(agg, nc, F), P.T @ F, rtol=0, atol=1e-12)
    # mean: (P^T P)^-1 P^T F
    M = np.diag(1.0 / np.diag(P.T @ P))
    assert np.allclose(oracle_mod.reduce_features(agg, nc, F, mean=True), M @ P.T @ F, rtol=0, atol=1e-12)


def test_reduce_features_invariants(oracle_mod):
    rng = np.random.default_rng(32)
    n, nc = 300, 40
    agg = np.concatenate([np.arange(nc), rng.integers(0, nc, n - nc)]).astype(np.int32)
    Fi = rng.integers(-50, 50, size=(n, 3)).astype(np.float64)  # integers: every sum exact
    R = oracle_mod.reduce_features(agg, nc, Fi)
    assert np.array_equal(R.sum(0), Fi.sum(0))
    assert np.array_equal(oracle_mod.reduce_features(np.arange(n, dtype=np.int32), n, Fi), Fi)
    c = np.full((n, 2), 2.5)
    assert np.array_equal(oracle_mod.reduce_features(agg, nc, c, mean=True), np.full((nc, 2), 2.5))


# ---------------------------------------------------------------------------
# Multicolour Gauss-Seidel (Sec. 3.2.1): colouring and sweeps
# ---------------------------------------------------------------------------
def _prio(oracle_mod, n, seed):
    return np.array([oracle_mod.splitmix64(seed, (1 << 62) + i) for i in range(n)], dtype=np.uint64)


@pytest.mark.parametrize("seed", [0, 7])
def test_colouring_is_greedy_and_proper(oracle_mod, seed):
    from colouring_ref import jones_plassmann
    for g in (W.random_sparse(300, 1500, seed=51), W.grid2d(12, 9), W.star(30), W.complete(12, 1.0),
              W.mesh3d(6, 5, 4, seed=52)):
        col, nc = oracle_mod.colour(g.n, g.u, g.v, seed)
        assert np.all(col[g.u] != col[g.v])
        deg = np.bincount(np.concatenate([g.u, g.v]), minlength=g.n)
        assert nc == col.max() + 1 and nc <= deg.max() + 1
        assert np.array_equal(col, jones_plassmann(g.n, g.u, g.v, _prio(oracle_mod, g.n, seed)))


def _sor_dense(oracle_mod, g, X, order, omega):
    """One sweep in matrix form: with A split by the visiting order into the
    part already updated (lower) and the rest (upper),
    (D - omega A_low) x_new = ((1 - omega) D + omega A_up) x_old."""
    from scipy.linalg import solve_triangular
    L = oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w)
    D = np.diag(L).copy()
    A = np.diag(D) - L
    pos = np.empty(g.n, np.int64)
    pos[order] = np.arange(g.n)
    Ap = A[np.ix_(order, order)]
    low, up = np.tril(Ap, -1), np.triu(Ap, 1)
    Dp = np.diag(D[order])
    rhs = ((1 - omega) * Dp + omega * up) @ X[order]
    Xn = solve_triangular(Dp - omega * low, rhs, lower=True)
    out = np.empty_like(X)
    out[order] = Xn
    return out


@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_gs_sweep_matrix_form(oracle_mod, omega):
    g = W.random_sparse(60, 250, seed=53)
    rng = np.random.default_rng(54)
    X = rng.normal(size=(g.n, 3))
    col, _ = oracle_mod.colour(g.n, g.u, g.v, 3)
    for order in (oracle_mod.gs_order(col), np.arange(g.n), rng.permutation(g.n)):
        got = oracle_mod.gs_sweeps(g.n, g.u, g.v, g.w, X, order, 1, omega)
        assert np.allclose(got, _sor_dense(oracle_mod, g, X, np.asarray(order), omega), rtol=0, atol=1e-12)


def test_gs_fixes_constants_and_colour_classes_are_independent(oracle_mod):
    g = W.mesh3d(5, 4, 3, seed=55)
    c = np.full((g.n, 2), 3.25)
    col, _ = oracle_mod.colour(g.n, g.u, g.v, 1)
    order = oracle_mod.gs_order(col)
    assert np.allclose(oracle_mod.gs_sweeps(g.n, g.u, g.v, g.w, c, order, 3), c, rtol=0, atol=1e-14)
    # inside one colour the visiting order does not matter: reversing the ids
    # within every colour class gives the same sweep, bit for bit
    rev = np.lexsort((-np.arange(g.n), col)).astype(np.int64)
    X = np.random.default_rng(56).normal(size=(g.n, 4))
    assert np.array_equal(oracle_mod.gs_sweeps(g.n, g.u, g.v, g.w, X, order, 2),
                          oracle_mod.gs_sweeps(g.n, g.u, g.v, g.w, X, rev, 2))


def test_smooth_gs_invariants(oracle_mod):
    g = W.random_sparse(200, 900, seed=57)
    X = oracle_mod.smooth_gs(g.n, g.u, g.v, g.w, 6, 4, 0.7, 3, 1, 5)
    assert np.allclose(X.sum(0), 0.0, rtol=0, atol=1e-12) and np.allclose((X * X).sum(0), 1.0, rtol=0, atol=1e-12)
    # the low-pass effect (Sec. 3.2.1): Rayleigh quotients fall below those of
    # the raw centred vectors
    L = oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w)
    X0 = oracle_mod.smooth_gs(g.n, g.u, g.v, g.w, 6, 0, 0.7, 3, 1, 5)
    assert np.all(np.sum(X * (L @ X), 0) < np.sum(X0 * (L @ X0), 0))


# ---------------------------------------------------------------------------
# Edge scaling (Alg. 1 driven by the loss gradient)
# ---------------------------------------------------------------------------
def _scaling_case(oracle_mod, seed=71):
    g = W.random_sparse(400, 1600, seed=seed)
    lv = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, 8, 5, final_target=60)
    agg = oracle_mod.compose_maps(lv)
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, 8, 5)
    return g, lv[-1], agg, X


def test_scale_edges_zero_step_and_monotone(oracle_mod):
    g, c, agg, X = _scaling_case(oracle_mod)
    w0, h0 = oracle_mod.scale_edges(g.n, g.u, g.v, g.w, c.nc, c.uc, c.vc, c.wc, agg, X, eta_max=0.0, kmax=5)
    assert np.array_equal(w0, c.wc) and len(h0) == 1 and h0[0][1] == 1.0
    w, h = oracle_mod.scale_edges(g.n, g.u, g.v, g.w, c.nc, c.uc, c.vc, c.wc, agg, X, eta_max=5.0, kmax=6, eps=0.0)
    assert len(h) == 6 and np.all(w >= c.wc) and np.any(w > c.wc)
    # descent: every update lowered the loss (a flipped gradient sign raises it)
    losses = [x[0] for x in h] + [oracle_mod.loss(g.n, g.u, g.v, g.w, c.nc, c.uc, c.vc, w, agg, X, 5)[0]]
    assert all(b < a for a, b in zip(losses, losses[1:]))


def test_scale_edges_lambda1_estimate_bounds_the_spectrum(oracle_mod):
    # Courant-Fischer: d_G(p)/d_P(p) is the quotient of the indicator of p,
    # whose part orthogonal to 1 has the same quotient, so the estimate is at
    # least the smallest generalised eigenvalue of (L_G, L_P) on 1-perp
    from scipy.linalg import eigh, null_space
    g, c, agg, X = _scaling_case(oracle_mod)
    w, h = oracle_mod.scale_edges(g.n, g.u, g.v, g.w, c.nc, c.uc, c.vc, c.wc, agg, X, eta_max=20.0, kmax=4, eps=0.0)
    LG = oracle_mod.dense_laplacian(c.nc, c.uc, c.vc, c.wc)
    LP = oracle_mod.dense_laplacian(c.nc, c.uc, c.vc, w)
    Q = null_space(np.ones((1, c.nc)))
    lam_min = eigh(Q.T @ LG @ Q, Q.T @ LP @ Q, eigvals_only=True)[0]
    assert h[-1][1] >= lam_min - 1e-12
    assert lam_min < 1.0  # the scaling moved the spectrum (the check is not vacuous)


def test_scale_edges_cap_binds_on_a_matching(oracle_mod):
    # fine graph: 30 disjoint weighted paths of 4 nodes, aggregates {0,1} and
    # {2,3} of each path, so the reduced graph is 30 disjoint edges: no two
    # edges share a node, every update sees the true degrees, and a huge step
    # is capped so that d_G(p)/d_P(p) equals the bound lambda_1 * Delta
    # (= delta_bar^(1/kmax) on the first iteration) at every node
    rng = np.random.default_rng(72)
    P = 30
    u = np.concatenate([4 * np.arange(P) + t for t in range(3)]).astype(np.int32)
    v = u + 1
    order = np.lexsort((v, u))
    u, v = u[order], v[order]
    w = rng.uniform(0.5, 2.0, len(u))
    n = 4 * P
    agg = (np.arange(n) // 2).astype(np.int32)
    uc, vc, wc = oracle_mod.coarsen(n, u, v, w, agg, 2 * P)
    assert len(uc) == P
    X = oracle_mod.smooth(n, u, v, w, 4, 2)
    kmax, delta_bar = 4, 0.3
    wn, h = oracle_mod.scale_edges(n, u, v, w, 2 * P, uc, vc, wc, agg, X, eta_max=1e9, delta_bar=delta_bar,
                                   kmax=1, eps=0.0)
    bound = delta_bar ** (1.0 / 1)
    assert np.allclose(wc / wn, bound, rtol=0, atol=1e-14) and h[0][1] == pytest.approx(bound, abs=1e-14)
    wn4, h4 = oracle_mod.scale_edges(n, u, v, w, 2 * P, uc, vc, wc, agg, X, eta_max=1e9, delta_bar=delta_bar,
                                     kmax=kmax, eps=0.0)
    step = delta_bar ** (1.0 / kmax)
    assert np.allclose([x[1] for x in h4], [step ** (k + 1) for k in range(kmax)], rtol=0, atol=1e-13)


def test_smallest_nontrivial_eigs_per_component(oracle_mod):
    # the per-component solve against one dense eigh of the whole Laplacian
    # with its c zeros skipped, through both the dense and the sparse branch
    parts = [W.random_sparse(60, 200, seed=s) for s in range(5)] + [W.grid2d(7, 9)]
    u = np.concatenate([q.u.astype(np.int64) + 60 * i for i, q in enumerate(parts)])
    v = np.concatenate([q.v.astype(np.int64) + 60 * i for i, q in enumerate(parts)])
    w = np.concatenate([q.w for q in parts])
    n = 60 * 5 + 63 + 4  # four isolated nodes at the end
    L = oracle_mod.sparse_laplacian(n, u, v, w).toarray()
    c = oracle_mod.n_components(n, u, v)
    assert c == 10
    ref = np.linalg.eigvalsh(L)[c:c + 12]
    for dmax in (8000, 40):
        got = oracle_mod.smallest_nontrivial_eigs(n, u, v, w, 12, dense_max=dmax)
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-11), (dmax, got, ref)
