"""Multilevel Laplacian eigensolver (Alg. 5) on the GPU against the oracle.

The hierarchy comes from the oracle's own reduction; the GPU contexts are
rebuilt from the oracle's aggregate maps with graph_reduce_coarsen, so both
sides solve the same problem and no oracle input comes from the CUDA path.
Eigenvectors are compared up to the sign of each column (the coarsest
solver -- Householder tridiagonalisation, bisection and inverse iteration up
to 4,096 nodes, a Chebyshev-filtered subspace iteration beyond -- fixes none); the graphs are connected and have random weights, so the
eigenvalues are simple.  k = 2, 4, 8, 16, 32 take the row-chunk smoothing
kernel, other k the thread-per-entry one.  Every case runs with each level's
own mass B (Alg. 5 as written) and with the Galerkin-consistent mass
B_l = P^T B_(l-1) P.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def gr():
    from paper_1812_08942_gb300 import build as B
    B.build()
    import paper_1812_08942_gb300 as gr
    gr.load()
    return gr


def _hierarchy(gr, oracle_mod, g, final, K=8, sweeps=5):
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, K, sweeps, final_target=final)
    graphs = [(g.n, g.u, g.v, g.w)] + [(lv.nc, lv.uc, lv.vc, lv.wc) for lv in levels]
    maps = [lv.agg for lv in levels]
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    ctxs = [G]
    for lv in levels:
        ctxs.append(gr.graph_reduce_coarsen(ctxs[-1], torch.from_numpy(lv.agg).to(DEV), lv.nc))
    return graphs, maps, ctxs


def _compare(U, Ur, tol):
    U = U.cpu().numpy()
    s = np.sign(np.sum(U * Ur, 0))
    s[s == 0] = 1.0
    return np.max(np.abs(U * s - Ur)) <= tol


CASES = [
    ("mesh_ratio", lambda: W.mesh3d(14, 12, 10, seed=21), 300, False, 6, 8),
    ("mesh_normalized_k8", lambda: W.mesh3d(14, 12, 10, seed=22), 300, True, 8, 8),
    ("rand_ratio_k16", lambda: W.random_sparse(3001, 12000, seed=29), 500, False, 16, 5),
    ("rand_normalized_k32", lambda: W.random_sparse(4000, 16000, seed=30), 600, True, 32, 4),
    ("rand_ratio_k13", lambda: W.random_sparse(3001, 12000, seed=23), 500, False, 13, 5),
    ("rand_normalized_k1", lambda: W.random_sparse(2500, 9000, seed=24), 400, True, 1, 5),
    ("knn_ratio", lambda: W.knn_gmm(4000, 8, 1, 6, 25), 250, False, 8, 10),
]


@pytest.mark.parametrize("galerkin_mass", [False, True], ids=["level_mass", "galerkin_mass"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_eigensolve_parity(gr, oracle_mod, case, galerkin_mass):
    _, make, final, normalized, k, iters = case
    g = make()
    assert oracle_mod.n_components(g.n, g.u, g.v) == 1  # else lambda = 0 repeats and bases differ
    graphs, maps, ctxs = _hierarchy(gr, oracle_mod, g, final)
    assert len(ctxs) >= 3
    Ur, lam_r = oracle_mod.multilevel_eigensolve(graphs, maps, k, normalized, 0.7, iters,
                                                 mass="galerkin" if galerkin_mass else "level")
    U, lam, rq = gr.graph_reduce_eigensolve(ctxs, k, normalized, 0.7, iters, galerkin_mass=galerkin_mass)
    assert np.allclose(lam, lam_r, rtol=1e-10, atol=1e-12)
    assert _compare(U, Ur, 1e-8)
    L = oracle_mod.sparse_laplacian(g.n, g.u, g.v, g.w)
    B = L.diagonal() if normalized else np.ones(g.n)
    rq_r = np.sum(Ur * (L @ Ur), 0) / np.sum(Ur * Ur * B[:, None], 0)
    assert np.allclose(rq, rq_r, rtol=1e-9, atol=1e-12)


def test_eigensolve_single_level_and_no_smoothing(gr, oracle_mod):
    g = W.random_sparse(600, 2500, seed=26)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    U, lam, rq = gr.graph_reduce_eigensolve([G], 5, False, 0.7, 10)
    ref = np.sort(np.linalg.eigvalsh(oracle_mod.dense_laplacian(g.n, g.u, g.v, g.w)))[:5]
    assert np.allclose(lam, ref, atol=1e-10) and np.allclose(rq, ref, atol=1e-10)
    Uh = U.cpu().numpy()
    assert np.allclose(Uh.T @ Uh, np.eye(5), atol=1e-12)
    # a graph no larger than the iteration's block (k + 8 columns): one
    # Rayleigh-Ritz step over the whole space, ratio and normalised cut
    t = W.random_sparse(12, 30, seed=31)
    assert oracle_mod.n_components(t.n, t.u, t.v) == 1
    T = gr.graph_reduce_create(t.n, t.u, t.v, t.w)
    Lt = oracle_mod.dense_laplacian(t.n, t.u, t.v, t.w)
    for normalized in (False, True):
        Ut, lt, _ = gr.graph_reduce_eigensolve([T], 8, normalized, 0.7, 0)
        dt = np.diag(Lt) if normalized else np.ones(t.n)
        ref_t = np.sort(np.linalg.eigvalsh(Lt / np.sqrt(np.outer(dt, dt))))[:8]
        assert np.allclose(lt, ref_t, atol=1e-12)
        Uh = Ut.cpu().numpy()
        assert np.allclose(Uh.T @ Uh, np.eye(8), atol=1e-12)
        if not normalized:  # B = I: the orthonormalised columns stay eigenvectors
            res = Lt @ Uh - Uh * np.asarray(lt)[None, :]
            assert np.max(np.abs(res)) <= 1e-10
    # iters = 0: the finest block is the mapped coarse block, orthonormalised
    graphs, maps, ctxs = _hierarchy(gr, oracle_mod, g, 100)
    Ur, _ = oracle_mod.multilevel_eigensolve(graphs, maps, 4, False, 0.7, 0)
    U0, _, _ = gr.graph_reduce_eigensolve(ctxs, 4, False, 0.7, 0)
    assert _compare(U0, Ur, 1e-9)


def test_eigensolve_many_components(gr, oracle_mod):
    # 24 components of 40 nodes with weights up to ~250: the null space is
    # wider than the iteration's block for k = 8 (the block grows) and the
    # nonzero eigenvalues sit far below the spectral bound
    parts = [W.random_sparse(40, 120, seed=100 + i) for i in range(24)]
    u = np.concatenate([q.u + 40 * i for i, q in enumerate(parts)]).astype(np.int32)
    v = np.concatenate([q.v + 40 * i for i, q in enumerate(parts)]).astype(np.int32)
    w = np.concatenate([q.w * 50.0 for q in parts])
    n = 40 * len(parts)
    assert oracle_mod.n_components(n, u, v) == 24
    G = gr.graph_reduce_create(n, u, v, w)
    L = oracle_mod.dense_laplacian(n, u, v, w)
    ev = np.sort(np.linalg.eigvalsh(L))
    beta = np.max(np.sum(np.abs(L), 1))
    for k in (8, 32):
        U, lam, rq = gr.graph_reduce_eigensolve([G], k, False, 0.7, 0)
        assert np.allclose(lam, ev[:k], rtol=1e-10, atol=1e-11 * beta), (k, lam, ev[:k])
        Uh = U.cpu().numpy()
        assert np.allclose(Uh.T @ Uh, np.eye(k), atol=1e-12)
        # columns of a repeated eigenvalue are any basis of its eigenspace:
        # check the residuals, not the vectors
        res = L @ Uh - Uh * np.asarray(lam)[None, :]
        assert np.max(np.abs(res)) <= 1e-10 * beta, (k, np.max(np.abs(res)))


def test_eigensolve_large_coarsest_level(gr, oracle_mod):
    # a coarsest level above the dense route's 4,096 nodes takes the
    # Chebyshev-filtered subspace iteration: eigenvalues against shift-invert
    # Lanczos, eigenpairs by their residuals, ratio cut
    g = W.mesh3d(20, 16, 17, seed=41)
    assert g.n > 4096 and oracle_mod.n_components(g.n, g.u, g.v) == 1
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    U, lam, rq = gr.graph_reduce_eigensolve([G], 8, False, 0.7, 0)
    ref = oracle_mod.smallest_nontrivial_eigs(g.n, g.u, g.v, g.w, 7)
    assert abs(lam[0]) <= 1e-11
    assert np.allclose(lam[1:], ref, rtol=1e-9, atol=1e-11), (lam, ref)
    L = oracle_mod.sparse_laplacian(g.n, g.u, g.v, g.w)
    Uh = U.cpu().numpy()
    res = L @ Uh - Uh * np.asarray(lam)[None, :]
    assert np.max(np.abs(res)) <= 1e-9


def test_eigensolve_rejects_bad_requests(gr, oracle_mod):
    g = W.random_sparse(500, 2000, seed=27)
    graphs, maps, ctxs = _hierarchy(gr, oracle_mod, g, 100)
    with pytest.raises(gr.GraphReduceError) as ei:
        gr.graph_reduce_eigensolve(ctxs, ctxs[-1].n + 1)
    assert ei.value.status == 1
    with pytest.raises(gr.GraphReduceError):
        gr.graph_reduce_eigensolve(ctxs, 33)
    with pytest.raises(gr.GraphReduceError):  # levels out of order
        gr.graph_reduce_eigensolve([ctxs[0], ctxs[2]], 4)
    big = W.mesh3d(30, 30, 20, seed=28)  # 18,000 nodes on the coarsest (only) level
    B = gr.graph_reduce_create(big.n, big.u, big.v, big.w)
    with pytest.raises(gr.GraphReduceError):
        gr.graph_reduce_eigensolve([B], 4)
