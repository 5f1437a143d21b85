"""kNN workloads: the 200k-point graph reduced to ~n/32 (FP64 maps bit-exact
against the oracle's own reduction; FP64 and FP32 paths' 10 eigenvalues within
1e-3 of the oracle's reduced graph), and the spectral-mismatch loss on
the 1M-point graph reduced to ~n/32 (GPU FP32 gradient against the FP64
oracle gradient at full size; central finite differences in FP64 on a
2,000-node ball of the graph)."""
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


@pytest.fixture(scope="module")
def knn1m():
    return W.knn_gmm(1_000_000, 16, 20, 15, 12350, device=DEV)


def test_knn200k_multilevel(gr, oracle_mod):
    g = W.knn_gmm(200_000, 10, 10, 10, 12347, device=DEV)
    K, S, final = 16, 5, 6250
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, K, S, final_target=final)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    g64, _ = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=K, sweeps=S, prec=gr.GR_F64, final_target=final))
    assert len(g64) == len(levels)
    for lv, gl in zip(levels, g64):
        assert np.array_equal(gr.graph_reduce_get_map(gl).cpu().numpy(), lv.agg)
    last = levels[-1]
    ev_ref = oracle_mod.smallest_nontrivial_eigs(last.nc, last.uc, last.vc, last.wc, 10)
    u, v, w = (t.numpy() for t in gr.graph_reduce_get_edges(g64[-1], on_host=True))
    ev = oracle_mod.smallest_nontrivial_eigs(g64[-1].n, u, v, w, 10)
    assert np.max(np.abs(ev - ev_ref) / ev_ref) <= 1e-3
    g32, _ = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=K, sweeps=S, prec=gr.GR_F32, final_target=final))
    u, v, w = (t.numpy() for t in gr.graph_reduce_get_edges(g32[-1], on_host=True))
    ev32 = oracle_mod.smallest_nontrivial_eigs(g32[-1].n, u, v, w, 10)
    err32 = np.max(np.abs(ev32 - ev_ref) / ev_ref)
    assert err32 <= 1e-3, "knn200k FP32 path: 10-eigenvalue max rel err vs oracle %.3e" % err32


def _ball(g, n_ball, root=0):
    """Induced subgraph on the BFS ball of n_ball nodes around root."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import breadth_first_order
    A = coo_matrix((np.ones(g.m), (g.u, g.v)), shape=(g.n, g.n)).tocsr()
    order = breadth_first_order(A + A.T, root, directed=False, return_predecessors=False)[:n_ball]
    keep = np.zeros(g.n, bool)
    keep[order] = True
    newid = -np.ones(g.n, np.int64)
    newid[np.sort(order)] = np.arange(len(order))
    sel = keep[g.u] & keep[g.v]
    u, v, w = W.canonicalize(len(order), newid[g.u[sel]], newid[g.v[sel]], g.w[sel])
    return W.Graph(len(order), u, v, w, "ball")


def _loss_case(gr, oracle_mod, g, K=16, S=5):
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    final = max(g.n // 32, 8)
    lev, _ = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=K, sweeps=S, prec=gr.GR_F32, final_target=final))
    agg = gr.graph_reduce_compose_maps(lev)
    C = lev[-1]
    X = torch.empty(g.n, K, dtype=torch.float32, device=DEV)
    gr.graph_reduce_smooth(G, X, S, 0.7, 5, 0)
    cu, cv, cw = (t.numpy() for t in gr.graph_reduce_get_edges(C, on_host=True))
    wc = (cw * np.random.default_rng(3).uniform(0.7, 1.4, size=len(cw))).astype(np.float32)
    return G, C, agg, X, cu, cv, wc


@pytest.mark.parametrize("S", [0, 5])
def test_knn1m_loss_gradient_fullsize(gr, oracle_mod, knn1m, S):
    g = knn1m
    G, C, agg, X, cu, cv, wc = _loss_case(gr, oracle_mod, g, S=5)
    w = torch.from_numpy(wc).to(DEV)
    loss, saved = gr.graph_reduce_loss_fwd(G, C, agg, X, w, S)
    gw = gr.graph_reduce_loss_bwd(C, saved, 16, w, S, 0.7, torch.ones(1, device=DEV)).cpu().numpy()
    L, gref, _, _ = oracle_mod.loss(g.n, g.u, g.v, g.w, C.n, cu, cv, wc.astype(np.float64), agg.cpu().numpy(),
                                    X.double().cpu().numpy(), S)
    assert abs(loss.item() - L) <= 1e-4 * abs(L) + 1e-7
    assert np.linalg.norm(gw - gref) / np.linalg.norm(gref) <= 1e-4


def test_knn1m_ball_finite_differences(gr, oracle_mod, knn1m):
    b = _ball(knn1m, 2000)
    S = 5
    G, C, agg, X, cu, cv, wc = _loss_case(gr, oracle_mod, b, S=S)
    aggh = agg.cpu().numpy()
    Xh = X.double().cpu().numpy()
    w64 = wc.astype(np.float64)
    L0, gref, _, _ = oracle_mod.loss(b.n, b.u, b.v, b.w, C.n, cu, cv, w64, aggh, Xh, S)
    h = 1e-4
    fd = np.empty(len(w64))
    for e in range(len(w64)):
        wp = w64.copy()
        wp[e] += h
        wm = w64.copy()
        wm[e] -= h
        fd[e] = (oracle_mod.loss(b.n, b.u, b.v, b.w, C.n, cu, cv, wp, aggh, Xh, S, want_grad=False)[0]
                 - oracle_mod.loss(b.n, b.u, b.v, b.w, C.n, cu, cv, wm, aggh, Xh, S, want_grad=False)[0]) / (2 * h)
    floor = 1e-10 * np.abs(gref).max()
    rel = np.abs(gref - fd) / np.maximum(np.abs(fd), floor)
    assert np.all((rel <= 1e-5) | (np.abs(gref - fd) <= floor)), rel.max()
    # the GPU adjoint against the FP64 gradient
    w = torch.from_numpy(wc).to(DEV)
    loss, saved = gr.graph_reduce_loss_fwd(G, C, agg, X, w, S)
    gw = gr.graph_reduce_loss_bwd(C, saved, 16, w, S, 0.7, torch.ones(1, device=DEV)).cpu().numpy()
    assert np.linalg.norm(gw - gref) / np.linalg.norm(gref) <= 1e-4
