"""Parity at the sizes and in the launch configuration bench.py times.

The oracle cannot redo every step at full size in seconds, so each step is
checked with what it can compute exactly:
  smoothing  the GPU's S-sweep block against one oracle sweep (+ centring and
             normalising) applied to the GPU's (S-1)-sweep block -- the same
             recurrence, at any size; plus the invariants of every column
  affinity   oracle distances on a random sample of edges, from the GPU block
  aggregate  the complete map, from the GPU's own FP32 distances (bit-exact)
  coarsen    the complete reduced graph from the GPU's map (pattern and
             weights bit-exact)
and the level loop in FP64 is compared map by map with the oracle's own
reduction of the 64^3 mesh, with the 10 eigenvalues of the final graphs (FP64
and FP32 paths within 1e-3 of the oracle's reduced graph).
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


def _col_relerr(A, B):
    return np.linalg.norm(A - B, axis=0) / np.linalg.norm(B, axis=0)


def _level_checks(gr, oracle_mod, g, K, S, omega=0.7, target_div=4, sample=200_000):
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    # smoothing: last sweep through the oracle's recurrence
    Xp = torch.empty(g.n, K, dtype=torch.float32, device=DEV)
    gr.graph_reduce_smooth(G, Xp, S - 1, omega, 0, 0)
    X = torch.empty(g.n, K, dtype=torch.float32, device=DEV)
    gr.graph_reduce_smooth(G, X, S, omega, 0, 0)
    Xh = X.double().cpu().numpy()
    ref = oracle_mod.center_normalize(oracle_mod.jacobi_sweep(g.n, g.u, g.v, g.w, Xp.double().cpu().numpy(), omega))
    err = _col_relerr(Xh, ref)
    assert err.max() <= 1e-5, err.max()
    assert np.all(np.abs(Xh.sum(0)) <= 1e-4) and np.allclose((Xh * Xh).sum(0), 1.0, atol=1e-5)
    # affinity on a sample of edges
    d = torch.empty(g.m, dtype=torch.float32, device=DEV)
    gr.graph_reduce_affinity(G, X, d)
    dh = d.cpu().numpy()
    idx = np.random.default_rng(1).choice(g.m, min(sample, g.m), replace=False)
    dref = oracle_mod.affinity(g.n, g.u[idx], g.v[idx], Xh)
    assert np.max(np.abs(dh[idx].astype(np.float64) - dref)) <= 1e-5
    # aggregation: the complete map from the GPU's own distances
    target = -(-g.n // target_div)
    agg, nc, proposals = gr.graph_reduce_aggregate(G, d, target, 2)
    ragg, rnc = oracle_mod.aggregate(g.n, g.u, g.v, dh.astype(np.float64), target, 2)
    assert nc == rnc and np.array_equal(agg.cpu().numpy(), ragg)
    # Galerkin: the complete reduced graph
    C = gr.graph_reduce_coarsen(G, agg, nc)
    uc, vc, wc = oracle_mod.coarsen(g.n, g.u, g.v, g.w, ragg, rnc)
    cu, cv, cw = (t.numpy() for t in gr.graph_reduce_get_edges(C, on_host=True))
    assert np.array_equal(cu, uc) and np.array_equal(cv, vc)
    assert np.max(np.abs(cw - wc) / wc) <= 1e-6
    return nc, proposals


def test_mesh128_fullsize_level(gr, oracle_mod):
    g = W.mesh3d(128, 128, 128)
    nc, proposals = _level_checks(gr, oracle_mod, g, K=24, S=8)
    assert 0.25 * g.n <= nc < 0.5 * g.n


def test_chunglu434k_fullsize_level(gr, oracle_mod):
    g = W.chung_lu()
    nc, proposals = _level_checks(gr, oracle_mod, g, K=16, S=5)
    assert nc < 0.5 * g.n


def test_mesh64_levels_f64_against_oracle_reduction(gr, oracle_mod):
    g = W.mesh3d(64, 64, 64)
    K, S, final = 24, 8, 4096
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, K, S, final_target=final)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    glev, stats = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=K, sweeps=S, prec=gr.GR_F64, final_target=final))
    assert len(glev) == len(levels)
    for lv, gl in zip(levels, glev):
        assert np.array_equal(gr.graph_reduce_get_map(gl).cpu().numpy(), lv.agg)
    u, v, w = (t.numpy() for t in gr.graph_reduce_get_edges(glev[-1], on_host=True))
    ev = oracle_mod.smallest_nontrivial_eigs(glev[-1].n, u, v, w, 10)
    last = levels[-1]
    ev_ref = oracle_mod.smallest_nontrivial_eigs(last.nc, last.uc, last.vc, last.wc, 10)
    assert np.max(np.abs(ev - ev_ref) / ev_ref) <= 1e-3
    # the FP32 path on the same graph: its final reduced graph's 10 smallest
    # nontrivial eigenvalues within 1e-3 of the oracle's reduced graph
    g32, _ = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=K, sweeps=S, prec=gr.GR_F32, final_target=final))
    u, v, w = (t.numpy() for t in gr.graph_reduce_get_edges(g32[-1], on_host=True))
    ev32 = oracle_mod.smallest_nontrivial_eigs(g32[-1].n, u, v, w, 10)
    err32 = np.max(np.abs(ev32 - ev_ref) / ev_ref)
    assert err32 <= 1e-3, "mesh64 FP32 path: 10-eigenvalue max rel err vs oracle %.3e" % err32


def test_chunglu_levels_against_oracle_reduction(gr, oracle_mod):
    # The Chung-Lu recipe (degree exponent 2.5, mean degree 73.5) at 1/4 of
    # the 434,000-node size: the coarse graphs stay dense, so the Galerkin
    # product of every level takes the global-sort path.  FP64 maps bit-exact
    # on every level against the oracle's own level loop; the 10 smallest
    # nontrivial eigenvalues of the final graphs within 1e-3 of the oracle's
    # for the FP64 and FP32 paths; BF16 storage reported.
    g = W.chung_lu(108_500, 4_000_000, max_deg=600.0)
    K, S, final = 16, 5, 3250
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, K, S, final_target=final)
    last = levels[-1]
    ev_ref = oracle_mod.smallest_nontrivial_eigs(last.nc, last.uc, last.vc, last.wc, 10)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    g64, _ = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=K, sweeps=S, prec=gr.GR_F64, final_target=final))
    assert len(g64) == len(levels) >= 2
    for lv, gl in zip(levels, g64):
        assert np.array_equal(gr.graph_reduce_get_map(gl).cpu().numpy(), lv.agg)
    u, v, w = (t.numpy() for t in gr.graph_reduce_get_edges(g64[-1], on_host=True))
    assert np.array_equal(u, last.uc) and np.array_equal(v, last.vc)
    assert np.max(np.abs(w - last.wc) / last.wc) <= 1e-6
    ev64 = oracle_mod.smallest_nontrivial_eigs(g64[-1].n, u, v, w, 10)
    assert np.max(np.abs(ev64 - ev_ref) / ev_ref) <= 1e-3
    g32, _ = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=K, sweeps=S, prec=gr.GR_F32, final_target=final))
    u, v, w = (t.numpy() for t in gr.graph_reduce_get_edges(g32[-1], on_host=True))
    ev32 = oracle_mod.smallest_nontrivial_eigs(g32[-1].n, u, v, w, 10)
    err32 = np.max(np.abs(ev32 - ev_ref) / ev_ref)
    assert err32 <= 1e-3, "chunglu FP32 path: 10-eigenvalue max rel err vs oracle %.3e" % err32
    gb, _ = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=K, sweeps=S, prec=gr.GR_BF16, final_target=final))
    u, v, w = (t.numpy() for t in gr.graph_reduce_get_edges(gb[-1], on_host=True))
    evb = oracle_mod.smallest_nontrivial_eigs(gb[-1].n, u, v, w, 10)
    print("chunglu BF16 storage: 10-eigenvalue max rel err vs oracle %.3e" % np.max(np.abs(evb - ev_ref) / ev_ref))
