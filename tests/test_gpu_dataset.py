"""Reduced data set F_R = P^T F (Alg. 6, step 4) on the GPU against the oracle.

The hierarchy is the oracle's; the GPU contexts are rebuilt from its maps
with graph_reduce_coarsen.  Both sides add each aggregate's rows in ascending
fine id in FP64, so sums and means agree bit for bit (FP32 data: after the
one rounding of the FP64 result).
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


def _gpu_levels(gr, g, levels):
    ctxs = [gr.graph_reduce_create(g.n, g.u, g.v, g.w)]
    for lv in levels:
        ctxs.append(gr.graph_reduce_coarsen(ctxs[-1], torch.from_numpy(lv.agg).to(DEV), lv.nc))
    return ctxs[1:]


@pytest.mark.parametrize("d", [1, 3, 16, 33])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mean", [False, True])
def test_reduce_data_parity(gr, oracle_mod, d, dtype, mean):
    g = W.knn_gmm(5000, 6, 3, 8, 41)
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, 8, 5, final_target=200)
    comp = oracle_mod.compose_maps(levels)
    nc = levels[-1].nc
    F = np.random.default_rng(d).normal(size=(g.n, d))
    if dtype == torch.float32:
        F = F.astype(np.float32)
    ref = oracle_mod.reduce_features(comp, nc, F.astype(np.float64), mean)
    ctxs = _gpu_levels(gr, g, levels)
    out = gr.graph_reduce_reduce_data(ctxs, torch.from_numpy(F).to(DEV), mean)
    assert out.shape == (nc, d) and out.dtype == dtype
    assert np.array_equal(out.cpu().numpy(), ref.astype(F.dtype))


def test_reduce_data_one_level_and_errors(gr, oracle_mod):
    g = W.mesh3d(9, 8, 7, seed=42)
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, 8, 5, final_target=100, max_levels=1)
    assert len(levels) == 1
    ctxs = _gpu_levels(gr, g, levels)
    F = torch.arange(g.n * 2, dtype=torch.float64, device=DEV).reshape(g.n, 2)
    out = gr.graph_reduce_reduce_data(ctxs, F)
    ref = oracle_mod.reduce_features(levels[0].agg, levels[0].nc, F.cpu().numpy())
    assert np.array_equal(out.cpu().numpy(), ref)
    assert torch.equal(out.sum(0), F.sum(0))  # integer-valued: exact
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    with pytest.raises(gr.GraphReduceError) as ei:  # the fine context has no parent map
        gr.graph_reduce_reduce_data([G], F)
    assert ei.value.status == 5
