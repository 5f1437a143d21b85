"""Edge-weight scaling of the reduced graph (Alg. 1 driven by the loss
gradient) on the GPU against the oracle.

The hierarchy, test vectors and initial weights come from the oracle; the
initial weights are rounded to FP32 on both sides, since the GPU scales FP32
weights.  The GPU evaluates the loss and its gradient in FP32 (the oracle in
FP64), so losses agree to about 1e-5 relative and the gradient to about 1e-4
in norm.  The per-edge update is min(dw, max(cap, 0)), a continuous function
of the step and the degrees, so a cap decision taken on either side of the
bound moves a weight by no more than that rounding: weights are compared per
edge, against the size of the change the scaling made.
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


def _setup(oracle_mod, n, deg, K, seed=31):
    g = W.random_sparse(n, deg * n, seed=seed)
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, 8, 5, final_target=max(n // 32, 8))
    agg = oracle_mod.compose_maps(levels)
    last = levels[-1]
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, 5, seed=1)
    w0 = last.wc.astype(np.float32).astype(np.float64)
    return g, last, agg, X, w0


def _run_gpu(gr, g, last, agg, X, w0, **kw):
    F = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    C = gr.graph_reduce_create(last.nc, last.uc, last.vc, last.wc)
    w = torch.from_numpy(w0).float().to(DEV)
    w, h = gr.graph_reduce_scale_edges(F, C, torch.from_numpy(agg).to(DEV), torch.from_numpy(X).float().to(DEV), w,
                                       **kw)
    return w.cpu().numpy().astype(np.float64), h


CASES = [
    ("rand2000_k16_eta1e4", 2000, 6, 16, dict(eta_max=1e4, kmax=6, eps=0.0)),
    ("rand6000_k8_eta1e3", 6000, 5, 8, dict(eta_max=1e3, kmax=6, eps=0.0)),
    ("rand2000_k16_momentum0", 2000, 6, 16, dict(eta_max=3e4, alpha=0.0, kmax=4, eps=0.0, delta_bar=0.8)),
    ("rand6000_k8_sweeps1", 6000, 5, 8, dict(eta_max=3e3, kmax=4, eps=0.0, sweeps_c=1)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_scale_edges_parity(gr, oracle_mod, case):
    _, n, deg, K, kw = case
    g, last, agg, X, w0 = _setup(oracle_mod, n, deg, K)
    okw = dict(kw)
    if "sweeps_c" in okw:
        okw["sweeps"] = okw.pop("sweeps_c")
    wr, hr = oracle_mod.scale_edges(g.n, g.u, g.v, g.w, last.nc, last.uc, last.vc, w0, agg, X, **okw)
    w, h = _run_gpu(gr, g, last, agg, X, w0, **kw)
    assert len(h) == len(hr) == kw["kmax"]
    L, lam = np.array([x[0] for x in h]), np.array([x[1] for x in h])
    Lr, lamr = np.array([x[0] for x in hr]), np.array([x[1] for x in hr])
    assert np.allclose(L, Lr, rtol=1e-4, atol=0), (L, Lr)
    assert np.allclose(lam, lamr, rtol=1e-4, atol=0), (lam, lamr)
    change = np.abs(wr - w0).max()
    assert change > 1e-2 * np.abs(w0).max()  # the scaling did something
    assert np.all(w >= w0)
    err = np.abs(w - wr).max()
    assert err <= 2e-3 * change + 2e-6 * np.abs(wr).max(), (err, change)


def test_scale_edges_stops_and_zero_step(gr, oracle_mod):
    g, last, agg, X, w0 = _setup(oracle_mod, 2000, 6, 16)
    # huge eps: the second loss never decreases enough, one update is made
    w, h = _run_gpu(gr, g, last, agg, X, w0, eta_max=1e4, kmax=6, eps=1e9)
    wr, hr = oracle_mod.scale_edges(g.n, g.u, g.v, g.w, last.nc, last.uc, last.vc, w0, agg, X, eta_max=1e4, kmax=6,
                                    eps=1e9)
    assert len(h) == len(hr) == 1
    assert np.abs(w - wr).max() <= 2e-3 * np.abs(wr - w0).max() + 2e-6 * np.abs(wr).max()
    # eta_max = 0: the weights never move (bit for bit), lambda_1 stays 1
    w, h = _run_gpu(gr, g, last, agg, X, w0, eta_max=0.0, kmax=3, eps=0.0)
    assert np.array_equal(w, w0) and len(h) == 3 and all(x[1] == 1.0 for x in h)


def test_scale_edges_cap_binds_on_a_matching(gr, oracle_mod):
    # 30 disjoint weighted 4-paths, aggregates {0,1} and {2,3}: the reduced
    # graph is a matching, and a huge step is capped at d_G/d_P = bound at
    # every node (bound = delta_bar^(k/kmax) after iteration k)
    rng = np.random.default_rng(72)
    P = 30
    u = np.concatenate([4 * np.arange(P) + t for t in range(3)]).astype(np.int32)
    v = u + 1
    o = np.lexsort((v, u))
    u, v = u[o], v[o]
    w = rng.uniform(0.5, 2.0, len(u))
    n = 4 * P
    agg = (np.arange(n) // 2).astype(np.int32)
    uc, vc, wc = oracle_mod.coarsen(n, u, v, w, agg, 2 * P)
    X = oracle_mod.smooth(n, u, v, w, 4, 2)
    F = gr.graph_reduce_create(n, u, v, w)
    C = gr.graph_reduce_create(2 * P, uc, vc, wc)
    w0 = wc.astype(np.float32).astype(np.float64)
    kmax, delta_bar = 4, 0.3
    wt = torch.from_numpy(w0).float().to(DEV)
    wt, h = gr.graph_reduce_scale_edges(F, C, torch.from_numpy(agg).to(DEV), torch.from_numpy(X).float().to(DEV), wt,
                                        eta_max=1e9, delta_bar=delta_bar, kmax=kmax, eps=0.0)
    step = delta_bar ** (1.0 / kmax)
    assert len(h) == kmax
    assert np.allclose([x[1] for x in h], [step ** (k + 1) for k in range(kmax)], rtol=2e-6, atol=0)
    wn = wt.cpu().numpy().astype(np.float64)
    assert np.allclose(w0 / wn, step ** kmax, rtol=2e-6, atol=0)


def test_scale_edges_rejects_bad_arguments(gr, oracle_mod):
    g, last, agg, X, w0 = _setup(oracle_mod, 2000, 6, 16)
    for kw in (dict(kmax=0), dict(delta_bar=0.0), dict(delta_bar=1.5), dict(alpha=1.0), dict(eta_max=-1.0),
               dict(omega=0.0)):
        with pytest.raises(gr.GraphReduceError) as ei:
            _run_gpu(gr, g, last, agg, X, w0, **kw)
        assert ei.value.status == 1
