"""GPU parity of the sweep kernels (Alg. 3 weighted-Jacobi sweeps, Sec.
3.2.1) against the FP64 oracle: each kernel is forced on each graph family
through graph_reduce_set_sweep_kernel, and the automatic choice is checked
(band kernel on a banded grid large enough to fill the GPU, not on smaller
graphs nor where random long edges scatter the neighbours).
The band kernel fits shared memory on every family and size here, so forcing
it runs it; its neighbours come from the window ring, the far runs and global
memory (random long edges, the hub's row past a stage's slot capacity).

Bars as for graph_reduce_smooth: per-column |dX|/|X| <= 1e-12 in FP64 and
<= 1e-5 in FP32.  The families mix short and long rows, a hub row, random
long edges, isolated rows and dense graphs, so each kernel meets rows of
every length.
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
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    return np.linalg.norm(A - B, axis=0) / np.maximum(np.linalg.norm(B, axis=0), 1e-300)


def _grid_plus(a, b, extra, hub_deg, seed):
    """a x b grid plus `extra` random long edges and one hub joined to
    hub_deg nodes: mostly local, with rows whose neighbours leave any window
    and one row whose slots overflow a band."""
    g = W.grid2d(a, b)
    rng = np.random.default_rng(seed)
    n = g.n
    u = [g.u.astype(np.int64)]
    v = [g.v.astype(np.int64)]
    p = rng.integers(0, n, extra)
    q = rng.integers(0, n, extra)
    u.append(p)
    v.append(q)
    hub = n // 2
    nb = rng.choice(n, hub_deg, replace=False)
    u.append(np.full(hub_deg, hub))
    v.append(nb)
    uu = np.concatenate(u)
    vv = np.concatenate(v)
    w = rng.lognormal(0.0, 0.5, len(uu))
    cu, cv, cw = W.canonicalize(n, uu, vv, w)
    return W.Graph(n, cu, cv, cw)


FAMILIES = {
    "grid64": lambda: W.grid2d(64, 64),
    "grid160x120": lambda: W.grid2d(160, 120),
    "mesh_ln": lambda: W.mesh3d(19, 17, 13, seed=4),
    "path_iso": lambda: W.Graph(3000, np.arange(0, 2500, dtype=np.int32), np.arange(1, 2501, dtype=np.int32),
                                np.linspace(0.5, 2.0, 2500)),  # nodes 2501..2999 isolated
    "grid_long_hub": lambda: _grid_plus(96, 80, 3000, 2500, seed=11),
    "rand_w": lambda: W.random_sparse(1537, 6000, seed=3),
    "star": lambda: W.star(300),
    "complete": lambda: W.complete(40, 0.5),
}

KINDS = ["ROW", "STREAM", "BAND", "AUTO"]
# the automatic choice leaves the band kernel to graphs large enough to give
# every SM a chunk of bands (test_auto_band_on_a_large_grid); these families
# are all smaller
AUTO_NOT_BAND = tuple(FAMILIES)


def _kind(gr, name):
    return getattr(gr, "GR_SWEEP_" + name)


def _smooth(gr, G, n, K, dtype, S, omega, seed, level):
    X = torch.empty(n, K, dtype=dtype, device=DEV)
    gr.graph_reduce_smooth(G, X, S, omega, seed, level)
    return X


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("name", list(FAMILIES))
def test_sweep_kernels_f64_f32(gr, oracle_mod, kind, name):
    g = FAMILIES[name]()
    S, omega, seed, level = 5, 0.7, 5, 1
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    gr.graph_reduce_set_sweep_kernel(G, _kind(gr, kind))
    for K in (4, 8, 16, 24, 32):
        ref = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, S, omega, seed, level)
        for dtype, bar in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
            plan = gr.graph_reduce_sweep_plan(G, K, dtype)
            if kind != "AUTO":
                assert plan == _kind(gr, kind)
            elif name in AUTO_NOT_BAND:
                assert plan != gr.GR_SWEEP_BAND, (K, plan)
            X = _smooth(gr, G, g.n, K, dtype, S, omega, seed, level)
            err = _col_relerr(X.double().cpu().numpy(), ref).max()
            assert err <= bar, (name, kind, K, dtype, err, plan)


@pytest.mark.parametrize("kind", ["ROW", "STREAM", "BAND"])
@pytest.mark.parametrize("K", [16, 24])
def test_sweep_kernels_large_grid(gr, oracle_mod, kind, K):
    # 64 x 12288 grid: grids of many blocks, every block several row groups
    g = W.grid2d(64, 12288)
    S, omega, seed, level = 6, 0.7, 2, 0
    ref = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, S, omega, seed, level)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    gr.graph_reduce_set_sweep_kernel(G, _kind(gr, kind))
    for dtype, bar in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        assert gr.graph_reduce_sweep_plan(G, K, dtype) == _kind(gr, kind)
        X = _smooth(gr, G, g.n, K, dtype, S, omega, seed, level)
        err = _col_relerr(X.double().cpu().numpy(), ref).max()
        assert err <= bar, (kind, K, dtype, err)


@pytest.mark.parametrize("K", [16, 24])
def test_row_kernel_on_a_large_l2_resident_block(gr, oracle_mod, K):
    # 420,000 nodes of mean degree 12.5: the row-group kernel with four slots
    # in flight, in FP32 with its registers fitted to four blocks per SM (a
    # block of this size stays in L2), in BF16 as the compiler fits them
    g = W.random_sparse(420_000, 2_205_000, seed=9)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    S, omega, seed, level = 3, 0.7, 4, 1
    ref = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, S, omega, seed, level)
    assert gr.graph_reduce_sweep_plan(G, K, torch.float32) == gr.GR_SWEEP_ROW
    for dtype, bar in ((torch.float32, 1e-5), (torch.bfloat16, None)):
        X = _smooth(gr, G, g.n, K, dtype, S, omega, seed, level)
        if bar is not None:
            err = _col_relerr(X.double().cpu().numpy(), ref).max()
            assert err <= bar, (K, err)
        else:
            assert torch.isfinite(X.float()).all()


@pytest.mark.parametrize("K", [16, 24])
def test_auto_band_on_a_large_grid(gr, oracle_mod, K):
    # 200 x 1100 grid (220,000 nodes, rows 200 apart): large enough for a
    # chunk of bands per SM and banded, so the automatic choice takes the band
    # kernel; a grid with random long edges of the same size does not
    g = W.grid2d(200, 1100, weights=lambda m: np.random.default_rng(7).lognormal(0.0, 0.5, m))
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    S, omega, seed, level = 5, 0.7, 3, 0
    ref = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, S, omega, seed, level)
    for dtype, bar in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        plan = gr.graph_reduce_sweep_plan(G, K, dtype)
        if dtype == torch.float32:
            assert plan == gr.GR_SWEEP_BAND, plan
        X = _smooth(gr, G, g.n, K, dtype, S, omega, seed, level)
        err = _col_relerr(X.double().cpu().numpy(), ref).max()
        assert err <= bar, (K, dtype, err, plan)
    h = _grid_plus(200, 1100, 60000, 100, seed=5)
    H = gr.graph_reduce_create(h.n, h.u, h.v, h.w)
    assert gr.graph_reduce_sweep_plan(H, K, torch.float32) != gr.GR_SWEEP_BAND


def test_sweep_kernels_bf16_agree(gr):
    # BF16 storage: both kernels store the same products in slot order, so
    # they agree to within a few BF16 roundings
    g = FAMILIES["grid_long_hub"]()
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    out = {}
    for kd in ("ROW", "STREAM", "BAND"):
        gr.graph_reduce_set_sweep_kernel(G, _kind(gr, kd))
        assert gr.graph_reduce_sweep_plan(G, 16, torch.bfloat16) == _kind(gr, kd)
        out[kd] = _smooth(gr, G, g.n, 16, torch.bfloat16, 5, 0.7, 1, 0).float().cpu().numpy()
    for kd in ("STREAM", "BAND"):
        err = _col_relerr(out[kd], out["ROW"]).max()
        assert err <= 2e-2, (kd, err)


def test_set_sweep_kernel_rejects_unknown(gr):
    g = W.grid2d(30, 30)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    with pytest.raises(gr.GraphReduceError) as e:
        gr.graph_reduce_set_sweep_kernel(G, 17)
    assert e.value.status == gr.GR_EINVAL
