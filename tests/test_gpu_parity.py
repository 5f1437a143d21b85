"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded
inputs.  Bars (the accuracy required of the reduction):
  smoothed X         per-column |dX|/|X| <= 1e-12 (FP64), <= 1e-5 (FP32)
  BF16-stored X      per-column <= 2 (S + 1) 2^-9 against the oracle started
                     from the same BF16-rounded block (S sweeps; derivation at
                     the test); against the unrounded start, reported
  distance d         FP64 bit-exact given the same X; FP32 |dd| <= 1e-5
  aggregates         bit-exact given the oracle's (or any shared) distances
  reduced graph      pattern bit-exact, weights <= 1e-6 relative
  10 eigenvalues     <= 1e-3 relative to the oracle's reduced graph
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


GRAPHS = {
    "grid13x9": lambda: W.grid2d(13, 9),
    "rand_w": lambda: W.random_sparse(1537, 6000, seed=3),
    "star": lambda: W.star(200),
    "complete": lambda: W.complete(40, 0.5),
    "path_iso": lambda: W.Graph(300, np.arange(0, 250, dtype=np.int32), np.arange(1, 251, dtype=np.int32),
                                np.linspace(0.5, 2.0, 250)),  # nodes 251..299 isolated
    "mesh_ln": lambda: W.mesh3d(11, 7, 5, seed=4),
    # long rows (mean degree >= 24): the streaming sweep kernel
    "chunglu_s": lambda: W.chung_lu(3001, 60000, mean_deg=40.0, max_deg=600.0, seed=5),
    "dense_rand": lambda: W.random_sparse(777, 15000, seed=6),
}


# ---------------------------------------------------------------------------
# create / edges round trip / input validation
# ---------------------------------------------------------------------------
def test_create_roundtrip_and_validation(gr, oracle_mod):
    g = W.random_sparse(777, 3000, seed=1)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    u, v, w = gr.graph_reduce_get_edges(G, on_host=True)
    assert np.array_equal(u.numpy(), g.u) and np.array_equal(v.numpy(), g.v) and np.array_equal(w.numpy(), g.w)
    # device inputs
    G2 = gr.graph_reduce_create(g.n, torch.from_numpy(g.u).to(DEV), torch.from_numpy(g.v).to(DEV),
                                torch.from_numpy(g.w).to(DEV))
    u2, _, _ = gr.graph_reduce_get_edges(G2)
    assert torch.equal(u2.cpu(), torch.from_numpy(g.u))
    # caller-provided outputs, larger than needed: pinned host and device
    for on_host in (True, False):
        kw = {"device": DEV} if not on_host else {}
        out = (torch.full((g.m + 5,), -1, dtype=torch.int32, **kw), torch.full((g.m + 5,), -1, dtype=torch.int32, **kw),
               torch.zeros(g.m + 5, dtype=torch.float64, **kw))
        if on_host:
            out = tuple(t.pin_memory() for t in out)
        u3, v3, w3 = gr.graph_reduce_get_edges(G2, on_host=on_host, out=out)
        torch.cuda.synchronize()
        assert u3.numel() == g.m and np.array_equal(u3.cpu().numpy(), g.u) and np.array_equal(v3.cpu().numpy(), g.v)
        assert np.array_equal(w3.cpu().numpy(), g.w) and int(out[0][g.m].item()) == -1
    bad = [
        (g.v, g.u, g.w),                                   # u > v
        (g.u[::-1].copy(), g.v[::-1].copy(), g.w),         # unsorted
        (g.u, g.v, -g.w),                                  # negative weight
        (np.concatenate([g.u, g.u[-1:]]), np.concatenate([g.v, g.v[-1:]]), np.concatenate([g.w, g.w[-1:]])),
    ]
    for bu, bv, bw in bad:
        for dev_inputs in (False, True):
            args = [np.ascontiguousarray(x) for x in (bu, bv, bw)]
            if dev_inputs:
                args = [torch.from_numpy(a).to(DEV) for a in args]
            with pytest.raises(gr.GraphReduceError) as ei:
                gr.graph_reduce_create(g.n, *args)
            assert ei.value.status == 1


def _star_last(n, seed):
    """Star whose centre is the last node: its lower part holds n - 1 edges."""
    rng = np.random.default_rng(seed)
    return W.Graph(n, np.arange(0, n - 1, dtype=np.int32), np.full(n - 1, n - 1, np.int32),
                   rng.uniform(0.5, 2.0, n - 1))


# The CSR build of a sparse graph sorts each row's lower part by the row's own
# thread (up to 32 entries) or by a warp (up to 2,048); past that, and for
# graphs of mean degree 32 or more, a global radix sort lists the lower parts.
@pytest.mark.parametrize("case", [("thread_to_warp", lambda: _star_last(40, 1)),
                                  ("warp", lambda: _star_last(1500, 2)),
                                  ("global_sort", lambda: _star_last(3000, 3)),
                                  ("dense_global_sort", lambda: W.random_sparse(700, 16000, seed=8))],
                         ids=lambda c: c[0])
def test_csr_lower_part_paths(gr, oracle_mod, case):
    g = case[1]()
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    gu, gv, gw = (t.numpy() for t in gr.graph_reduce_get_edges(G, on_host=True))
    assert np.array_equal(gu, g.u) and np.array_equal(gv, g.v) and np.array_equal(gw, g.w)
    K, S = 8, 3
    ref = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, S, 0.7, 2, 0)
    X = torch.empty(g.n, K, dtype=torch.float64, device=DEV)
    gr.graph_reduce_smooth(G, X, S, 0.7, 2, 0)
    assert _col_relerr(X.cpu().numpy(), ref).max() <= 1e-12
    # and the FP64 distances of every edge from that block, bit-exact
    d = torch.empty(g.m, dtype=torch.float64, device=DEV)
    gr.graph_reduce_affinity(G, X, d)
    dref = oracle_mod.affinity(g.n, g.u, g.v, X.cpu().numpy())
    assert np.array_equal(d.cpu().numpy(), dref)


# ---------------------------------------------------------------------------
# smoothing
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("K", [4, 8, 16, 24, 32])
def test_smooth_parity_f64_f32(gr, oracle_mod, name, K):
    g = GRAPHS[name]()
    S, omega, seed, level = 5, 0.7, 7, 2
    ref = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, S, omega, seed, level)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    X64 = torch.empty(g.n, K, dtype=torch.float64, device=DEV)
    gr.graph_reduce_smooth(G, X64, S, omega, seed, level)
    e64 = _col_relerr(X64.cpu().numpy(), ref)
    assert e64.max() <= 1e-12, e64.max()
    X32 = torch.empty(g.n, K, dtype=torch.float32, device=DEV)
    gr.graph_reduce_smooth(G, X32, S, omega, seed, level)
    e32 = _col_relerr(X32.cpu().numpy(), ref)
    assert e32.max() <= 1e-5, e32.max()
    # deterministic: a second run is bitwise identical
    X32b = torch.empty_like(X32)
    gr.graph_reduce_smooth(G, X32b, S, omega, seed, level)
    assert torch.equal(X32, X32b)


@pytest.mark.parametrize("K", [8, 16, 24])
def test_smooth_bf16_reported(gr, oracle_mod, K):
    g = W.grid2d(64, 64)
    ref = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, 5)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    X = torch.empty(g.n, K, dtype=torch.bfloat16, device=DEV)
    gr.graph_reduce_smooth(G, X, 5)
    e = _col_relerr(X.float().cpu().numpy(), ref)
    print("bf16 storage K=%d: max per-column relative error %.3e" % (K, e.max()))
    assert e.max() < 3e-2


def _bf16_round(x):
    """FP64 -> FP32 -> BF16, each rounded to nearest even (the storage rule of
    the test vectors in BF16), returned as FP64."""
    return torch.from_numpy(np.asarray(x, np.float64).astype(np.float32)).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("name", ["grid13x9", "rand_w", "mesh_ln", "path_iso"])
@pytest.mark.parametrize("K", [8, 16, 24, 32])
def test_smooth_bf16_against_oracle_from_bf16_start(gr, oracle_mod, name, K):
    # BF16 storage rounds every stored entry to 8 significant bits, a relative
    # error of at most 2^-9.  Started from the same BF16-rounded block X0, the
    # oracle's FP64 sweeps (Alg. 3, centring and normalising after each)
    # differ from the GPU's only by the roundings of the S stored sweep
    # outputs and of the final centred, scaled block: each moves a column by at
    # most 2^-9 of its norm, and a weighted-Jacobi sweep does not amplify it
    # (J is a contraction in the D-inner product, and renormalising scales
    # error and signal alike), so the per-column error is at most (S + 1) 2^-9;
    # the bar doubles that for the change of norm between the D- and 2-norms.
    g = GRAPHS[name]()
    S, omega, seed, level = 5, 0.7, 3, 1
    X = oracle_mod.center_normalize(_bf16_round(oracle_mod.test_vectors_raw(g.n, K, seed, level)))
    for _ in range(S):
        X = oracle_mod.center_normalize(oracle_mod.jacobi_sweep(g.n, g.u, g.v, g.w, X, omega))
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    Xb = torch.empty(g.n, K, dtype=torch.bfloat16, device=DEV)
    gr.graph_reduce_smooth(G, Xb, S, omega, seed, level)
    e = _col_relerr(Xb.double().cpu().numpy(), X)
    bar = 2 * (S + 1) * 2.0 ** -9
    assert e.max() <= bar, "bf16 %s K=%d: max per-column relative error %.3e > %.3e" % (name, K, e.max(), bar)


# Seeds whose entry (0, 0) at level 0 is an exact FP32 rounding tie, found by
# a search over seeds with the generator's published definition: in the
# first four the even neighbour lies away from zero, in the last four toward
# zero.  Each tie is re-checked from the oracle's FP64 value.
TIE_SEEDS = [10321499452505097468, 16768298687547371051, 4216642587411190979, 7405899825047084056,
             564142939147497088, 6640898608586900197, 11386581579030157594, 17095584376417309847]


@pytest.mark.parametrize("K", [4, 8, 24, 32])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_test_vectors_bit_exact(gr, oracle_mod, K, dtype):
    # ragged row count, a level and a seed above 2^63: every entry equals the
    # oracle's FP64 value rounded once to the storage type
    n, seed, level = 3037, (1 << 63) + 12345, 3
    G = gr.graph_reduce_create(n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    X = torch.empty(n, K, dtype=dtype, device=DEV)
    gr.graph_reduce_test_vectors(G, X, seed, level)
    ref = oracle_mod.test_vectors_raw(n, K, seed, level)
    if dtype == torch.float64:
        exp = torch.from_numpy(ref)
    else:
        exp = torch.from_numpy(ref.astype(np.float32)).to(dtype)
    assert torch.equal(X.cpu(), exp)


def test_test_vectors_round_ties_to_even(gr, oracle_mod):
    G = gr.graph_reduce_create(1, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    X = torch.empty(1, 4, dtype=torch.float32, device=DEV)
    ups = 0
    for seed in TIE_SEEDS:
        x = oracle_mod.test_vectors_raw(1, 4, seed, 0)[0, 0]
        lo = np.float32(x)
        if float(lo) > x:
            lo = np.nextafter(lo, np.float32(-np.inf))
        hi = np.nextafter(lo, np.float32(np.inf))
        assert (float(lo) + float(hi)) / 2.0 == x  # an exact tie
        even = lo if (lo.view(np.uint32) & 1) == 0 else hi
        ups += int(abs(float(even)) > abs(x))
        gr.graph_reduce_test_vectors(G, X, seed, 0)
        assert X[0, 0].item() == float(even)
    assert ups == 4


def test_smooth_zero_sweeps_and_edgeless(gr, oracle_mod):
    # no sweep: the centred, normalised random block itself
    g = W.grid2d(10, 10)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    X = torch.empty(g.n, 8, dtype=torch.float64, device=DEV)
    gr.graph_reduce_smooth(G, X, 0, 0.7, 3, 1)
    ref = oracle_mod.center_normalize(oracle_mod.test_vectors_raw(g.n, 8, 3, 1))
    assert _col_relerr(X.cpu().numpy(), ref).max() <= 1e-13
    # a graph without edges: every node is isolated and keeps its value
    E = gr.graph_reduce_create(50, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    X = torch.empty(50, 4, dtype=torch.float64, device=DEV)
    gr.graph_reduce_smooth(E, X, 3)
    ref = oracle_mod.smooth(50, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), 4, 3)
    assert _col_relerr(X.cpu().numpy(), ref).max() <= 1e-13


# ---------------------------------------------------------------------------
# affinity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("K", [4, 8, 16, 24, 32])
def test_affinity_parity(gr, oracle_mod, K):
    g = W.random_sparse(3001, 12000, seed=5)
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, 4)
    X[17] = 0.0  # a zero row: a = 0, d = 1
    dref, aref = oracle_mod.affinity(g.n, g.u, g.v, X, want_a=True)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    Xd = torch.from_numpy(X).to(DEV)
    d = torch.empty(g.m, dtype=torch.float64, device=DEV)
    a = torch.empty(g.m, dtype=torch.float64, device=DEV)
    gr.graph_reduce_affinity(G, Xd, d, a)
    assert np.array_equal(d.cpu().numpy(), dref)  # FP64: bit-exact given the same X
    assert np.array_equal(a.cpu().numpy(), aref)
    d32 = torch.empty(g.m, dtype=torch.float32, device=DEV)
    gr.graph_reduce_affinity(G, Xd.float(), d32)
    dref32 = oracle_mod.affinity(g.n, g.u, g.v, Xd.float().double().cpu().numpy())
    err = np.abs(d32.cpu().numpy().astype(np.float64) - dref32).max()
    assert err <= 1e-5, err


# ---------------------------------------------------------------------------
# aggregation: bit-exact given the oracle's distances
# ---------------------------------------------------------------------------
AGG_CASES = [
    ("grid", lambda: W.grid2d(64, 64), 1024, 2),
    ("grid_trunc", lambda: W.grid2d(40, 30), 500, 2),
    ("rand", lambda: W.random_sparse(5003, 20000, seed=8), 1250, 2),
    ("rand3", lambda: W.random_sparse(2000, 9000, seed=9), 1, 3),
    ("star", lambda: W.star(300), 1, 2),
    ("path_iso", GRAPHS["path_iso"], 1, 2),
    ("mesh", lambda: W.mesh3d(12, 10, 9, seed=2), 270, 2),
]


@pytest.mark.parametrize("case", AGG_CASES, ids=[c[0] for c in AGG_CASES])
def test_aggregate_bitexact_oracle_d(gr, oracle_mod, case):
    _, make, target, passes = case
    g = make()
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, 8, 5)
    d = oracle_mod.affinity(g.n, g.u, g.v, X)
    ref, rnc = oracle_mod.aggregate(g.n, g.u, g.v, d, target, passes)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    agg, nc, _ = gr.graph_reduce_aggregate(G, torch.from_numpy(d).to(DEV), target, passes)
    assert nc == rnc
    assert np.array_equal(agg.cpu().numpy(), ref)
    # FP32 keys: the same order as the oracle run on the FP32-rounded distances
    d32 = d.astype(np.float32)
    ref32, rnc32 = oracle_mod.aggregate(g.n, g.u, g.v, d32.astype(np.float64), target, passes)
    agg32, nc32, _ = gr.graph_reduce_aggregate(G, torch.from_numpy(d32).to(DEV), target, passes)
    assert nc32 == rnc32 and np.array_equal(agg32.cpu().numpy(), ref32)


@pytest.mark.parametrize("n, drop", [(60000, 9000), (200000, 50000)])
def test_aggregate_truncation_select_and_sort(gr, oracle_mod, n, drop):
    # one pass with a target below what the matching reaches, so only the
    # `allowed` smallest pairs merge: one block selects them up to 65,536
    # pairs, the radix sort above that; 50 distinct distances, so edge ids
    # break most ties
    g = W.random_sparse(n, 4 * n, seed=n)
    d = np.random.default_rng(n).integers(0, 50, g.m).astype(np.float64) / 50.0
    target = n - drop
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    for dd in (d, d.astype(np.float32)):
        ref, rnc = oracle_mod.aggregate(g.n, g.u, g.v, dd.astype(np.float64), target, 1)
        agg, nc, _ = gr.graph_reduce_aggregate(G, torch.from_numpy(dd).to(DEV), target, 1)
        assert nc == rnc == target
        assert np.array_equal(agg.cpu().numpy(), ref)


def test_aggregate_ties_and_errors(gr, oracle_mod):
    g = W.grid2d(30, 30)
    d = np.round(np.random.default_rng(1).uniform(size=g.m), 1)  # heavy ties -> edge id decides
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    for passes, target in ((1, 1), (2, 225), (3, 1)):
        ref, rnc = oracle_mod.aggregate(g.n, g.u, g.v, d, target, passes)
        agg, nc, _ = gr.graph_reduce_aggregate(G, torch.from_numpy(d).to(DEV), target, passes)
        assert nc == rnc and np.array_equal(agg.cpu().numpy(), ref)
    # a pass makes at least one proposal per matched node (64 on this path):
    # a budget of 3 turns that into GR_ETIMEOUT
    p = W.path(64)
    P = gr.graph_reduce_create(p.n, p.u, p.v, p.w)
    dp = torch.linspace(0.01, 0.9, p.m, dtype=torch.float64, device=DEV)
    with pytest.raises(gr.GraphReduceError) as ei:
        gr.graph_reduce_aggregate(P, dp, 1, 1, max_proposals=3)
    assert ei.value.status == 4
    agg, nc, proposals = gr.graph_reduce_aggregate(P, dp, 1, 1)
    ref, rnc = oracle_mod.aggregate(p.n, p.u, p.v, dp.cpu().numpy(), 1, 1)
    assert nc == rnc and np.array_equal(agg.cpu().numpy(), ref) and proposals >= 64
    with pytest.raises(gr.GraphReduceError) as ei:
        gr.graph_reduce_aggregate(P, -dp, 1, 1)
    assert ei.value.status == 1


# ---------------------------------------------------------------------------
# Galerkin coarsening: pattern bit-exact, weights <= 1e-6 relative
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", AGG_CASES[:4] + AGG_CASES[5:], ids=[c[0] for c in AGG_CASES[:4] + AGG_CASES[5:]])
def test_coarsen_parity(gr, oracle_mod, case):
    _, make, target, passes = case
    g = make()
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, 8, 5)
    d = oracle_mod.affinity(g.n, g.u, g.v, X)
    agg, nc = oracle_mod.aggregate(g.n, g.u, g.v, d, target, passes)
    uc, vc, wc = oracle_mod.coarsen(g.n, g.u, g.v, g.w, agg, nc)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    C = gr.graph_reduce_coarsen(G, torch.from_numpy(agg).to(DEV), nc)
    assert C.n == nc and C.m == len(uc)
    gu, gv, gw = (t.numpy() for t in gr.graph_reduce_get_edges(C, on_host=True))
    assert np.array_equal(gu, uc) and np.array_equal(gv, vc)
    assert np.max(np.abs(gw - wc) / wc) <= 1e-6
    assert np.array_equal(gw, wc)  # same summation order: exact
    assert np.array_equal(gr.graph_reduce_get_map(C).cpu().numpy(), agg)


def _tier_labels(n, sizes, seed):
    """Labels of aggregates with the given member counts, members scattered
    over the node range and labels in a random order."""
    rng = np.random.default_rng(seed)
    lab = np.repeat(np.arange(len(sizes)), sizes)[:n]
    lab = np.concatenate([lab, np.arange(len(sizes), len(sizes) + n - len(lab))])
    perm = rng.permutation(lab.max() + 1)
    return perm[rng.permutation(lab)].astype(np.int32)


# Coarse rows of up to 128 slots are assembled by the small-row kernel, up to
# 1,024 by the medium one; a longer row sends the whole product to the global
# sort.  Aggregates of 1-3, 40, 600 and 3,000 members of a graph of mean degree
# ~10 reach each path.
TIER_CASES = [
    ("all_medium", [40] * 150),
    ("small_and_medium", [1] * 3000 + [3] * 900 + [40] * 7),
    ("global_sort_long", [600] * 10),
    ("global_sort_two_long", [3000, 3000]),
    ("mixed", [1] * 500 + [3] * 300 + [40] * 60 + [600] * 4 + [2000]),
]


@pytest.mark.parametrize("case", TIER_CASES, ids=[c[0] for c in TIER_CASES])
def test_coarsen_row_tiers(gr, oracle_mod, case):
    _, sizes = case
    g = W.random_sparse(6000, 30000, seed=21)
    agg = _tier_labels(g.n, sizes, seed=3)
    nc = int(agg.max()) + 1
    uc, vc, wc = oracle_mod.coarsen(g.n, g.u, g.v, g.w, agg, nc)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    C = gr.graph_reduce_coarsen(G, torch.from_numpy(agg).to(DEV), nc)
    assert C.n == nc and C.m == len(uc)
    gu, gv, gw = (t.numpy() for t in gr.graph_reduce_get_edges(C, on_host=True))
    assert np.array_equal(gu, uc) and np.array_equal(gv, vc) and np.array_equal(gw, wc)
    # the coarse CSR and degrees, through a smoothing run on the coarse graph
    K, S = 8, 3
    ref = oracle_mod.smooth(nc, uc, vc, wc, K, S, 0.7, 5, 1)
    X = torch.empty(nc, K, dtype=torch.float64, device=DEV)
    gr.graph_reduce_smooth(C, X, S, 0.7, 5, 1)
    assert _col_relerr(X.cpu().numpy(), ref).max() <= 1e-12


def test_degenerate_graphs(gr, oracle_mod):
    e, ew = np.zeros(0, np.int32), np.zeros(0)
    # edgeless graphs: nothing merges, the identity map's coarse graph has no
    # edge, and the level loop makes no level
    for n in (7, 1):
        G = gr.graph_reduce_create(n, e, e, ew)
        agg, nc, _ = gr.graph_reduce_aggregate(G, torch.zeros(0, dtype=torch.float64, device=DEV), 1, 2)
        ref, rnc = oracle_mod.aggregate(n, e, e, ew, 1, 2)
        assert nc == rnc == n and np.array_equal(agg.cpu().numpy(), ref)
        C = gr.graph_reduce_coarsen(G, agg, nc)
        assert C.n == n and C.m == 0
        levels, _ = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=4, sweeps=3, prec=gr.GR_F64, final_target=1))
        assert len(levels) == len(oracle_mod.reduce_multilevel(n, e, e, ew, 4, 3, final_target=1)) == 0
    # one edge: one merge, a coarse graph of one node and no edge
    u, v, w = np.array([0], np.int32), np.array([1], np.int32), np.array([2.5])
    G = gr.graph_reduce_create(2, u, v, w)
    agg, nc, _ = gr.graph_reduce_aggregate(G, torch.tensor([0.3], dtype=torch.float64, device=DEV), 1, 2)
    assert nc == 1 and agg.cpu().tolist() == [0, 0]
    C = gr.graph_reduce_coarsen(G, agg, 1)
    assert C.n == 1 and C.m == 0
    levels, _ = gr.graph_reduce_multilevel(G, gr.ReduceParams(K=4, sweeps=3, prec=gr.GR_F64, final_target=1))
    ref = oracle_mod.reduce_multilevel(2, u, v, w, 4, 3, final_target=1)
    assert len(levels) == len(ref) == 1 and levels[0].n == 1 and levels[0].m == 0
    assert np.array_equal(gr.graph_reduce_get_map(levels[0]).cpu().numpy(), ref[0].agg)
    # identity map: the coarse graph is the fine graph, weights bit for bit
    g = W.random_sparse(1537, 6000, seed=4)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    C = gr.graph_reduce_coarsen(G, torch.arange(g.n, dtype=torch.int32, device=DEV), g.n)
    cu, cv, cw = (t.numpy() for t in gr.graph_reduce_get_edges(C, on_host=True))
    assert np.array_equal(cu, g.u) and np.array_equal(cv, g.v) and np.array_equal(cw, g.w)


def test_coarsen_rejects_bad_labels(gr):
    g = W.grid2d(8, 8)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    agg = torch.zeros(g.n, dtype=torch.int32, device=DEV)
    agg[5] = 3  # labels 1 and 2 unused
    with pytest.raises(gr.GraphReduceError):
        gr.graph_reduce_coarsen(G, agg, 4)
    agg[5] = 9
    with pytest.raises(gr.GraphReduceError):
        gr.graph_reduce_coarsen(G, agg, 4)


# ---------------------------------------------------------------------------
# level loop, FP64 end to end against the oracle's reduction
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,final", [((64, 64), 1024), ((160, 120), 700)])
def test_multilevel_f64_eigs(gr, oracle_mod, shape, final):
    g = W.grid2d(*shape)
    K, S = 8, 5
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, K, S, final_target=final)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    p = gr.ReduceParams(K=K, sweeps=S, prec=gr.GR_F64, final_target=final)
    glev, stats = gr.graph_reduce_multilevel(G, p)
    assert len(glev) == len(levels)
    for lv, gl in zip(levels, glev):
        assert gl.n == lv.nc and gl.m == len(lv.uc)
        assert np.array_equal(gr.graph_reduce_get_map(gl).cpu().numpy(), lv.agg)
    u, v, w = (t.numpy() for t in gr.graph_reduce_get_edges(glev[-1], on_host=True))
    ev_gpu = oracle_mod.smallest_nontrivial_eigs(glev[-1].n, u, v, w, 10)
    last = levels[-1]
    ev_ref = oracle_mod.smallest_nontrivial_eigs(last.nc, last.uc, last.vc, last.wc, 10)
    assert np.max(np.abs(ev_gpu - ev_ref) / ev_ref) <= 1e-3
    comp = gr.graph_reduce_compose_maps(glev).cpu().numpy()
    assert np.array_equal(comp, oracle_mod.compose_maps(levels))
    assert all(s["proposals"] > 0 for s in stats)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("S", [4, 5])
@pytest.mark.parametrize("name", ["grid160x120", "rand_w", "dense_rand"])
def test_multilevel_equals_the_calls_it_chains(gr, name, S, dtype):
    # on sparse graphs the level loop hands the smoothed block to the
    # affinity unnormalised (the affinity applies the last normalisation;
    # dense_rand, of mean degree 39, keeps the separate pass): its first two
    # levels must equal smoothing, affinity, aggregation and coarsening called
    # one by one, bit for bit, for every storage type and sweep-count parity
    g = W.grid2d(160, 120) if name == "grid160x120" else GRAPHS[name]()
    K, seed, ratio = 16, 7, 4
    prec = {torch.float64: gr.GR_F64, torch.float32: gr.GR_F32, torch.bfloat16: gr.GR_BF16}[dtype]
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    p = gr.ReduceParams(K=K, sweeps=S, seed=seed, prec=prec, level_ratio=ratio, final_target=8, max_levels=2)
    glev, _ = gr.graph_reduce_multilevel(G, p)
    assert len(glev) == 2
    cur = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    for lvl in range(2):
        X = torch.empty(cur.n, K, dtype=dtype, device=DEV)
        gr.graph_reduce_smooth(cur, X, S, 0.7, seed, lvl)
        d = torch.empty(cur.m, dtype=torch.float64 if dtype == torch.float64 else torch.float32, device=DEV)
        gr.graph_reduce_affinity(cur, X, d)
        agg, nc, _ = gr.graph_reduce_aggregate(cur, d, max((cur.n + ratio - 1) // ratio, 8))
        nxt = gr.graph_reduce_coarsen(cur, agg, nc)
        assert torch.equal(gr.graph_reduce_get_map(glev[lvl]), agg), lvl
        for a, b in zip(gr.graph_reduce_get_edges(glev[lvl]), gr.graph_reduce_get_edges(nxt)):
            assert torch.equal(a, b), lvl
        cur = nxt


# ---------------------------------------------------------------------------
# spectral-mismatch loss and its adjoint
# ---------------------------------------------------------------------------
def _loss_setup(gr, oracle_mod, n=2000, K=16, seed=31):
    g = W.random_sparse(n, 6 * n, seed=seed)
    levels = oracle_mod.reduce_multilevel(g.n, g.u, g.v, g.w, 8, 5, final_target=max(n // 32, 8))
    agg = oracle_mod.compose_maps(levels)
    last = levels[-1]
    X = oracle_mod.smooth(g.n, g.u, g.v, g.w, K, 5, seed=1)
    return g, X, agg, last


@pytest.mark.parametrize("S", [0, 1, 5])
def test_loss_and_adjoint_parity(gr, oracle_mod, S):
    g, X, agg, last = _loss_setup(gr, oracle_mod)
    rng = np.random.default_rng(2)
    wc = last.wc * rng.uniform(0.5, 2.0, size=len(last.wc))  # free weights
    L_ref, g_ref, _, _ = oracle_mod.loss(g.n, g.u, g.v, g.w, last.nc, last.uc, last.vc, wc, agg, X, S)
    F = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    C = gr.graph_reduce_create(last.nc, last.uc, last.vc, last.wc)
    Xd = torch.from_numpy(X).float().to(DEV)
    aggd = torch.from_numpy(agg).to(DEV)
    w = torch.from_numpy(wc).float().to(DEV)
    loss, saved = gr.graph_reduce_loss_fwd(F, C, aggd, Xd, w, S)
    assert abs(loss.item() - L_ref) <= 1e-4 * abs(L_ref) + 1e-7
    gw = gr.graph_reduce_loss_bwd(C, saved, X.shape[1], w, S, 0.7, torch.ones(1, device=DEV)).cpu().numpy()
    err = np.linalg.norm(gw - g_ref) / np.linalg.norm(g_ref)
    assert err <= 1e-4, err
    # through torch.autograd
    wt = w.clone().requires_grad_(True)
    lt = gr.spectral_mismatch_loss(wt, F, C, aggd, Xd, S, 0.7)
    (3.0 * lt).backward()
    assert torch.allclose(wt.grad, 3.0 * torch.from_numpy(gw).to(DEV), rtol=1e-5, atol=1e-6 * float(np.abs(gw).max()))
