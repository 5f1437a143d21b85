"""The allocation-free smoothing entry point (graph_reduce_smooth_noalloc).

It serves callers that must not allocate device memory once running (a fixed
pre-reserved budget, or another framework's allocator): instead of the
context's workspace it uses one fixed 32 MiB device array inside the library.
It runs graph_reduce_smooth's own launch sequence, so the check is bitwise:
through the C ABI, two calls in a row give exactly the vectors
graph_reduce_smooth gives, for FP64, FP32 and BF16 storage, each sweep kernel
and the automatic choice, on a random and a banded graph, and 0, 4 and 5
sweeps (an even count ends in place in X).  The first calls run on a fresh
context, so the FP64 packed slots, the streaming kernel's row partition and
the band kernel's tables are built inside the fixed array; a block too large
for the array is refused.  This file is named to be collected last.
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


GRAPHS = {
    "random": lambda: W.random_sparse(20011, 90000, seed=17),
    "grid": lambda: W.grid2d(200, 1100),  # banded and large: the automatic choice takes the band kernel
}


@pytest.mark.parametrize("sweeps", [0, 4, 5])
@pytest.mark.parametrize("kernel", ["ROW", "STREAM", "BAND", "AUTO"])
@pytest.mark.parametrize("dtype,K", [(torch.float64, 8), (torch.float32, 16), (torch.float32, 24),
                                     (torch.bfloat16, 16)])
@pytest.mark.parametrize("graph", list(GRAPHS))
def test_noalloc_equals_smooth_bitwise(gr, graph, dtype, K, kernel, sweeps):
    g = GRAPHS[graph]()
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)  # fresh: holds no packed slots, partition nor band tables
    gr.graph_reduce_set_sweep_kernel(G, getattr(gr, "GR_SWEEP_" + kernel))
    outs = []
    for _ in range(2):
        X = torch.full((g.n, K), float("nan"), dtype=dtype, device=DEV)
        gr.graph_reduce_smooth_noalloc(G, X, sweeps, 0.7, 11, 1)
        torch.cuda.synchronize()
        outs.append(X)
    ref = torch.empty(g.n, K, dtype=dtype, device=DEV)
    gr.graph_reduce_smooth(G, ref, sweeps, 0.7, 11, 1)
    torch.cuda.synchronize()
    assert torch.isfinite(ref.float()).all()
    for X in outs:
        assert torch.equal(X, ref)
    if graph == "grid" and kernel == "AUTO" and dtype == torch.float32 and K == 16:
        assert gr.graph_reduce_sweep_plan(G, K, dtype) == gr.GR_SWEEP_BAND


def test_noalloc_rejects_blocks_beyond_the_scratch(gr):
    n = 600_000  # 600k x 16 floats = 38.4 MB > 32 MiB
    E = gr.graph_reduce_create(n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    X = torch.empty(n, 16, dtype=torch.float32, device=DEV)
    with pytest.raises(gr.GraphReduceError) as ei:
        gr.graph_reduce_smooth_noalloc(E, X, 2)
    assert ei.value.status == gr.GR_EINVAL
