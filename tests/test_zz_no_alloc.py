"""The allocation-free smoothing entry point (graph_reduce_smooth_noalloc).

It serves callers that must not allocate device memory once running (a fixed
pre-reserved budget, or another framework's allocator): instead of the
context's workspace it uses one fixed 32 MiB device array inside the library.
The check: through the C ABI, two calls in a row give the same vectors as
graph_reduce_smooth within the smoothing tolerances of the parity tests
(per-column relative error 1e-12 in FP64, 1e-5 in FP32), and a block too large
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


def _relerr(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


@pytest.mark.parametrize("dtype,K,tol", [(torch.float32, 16, 1e-5), (torch.float64, 8, 1e-12),
                                         (torch.float32, 24, 1e-5)])
def test_noalloc_matches_smooth_twice(gr, dtype, K, tol):
    g = W.random_sparse(20011, 90000, seed=17)
    G = gr.graph_reduce_create(g.n, g.u, g.v, g.w)
    ref = torch.empty(g.n, K, dtype=dtype, device=DEV)
    gr.graph_reduce_smooth(G, ref, 5, 0.7, 11, 1)
    for _ in range(2):
        X = torch.full((g.n, K), float("nan"), dtype=dtype, device=DEV)
        gr.graph_reduce_smooth_noalloc(G, X, 5, 0.7, 11, 1)
        torch.cuda.synchronize()
        assert _relerr(X, ref) <= tol


def test_noalloc_rejects_blocks_beyond_the_scratch(gr):
    n = 600_000  # 600k x 16 floats = 38.4 MB > 32 MiB
    E = gr.graph_reduce_create(n, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    X = torch.empty(n, 16, dtype=torch.float32, device=DEV)
    with pytest.raises(gr.GraphReduceError) as ei:
        gr.graph_reduce_smooth_noalloc(E, X, 2)
    assert ei.value.status == 1
