"""GB300 (sm_103a) spectral node aggregation: the Phase (A) hot path of
"Nearly-Linear Time Spectral Graph Reduction" (Zhao, Wang, Feng; arXiv
1812.08942) -- test-vector smoothing, spectral affinity, aggregation and
Galerkin coarsening -- as hand-written CUDA behind the C ABI in
include/graph_reduce.h, with a thin ctypes binding of the same names.
"""
from .binding import (  # noqa: F401
    GR_BF16, GR_EINVAL, GR_F32, GR_F64, GR_SWEEP_AUTO, GR_SWEEP_BAND, GR_SWEEP_ROW, GR_SWEEP_STREAM,
    Graph, GraphReduceError, ReduceParams, graph_reduce_affinity,
    graph_reduce_aggregate, graph_reduce_coarsen, graph_reduce_colour, graph_reduce_compose_maps, graph_reduce_create,
    graph_reduce_eigensolve, graph_reduce_get_edges, graph_reduce_get_map, graph_reduce_loss_bwd, graph_reduce_loss_fwd,
    graph_reduce_launch_count, graph_reduce_multilevel, graph_reduce_reduce_data, graph_reduce_scale_edges, graph_reduce_smooth, graph_reduce_smooth_gs, graph_reduce_test_vectors, graph_reduce_smooth_noalloc,
    graph_reduce_set_sweep_kernel, graph_reduce_sweep_plan, lib_path, load,
)
from .autograd import SpectralMismatchLoss, spectral_mismatch_loss  # noqa: F401
