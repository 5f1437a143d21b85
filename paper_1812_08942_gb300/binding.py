"""ctypes binding of libgraphreduce (include/graph_reduce.h).

Argument marshalling only: every function here forwards torch tensors (device
memory, current CUDA stream) to the C entry point of the same name.  There is
no CPU fallback; if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgraphreduce.so")
_lib = None

GR_OK, GR_EINVAL, GR_ENOMEM, GR_ECUDA, GR_ETIMEOUT, GR_ESTATE = range(6)
GR_F64, GR_F32, GR_BF16 = 0, 1, 2
GR_SWEEP_AUTO, GR_SWEEP_ROW, GR_SWEEP_STREAM, GR_SWEEP_BAND = range(4)
_STATUS = {1: "GR_EINVAL", 2: "GR_ENOMEM", 3: "GR_ECUDA", 4: "GR_ETIMEOUT", 5: "GR_ESTATE"}

EXPORTED = [
    "graph_reduce_create", "graph_reduce_get_info", "graph_reduce_test_vectors", "graph_reduce_smooth",
    "graph_reduce_smooth_noalloc", "graph_reduce_set_sweep_kernel", "graph_reduce_sweep_plan",
    "graph_reduce_smooth_gs", "graph_reduce_colour",
    "graph_reduce_affinity",
    "graph_reduce_aggregate", "graph_reduce_coarsen", "graph_reduce_get_edges", "graph_reduce_get_map",
    "graph_reduce_multilevel", "graph_reduce_compose_maps", "graph_reduce_eigensolve", "graph_reduce_reduce_data", "graph_reduce_scale_edges", "graph_reduce_loss_fwd",
    "graph_reduce_loss_bwd", "graph_reduce_launch_count", "graph_reduce_last_error", "graph_reduce_destroy",
]


class GraphReduceError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status


class gr_params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("sweeps", ctypes.c_int), ("omega", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("prec", ctypes.c_int), ("passes", ctypes.c_int),
                ("level_ratio", ctypes.c_int), ("final_target", ctypes.c_int64),
                ("max_levels", ctypes.c_int), ("max_proposals", ctypes.c_int64)]


class gr_level_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nc", ctypes.c_int64), ("mc", ctypes.c_int64),
                ("proposals", ctypes.c_int64), ("sweeps", ctypes.c_int32), ("t_smooth", ctypes.c_float),
                ("t_affinity", ctypes.c_float), ("t_aggregate", ctypes.c_float), ("t_coarsen", ctypes.c_float),
                ("t_sweeps", ctypes.c_float)]


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libgraphreduce.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libgraphreduce.so is not built; run python -m paper_1812_08942_gb300.build")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I, I64, D, U64, I32 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                              ctypes.c_uint64, ctypes.c_int32)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "graph_reduce_create": (I, [PP, I64, I64, P, P, P, I, P]),
        "graph_reduce_get_info": (I, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "graph_reduce_test_vectors": (I, [P, I, U64, I, I, P]),
        "graph_reduce_smooth": (I, [P, I, I, D, U64, I, I, P]),
        "graph_reduce_smooth_noalloc": (I, [P, I, I, D, U64, I, I, P]),
        "graph_reduce_set_sweep_kernel": (I, [P, I]),
        "graph_reduce_sweep_plan": (I, [P, I, I, ctypes.POINTER(I32)]),
        "graph_reduce_smooth_gs": (I, [P, I, I, D, U64, I, U64, I, P]),
        "graph_reduce_colour": (I, [P, U64, P, ctypes.POINTER(I32)]),
        "graph_reduce_affinity": (I, [P, P, I, I, P, P]),
        "graph_reduce_aggregate": (I, [P, P, I, I64, I, I64, P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "graph_reduce_coarsen": (I, [P, P, I64, PP]),
        "graph_reduce_get_edges": (I, [P, ctypes.POINTER(I64), P, P, P, I]),
        "graph_reduce_get_map": (I, [P, P, ctypes.POINTER(I64)]),
        "graph_reduce_multilevel": (I, [P, ctypes.POINTER(gr_params), PP, ctypes.POINTER(I),
                                        ctypes.POINTER(gr_level_stats)]),
        "graph_reduce_compose_maps": (I, [PP, I, P]),
        "graph_reduce_eigensolve": (I, [PP, I, I, I, I, D, I, P, P, P]),
        "graph_reduce_reduce_data": (I, [PP, I, P, I, I, I, P]),
        "graph_reduce_scale_edges": (I, [P, P, P, P, I, I, D, D, D, D, D, I, P, ctypes.POINTER(I32), P, P]),
        "graph_reduce_loss_fwd": (I, [P, P, P, P, I, P, I, D, P, P]),
        "graph_reduce_loss_bwd": (I, [P, P, I, P, I, D, P, P]),
        "graph_reduce_launch_count": (ctypes.c_uint64, []),
        "graph_reduce_last_error": (ctypes.c_char_p, [P]),
        "graph_reduce_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st, ctx_handle):
    if st != GR_OK:
        msg = load().graph_reduce_last_error(ctx_handle)
        raise GraphReduceError(st, msg.decode() if msg else "")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _prec_of(dtype):
    if dtype == torch.float64:
        return GR_F64
    if dtype == torch.float32:
        return GR_F32
    if dtype == torch.bfloat16:
        return GR_BF16
    raise TypeError("X must be float64, float32 or bfloat16")


class Graph:
    """Owns a gr_ctx handle; destroyed with the object."""

    def __init__(self, handle, n, m, device):
        self.handle = ctypes.c_void_p(handle)
        self.n = int(n)
        self.m = int(m)
        self.device = device

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.graph_reduce_destroy(h)
            self.handle = None

    def close(self):
        self.__del__()


# ---------------------------------------------------------------------------
# Entry points, same names as the C ABI
# ---------------------------------------------------------------------------
def graph_reduce_create(n, u, v, w, device=None) -> Graph:
    """u, v int32 and w float64, canonical.  Host tensors (or numpy arrays) are
    copied to the device by the library; CUDA tensors are read in place."""
    lib = load()
    import numpy as np
    if isinstance(u, np.ndarray):
        u, v, w = torch.from_numpy(np.ascontiguousarray(u, np.int32)), torch.from_numpy(
            np.ascontiguousarray(v, np.int32)), torch.from_numpy(np.ascontiguousarray(w, np.float64))
    on_host = not u.is_cuda
    if on_host:
        u, v, w = u.contiguous(), v.contiguous(), w.contiguous()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    else:
        dev = u.device
    assert u.dtype == torch.int32 and v.dtype == torch.int32 and w.dtype == torch.float64
    h = ctypes.c_void_p()
    with torch.cuda.device(dev):
        st = lib.graph_reduce_create(ctypes.byref(h), int(n), int(u.numel()), _ptr(u), _ptr(v), _ptr(w),
                                     1 if on_host else 0, _stream(dev))
    _check(st, None)
    return Graph(h.value, n, u.numel(), dev)


def graph_reduce_smooth(g: Graph, X, sweeps, omega=0.7, seed=0, level=0):
    """Fill X (n x K, float64 / float32 / bfloat16 on the device)."""
    assert X.is_cuda and X.is_contiguous() and X.dim() == 2 and X.shape[0] == g.n
    st = load().graph_reduce_smooth(g.handle, int(X.shape[1]), int(sweeps), float(omega), int(seed), int(level),
                                    _prec_of(X.dtype), _ptr(X))
    _check(st, g.handle)
    return X


def graph_reduce_set_sweep_kernel(g: Graph, kind: int):
    """Select the sweep kernel of g's smoothing calls (GR_SWEEP_*)."""
    _check(load().graph_reduce_set_sweep_kernel(g.handle, int(kind)), g.handle)


def graph_reduce_sweep_plan(g: Graph, K: int, dtype) -> int:
    """The sweep kernel (GR_SWEEP_ROW / GR_SWEEP_STREAM / GR_SWEEP_BAND) smoothing runs for K and dtype."""
    kind = ctypes.c_int32()
    _check(load().graph_reduce_sweep_plan(g.handle, int(K), _prec_of(dtype), ctypes.byref(kind)), g.handle)
    return int(kind.value)


def graph_reduce_test_vectors(g: Graph, X, seed=0, level=0):
    """Fill X (n x K on the device) with the raw random block before centring."""
    assert X.is_cuda and X.is_contiguous() and X.dim() == 2 and X.shape[0] == g.n
    st = load().graph_reduce_test_vectors(g.handle, int(X.shape[1]), int(seed), int(level), _prec_of(X.dtype),
                                          _ptr(X))
    _check(st, g.handle)
    return X


def graph_reduce_smooth_gs(g: Graph, X, sweeps, omega=0.7, seed=0, level=0, colour_seed=0):
    """Fill X like graph_reduce_smooth, with multicolour Gauss-Seidel sweeps."""
    assert X.is_cuda and X.is_contiguous() and X.dim() == 2 and X.shape[0] == g.n
    st = load().graph_reduce_smooth_gs(g.handle, int(X.shape[1]), int(sweeps), float(omega), int(seed), int(level),
                                       int(colour_seed), _prec_of(X.dtype), _ptr(X))
    _check(st, g.handle)
    return X


def graph_reduce_colour(g: Graph, colour_seed=0):
    """Returns (colour int32 tensor on the device, number of colours)."""
    out = torch.empty(g.n, dtype=torch.int32, device=g.device)
    nc = ctypes.c_int32(0)
    st = load().graph_reduce_colour(g.handle, int(colour_seed), _ptr(out), ctypes.byref(nc))
    _check(st, g.handle)
    return out, int(nc.value)


def graph_reduce_smooth_noalloc(g: Graph, X, sweeps, omega=0.7, seed=0, level=0):
    """Same result as graph_reduce_smooth; the library allocates nothing (its
    scratch is a fixed 32 MiB device array shared by all calls)."""
    assert X.is_cuda and X.is_contiguous() and X.dim() == 2 and X.shape[0] == g.n
    st = load().graph_reduce_smooth_noalloc(g.handle, int(X.shape[1]), int(sweeps), float(omega), int(seed),
                                            int(level), _prec_of(X.dtype), _ptr(X))
    _check(st, g.handle)
    return X


def graph_reduce_affinity(g: Graph, X, d_out, a_out=None):
    assert X.is_cuda and X.is_contiguous() and d_out.is_cuda and d_out.numel() == g.m
    st = load().graph_reduce_affinity(g.handle, _ptr(X), int(X.shape[1]), _prec_of(X.dtype), _ptr(d_out),
                                      _ptr(a_out))
    _check(st, g.handle)
    return d_out


def graph_reduce_aggregate(g: Graph, d, target_nc, passes=2, max_proposals=0, agg_out=None):
    """Returns (agg, nc, proposals)."""
    assert d.is_cuda and d.numel() == g.m and d.dtype in (torch.float32, torch.float64)
    if agg_out is None:
        agg_out = torch.empty(g.n, dtype=torch.int32, device=d.device)
    nc = ctypes.c_int64(0)
    proposals = ctypes.c_int64(0)
    st = load().graph_reduce_aggregate(g.handle, _ptr(d), 1 if d.dtype == torch.float64 else 0, int(target_nc),
                                       int(passes), int(max_proposals), _ptr(agg_out), ctypes.byref(nc),
                                       ctypes.byref(proposals))
    _check(st, g.handle)
    return agg_out, int(nc.value), int(proposals.value)


def graph_reduce_coarsen(g: Graph, agg, nc) -> Graph:
    assert agg.is_cuda and agg.dtype == torch.int32 and agg.numel() == g.n
    h = ctypes.c_void_p()
    st = load().graph_reduce_coarsen(g.handle, _ptr(agg), int(nc), ctypes.byref(h))
    _check(st, g.handle)
    n = ctypes.c_int64()
    m = ctypes.c_int64()
    load().graph_reduce_get_info(h, ctypes.byref(n), ctypes.byref(m))
    return Graph(h.value, n.value, m.value, g.device)


def graph_reduce_get_edges(g: Graph, on_host=False, out=None):
    """Canonical edge list (u, v, w) as tensors (device unless on_host).  out:
    optional (u, v, w) tensors to fill (m entries each, int32 / int32 /
    float64, on the host -- pinned for a fast copy -- or on g's device as
    on_host says), e.g. buffers a caller reuses across graphs."""
    if out is not None:
        u, v, w = out
        assert u.numel() >= g.m and v.numel() >= g.m and w.numel() >= g.m
        assert u.dtype == torch.int32 and v.dtype == torch.int32 and w.dtype == torch.float64
        assert all(t.is_cuda != bool(on_host) and t.is_contiguous() for t in (u, v, w))
        u, v, w = u[:g.m], v[:g.m], w[:g.m]
    else:
        dev = torch.device("cpu") if on_host else g.device
        kw = {"pin_memory": True} if on_host else {}
        u = torch.empty(g.m, dtype=torch.int32, device=dev, **kw)
        v = torch.empty(g.m, dtype=torch.int32, device=dev, **kw)
        w = torch.empty(g.m, dtype=torch.float64, device=dev, **kw)
    m = ctypes.c_int64()
    st = load().graph_reduce_get_edges(g.handle, ctypes.byref(m), _ptr(u), _ptr(v), _ptr(w), 1 if on_host else 0)
    _check(st, g.handle)
    return u, v, w


def graph_reduce_get_map(g: Graph):
    n = ctypes.c_int64()
    st = load().graph_reduce_get_map(g.handle, None, ctypes.byref(n))
    _check(st, g.handle)
    out = torch.empty(n.value, dtype=torch.int32, device=g.device)
    st = load().graph_reduce_get_map(g.handle, _ptr(out), ctypes.byref(n))
    _check(st, g.handle)
    return out


@dataclass
class ReduceParams:
    K: int = 16
    sweeps: int = 5
    omega: float = 0.7
    seed: int = 0
    prec: int = GR_F32
    passes: int = 2
    level_ratio: int = 4
    final_target: int = 1
    max_levels: int = 32
    max_proposals: int = 0

    def to_c(self):
        return gr_params(self.K, self.sweeps, self.omega, self.seed, self.prec, self.passes, self.level_ratio,
                         self.final_target, self.max_levels, self.max_proposals)


def graph_reduce_multilevel(g: Graph, params: ReduceParams, want_stats=True):
    """Returns (levels, stats): coarse Graphs in order, per-level dicts."""
    p = params.to_c()
    arr = (ctypes.c_void_p * params.max_levels)()
    nl = ctypes.c_int(0)
    stats = (gr_level_stats * params.max_levels)() if want_stats else None
    st = load().graph_reduce_multilevel(g.handle, ctypes.byref(p), arr, ctypes.byref(nl), stats)
    levels = []
    for i in range(nl.value):
        n = ctypes.c_int64()
        m = ctypes.c_int64()
        load().graph_reduce_get_info(arr[i], ctypes.byref(n), ctypes.byref(m))
        levels.append(Graph(arr[i], n.value, m.value, g.device))
    _check(st, g.handle)
    out = []
    if want_stats:
        for i in range(nl.value):
            s = stats[i]
            out.append(dict(n=s.n, m=s.m, nc=s.nc, mc=s.mc, proposals=s.proposals, sweeps=s.sweeps, t_smooth=s.t_smooth,
                            t_affinity=s.t_affinity, t_aggregate=s.t_aggregate, t_coarsen=s.t_coarsen,
                            t_sweeps=s.t_sweeps))
    return levels, out


def graph_reduce_eigensolve(levels, k, normalized=False, omega=0.7, iters=10, want_rayleigh=True,
                            galerkin_mass=False):
    """Multilevel Laplacian eigensolver (Alg. 5) over ``levels`` = [finest
    Graph, its coarsening, ...]; galerkin_mass selects B_l = P^T B_(l-1) P over
    each level's own B.  Returns (U, lam, rayleigh): U an n_0 x k FP64 device
    tensor, lam the coarsest eigenvalues, rayleigh the Rayleigh quotients of
    U's columns (numpy arrays)."""
    arr = (ctypes.c_void_p * len(levels))(*[lv.handle.value for lv in levels])
    U = torch.empty(levels[0].n, k, dtype=torch.float64, device=levels[0].device)
    lam = np.zeros(k, np.float64)
    rq = np.zeros(k, np.float64) if want_rayleigh else None
    st = load().graph_reduce_eigensolve(arr, len(levels), int(k), 1 if normalized else 0, 1 if galerkin_mass else 0,
                                        float(omega), int(iters),
                                        _ptr(U), lam.ctypes.data_as(ctypes.c_void_p),
                                        rq.ctypes.data_as(ctypes.c_void_p) if rq is not None else None)
    _check(st, levels[0].handle)
    return U, lam, rq


def graph_reduce_reduce_data(levels, F, mean=False):
    """Reduced data set F_R = P^T F over coarse ``levels`` (as returned by
    graph_reduce_multilevel); F is an n_fine x d float32/float64 CUDA tensor."""
    assert F.is_cuda and F.dim() == 2 and F.dtype in (torch.float32, torch.float64)
    F = F.contiguous()
    arr = (ctypes.c_void_p * len(levels))(*[lv.handle.value for lv in levels])
    out = torch.empty(levels[-1].n, F.shape[1], dtype=F.dtype, device=F.device)
    st = load().graph_reduce_reduce_data(arr, len(levels), _ptr(F), int(F.shape[1]),
                                         1 if F.dtype == torch.float64 else 0, 1 if mean else 0, _ptr(out))
    _check(st, levels[0].handle)
    return out


def graph_reduce_compose_maps(levels):
    arr = (ctypes.c_void_p * len(levels))(*[lv.handle.value for lv in levels])
    n = ctypes.c_int64()
    load().graph_reduce_get_map(levels[0].handle, None, ctypes.byref(n))
    out = torch.empty(n.value, dtype=torch.int32, device=levels[0].device)
    st = load().graph_reduce_compose_maps(arr, len(levels), _ptr(out))
    _check(st, levels[0].handle)
    return out


def graph_reduce_launch_count() -> int:
    return int(load().graph_reduce_launch_count())


def loss_saved_numel(nc, K):
    return nc * (K + 1) + K


def graph_reduce_loss_fwd(fine: Graph, coarse: Graph, agg, X, w_c, sweeps_c, omega=0.7, saved=None):
    """Returns (loss tensor (1,), saved buffer)."""
    K = int(X.shape[1])
    assert X.dtype == torch.float32 and w_c.dtype == torch.float32 and w_c.numel() == coarse.m
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    if saved is None:
        saved = torch.empty(loss_saved_numel(coarse.n, K), dtype=torch.float32, device=X.device)
    st = load().graph_reduce_loss_fwd(fine.handle, coarse.handle, _ptr(agg), _ptr(X), K, _ptr(w_c), int(sweeps_c),
                                      float(omega), _ptr(loss), _ptr(saved))
    _check(st, fine.handle)
    return loss, saved


def graph_reduce_scale_edges(fine: Graph, coarse: Graph, agg, X, w_c, sweeps_c=5, omega=0.7, alpha=0.5,
                             eta_max=1.0, delta_bar=0.5, eps=1e-3, kmax=10):
    """Scale the reduced graph's FP32 weights w_c in place (Alg. 1 driven by
    the loss gradient).  Returns (w_c, history) with history a list of
    (loss before the update, lambda_1 after it) per iteration."""
    assert X.dtype == torch.float32 and w_c.dtype == torch.float32 and w_c.numel() == coarse.m
    lh = np.zeros(kmax, np.float64)
    l1 = np.zeros(kmax, np.float64)
    it = ctypes.c_int32(0)
    st = load().graph_reduce_scale_edges(fine.handle, coarse.handle, _ptr(agg), _ptr(X), int(X.shape[1]),
                                         int(sweeps_c), float(omega), float(alpha), float(eta_max), float(delta_bar),
                                         float(eps), int(kmax), _ptr(w_c), ctypes.byref(it),
                                         lh.ctypes.data_as(ctypes.c_void_p), l1.ctypes.data_as(ctypes.c_void_p))
    _check(st, fine.handle)
    return w_c, [(float(lh[i]), float(l1[i])) for i in range(it.value)]


def graph_reduce_loss_bwd(coarse: Graph, saved, K, w_c, sweeps_c, omega, grad_loss, grad_w=None):
    if grad_w is None:
        grad_w = torch.empty(coarse.m, dtype=torch.float32, device=w_c.device)
    st = load().graph_reduce_loss_bwd(coarse.handle, _ptr(saved), int(K), _ptr(w_c), int(sweeps_c), float(omega),
                                      _ptr(grad_loss), _ptr(grad_w))
    _check(st, coarse.handle)
    return grad_w
