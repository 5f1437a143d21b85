"""FP64 CPU oracle for the spectral node-aggregation path (arXiv 1812.08942,
Sec. 3.2 Phase A and Alg. 3).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that the
CUDA library is checked against.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library itself
never does, and the two share no code.  The arithmetic lives in ``oracle.c``
(plain C, binary64, single thread, built with ``-ffp-contract=off``); this
module only marshals numpy arrays into it, runs the level loop, and holds the
eigenvalue checks (numpy / scipy FP64 solvers).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    D = ctypes.c_double
    U64 = ctypes.c_uint64
    sig = {
        "oracle_degrees": (I, [I64, I64, P, P, P, P]),
        "oracle_laplacian_apply": (I, [I64, I64, P, P, P, I, P, P]),
        "oracle_splitmix64": (U64, [U64, U64]),
        "oracle_test_vectors_raw": (None, [I64, I, U64, I, P]),
        "oracle_center_normalize": (None, [I64, I, P]),
        "oracle_jacobi_sweep": (I, [I64, I64, P, P, P, P, I, D, P, P]),
        "oracle_smooth": (I, [I64, I64, P, P, P, I, I, D, U64, I, P]),
        "oracle_affinity": (I, [I64, I64, P, P, I, P, P, P]),
        "oracle_aggregate": (I, [I64, I64, P, P, P, I64, I, P, P, P]),
        "oracle_coarsen": (I, [I64, I64, P, P, P, P, I64, P, P, P, P]),
        "oracle_loss": (I, [I64, I64, P, P, P, I64, I64, P, P, P, P, I, P, I, D, P, P, P, P]),
        "oracle_shifted_jacobi": (I, [I64, I64, P, P, P, I, P, I, D, I, P]),
        "oracle_shifted_jacobi_mass": (I, [I64, I64, P, P, P, I, P, P, D, I, P]),
        "oracle_colour": (I, [I64, I64, P, P, U64, P, P]),
        "oracle_gs_sweeps": (I, [I64, I64, P, P, P, I, P, I, D, P]),
        "oracle_smooth_gs": (I, [I64, I64, P, P, P, I, I, D, U64, I, U64, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st, what):
    if st != 0:
        raise ValueError("oracle %s failed with status %d" % (what, st))


# --------------------------------------------------------------------------
# Graph primitives (Sec. 2.1)
# --------------------------------------------------------------------------
def degrees(n, u, v, w):
    u, v, w = _i32(u), _i32(v), _f64(w)
    deg = np.empty(n, np.float64)
    _check(_load().oracle_degrees(n, len(u), _p(u), _p(v), _p(w), _p(deg)), "degrees")
    return deg


def laplacian_apply(n, u, v, w, X):
    """L X for an n x K block (or a length-n vector)."""
    u, v, w = _i32(u), _i32(v), _f64(w)
    X = _f64(X)
    vec = X.ndim == 1
    Xb = X.reshape(n, -1)
    K = Xb.shape[1]
    Y = np.empty_like(Xb)
    _check(_load().oracle_laplacian_apply(n, len(u), _p(u), _p(v), _p(w), K, _p(Xb), _p(Y)), "L apply")
    return Y.reshape(-1) if vec else Y


def dense_laplacian(n, u, v, w):
    """L as a dense matrix, column by column through ``laplacian_apply``."""
    return laplacian_apply(n, u, v, w, np.eye(n))


# --------------------------------------------------------------------------
# Test vectors and smoothing (Sec. 3.2.1, Alg. 3)
# --------------------------------------------------------------------------
def splitmix64(seed: int, c: int) -> int:
    return int(_load().oracle_splitmix64(seed, c))


def test_vectors_raw(n, K, seed=0, level=0):
    X = np.empty((n, K), np.float64)
    _load().oracle_test_vectors_raw(n, K, seed, level, _p(X))
    return X


def center_normalize(X):
    X = _f64(X).copy()
    n, K = X.shape
    _load().oracle_center_normalize(n, K, _p(X))
    return X


def jacobi_sweep(n, u, v, w, X, omega):
    """One raw weighted-Jacobi sweep of Alg. 3 (no centring / normalising)."""
    u, v, w = _i32(u), _i32(v), _f64(w)
    X = _f64(X)
    K = X.shape[1]
    deg = degrees(n, u, v, w)
    Y = np.empty_like(X)
    _check(_load().oracle_jacobi_sweep(n, len(u), _p(u), _p(v), _p(w), _p(deg), K, omega, _p(X), _p(Y)), "sweep")
    return Y


def smooth(n, u, v, w, K, sweeps, omega=0.7, seed=0, level=0):
    u, v, w = _i32(u), _i32(v), _f64(w)
    X = np.empty((n, K), np.float64)
    _check(_load().oracle_smooth(n, len(u), _p(u), _p(v), _p(w), K, sweeps, omega, seed, level, _p(X)), "smooth")
    return X


# --------------------------------------------------------------------------
# Affinity / algebraic distance (Eq. eqn:agg, Sec. 3.2.2)
# --------------------------------------------------------------------------
def affinity(n, u, v, X, want_a=False):
    u, v = _i32(u), _i32(v)
    X = _f64(X)
    K = X.shape[1]
    m = len(u)
    d = np.empty(m, np.float64)
    a = np.empty(m, np.float64) if want_a else None
    _check(_load().oracle_affinity(n, m, _p(u), _p(v), K, _p(X), _p(d), _p(a)), "affinity")
    return (d, a) if want_a else d


# --------------------------------------------------------------------------
# Aggregation (Sec. 3.2.2) and Galerkin coarsening (L_R = H_G^R L_G H_R^G)
# --------------------------------------------------------------------------
def aggregate(n, u, v, d, target_nc, passes=2):
    u, v, d = _i32(u), _i32(v), _f64(d)
    agg = np.empty(n, np.int32)
    nc = ctypes.c_int64(0)
    merges = np.zeros(max(passes, 1), np.int64)
    _check(_load().oracle_aggregate(n, len(u), _p(u), _p(v), _p(d), int(target_nc), passes,
                                    _p(agg), ctypes.byref(nc), _p(merges)), "aggregate")
    return agg, int(nc.value)


def coarsen(n, u, v, w, agg, nc):
    u, v, w, agg = _i32(u), _i32(v), _f64(w), _i32(agg)
    m = len(u)
    uc = np.empty(max(m, 1), np.int32)
    vc = np.empty(max(m, 1), np.int32)
    wc = np.empty(max(m, 1), np.float64)
    mc = ctypes.c_int64(0)
    _check(_load().oracle_coarsen(n, m, _p(u), _p(v), _p(w), _p(agg), int(nc), ctypes.byref(mc),
                                  _p(uc), _p(vc), _p(wc)), "coarsen")
    k = int(mc.value)
    return uc[:k].copy(), vc[:k].copy(), wc[:k].copy()


# --------------------------------------------------------------------------
# Spectral-mismatch loss and its hand-derived gradient
# --------------------------------------------------------------------------
def loss(n, u, v, w, nc, uc, vc, wc, agg, X, sweeps, omega=0.7, want_grad=True):
    u, v, w = _i32(u), _i32(v), _f64(w)
    uc, vc, wc, agg = _i32(uc), _i32(vc), _f64(wc), _i32(agg)
    X = _f64(X)
    K = X.shape[1]
    out = ctypes.c_double(0.0)
    g = np.empty(len(uc), np.float64) if want_grad else None
    Rf = np.empty(K, np.float64)
    Rc = np.empty(K, np.float64)
    _check(_load().oracle_loss(n, len(u), _p(u), _p(v), _p(w), int(nc), len(uc), _p(uc), _p(vc), _p(wc),
                               _p(agg), K, _p(X), sweeps, omega, ctypes.byref(out), _p(g), _p(Rf), _p(Rc)),
           "loss")
    return float(out.value), g, Rf, Rc


# --------------------------------------------------------------------------
# Edge-weight scaling of the reduced graph by constrained SGD with momentum
# (Alg. 1), driven by the exact gradient of the spectral-mismatch
# loss.  Readings: L_P is the reduced graph with the weights being scaled and
# L_G the same graph with its initial weights, so lambda_1 ~ min_p
# d_G(p) / d_P(p) (Eq. courant-fischer-3) starts at 1; the loss replaces
# lambda_n as the objective (sensitivity = d loss / d w, step size and
# convergence test from its ratio and relative decrease); every edge of an
# iteration updates from the degrees at the iteration's start (the paper
# gives no edge order); updates never go below zero (the scheme scales up).
# --------------------------------------------------------------------------
def scale_edges(n, u, v, w, nc, uc, vc, wc0, agg, X, sweeps=5, omega=0.7, alpha=0.5, eta_max=1.0,
                delta_bar=0.5, eps=1e-3, kmax=10):
    """Returns (wc, history): the scaled weights and, per iteration, the loss
    before its update and the lambda_1 estimate after it."""
    uc = np.asarray(uc, np.int64)
    vc = np.asarray(vc, np.int64)
    wc = np.array(wc0, dtype=np.float64, copy=True)
    dG = degrees(nc, uc, vc, wc)
    dP = dG.copy()
    dw = np.zeros_like(wc)
    step_delta = delta_bar ** (1.0 / kmax)  # per-iteration share of the bound
    nz = dP > 0
    lam1 = float(np.min(dG[nz] / dP[nz])) if nz.any() else 1.0
    eta = eta_max
    L0 = None
    L_prev = None
    history = []
    for k in range(1, kmax + 1):
        L, g, _, _ = loss(n, u, v, w, nc, uc, vc, wc, agg, X, sweeps, omega)
        if L0 is None:
            L0 = L
        if L_prev is not None and (L_prev - L) / L < eps:  # convergence test
            break
        dw = np.maximum(alpha * dw - eta * g, 0.0)  # momentum step, scaling up only
        bound = lam1 * step_delta
        phi_p = dG[uc] / (dP[uc] + dw)  # degree ratios after the step
        phi_q = dG[vc] / (dP[vc] + dw)
        cap = np.minimum(dG[uc] / bound - dP[uc], dG[vc] / bound - dP[vc])  # lambda_1 guard
        dw = np.where(np.minimum(phi_p, phi_q) <= bound, np.maximum(cap, 0.0), dw)
        wc = wc + dw  # weight update
        dP = degrees(nc, uc, vc, wc)
        eta = (L / L0) * eta_max  # step size from the loss ratio
        nz = dP > 0
        lam1 = float(np.min(dG[nz] / dP[nz])) if nz.any() else 1.0  # new lambda_1 estimate
        history.append((L, lam1))
        L_prev = L
    return wc, history


# --------------------------------------------------------------------------
# Level loop (the paper repeats Phase A level by level; Alg. 5 consumes the
# hierarchy).  Per-level target max(ceil(n/4), final_target).
# --------------------------------------------------------------------------
@dataclass
class Level:
    n: int
    m: int
    agg: np.ndarray
    nc: int
    uc: np.ndarray
    vc: np.ndarray
    wc: np.ndarray
    d: np.ndarray = field(repr=False, default=None)
    X: np.ndarray = field(repr=False, default=None)


def reduce_multilevel(n, u, v, w, K, sweeps, omega=0.7, seed=0, final_target=1, passes=2,
                      max_levels=64, keep=False, level_ratio=4):
    """Run smooth -> affinity -> aggregate -> coarsen until n <= final_target or
    a level makes no progress.  Returns the list of Level records."""
    levels = []
    cu, cv, cw, cn = _i32(u), _i32(v), _f64(w), int(n)
    for lvl in range(max_levels):
        if cn <= final_target or len(cu) == 0:
            break
        X = smooth(cn, cu, cv, cw, K, sweeps, omega, seed, lvl)
        d = affinity(cn, cu, cv, X)
        target = max(-(-cn // level_ratio), final_target)
        agg, nc = aggregate(cn, cu, cv, d, target, passes)
        if nc == cn:
            break
        uc, vc, wc = coarsen(cn, cu, cv, cw, agg, nc)
        levels.append(Level(cn, len(cu), agg, nc, uc, vc, wc, d if keep else None, X if keep else None))
        cu, cv, cw, cn = uc, vc, wc, nc
    return levels


def compose_maps(levels):
    """Fine-to-coarsest aggregate map: agg_L(...agg_1(i))."""
    if not levels:
        return None
    out = levels[0].agg.astype(np.int64)
    for lv in levels[1:]:
        out = lv.agg[out].astype(np.int64)
    return out.astype(np.int32)


# --------------------------------------------------------------------------
# Multicolour Gauss-Seidel smoothing (the relaxation named in Sec. 3.2.1)
# --------------------------------------------------------------------------
def colour(n, u, v, seed=0):
    """Greedy colouring in descending SplitMix64 priority (oracle_colour)."""
    lib = _load()
    u, v = _i32(u), _i32(v)
    out = np.empty(n, np.int32)
    nc = ctypes.c_int32(0)
    _check(lib.oracle_colour(n, len(u), _p(u), _p(v), ctypes.c_uint64(seed), _p(out), ctypes.byref(nc)), "colour")
    return out, int(nc.value)


def gs_order(colours):
    """Nodes in ascending (colour, id)."""
    colours = np.asarray(colours)
    return np.lexsort((np.arange(len(colours)), colours)).astype(np.int64)


def gs_sweeps(n, u, v, w, X, order, sweeps=1, omega=0.7):
    """Bare Gauss-Seidel sweeps in the given node order (no normalisation)."""
    X = np.array(X, dtype=np.float64, order="C", copy=True)
    order = np.ascontiguousarray(order, dtype=np.int64)
    lib = _load()
    u, v, w = _i32(u), _i32(v), _f64(w)
    _check(lib.oracle_gs_sweeps(n, len(u), _p(u), _p(v), _p(w), X.shape[1], _p(order), int(sweeps), float(omega),
                                _p(X)), "gs_sweeps")
    return X


def smooth_gs(n, u, v, w, K, sweeps, omega=0.7, seed=0, level=0, colour_seed=0):
    """Test vectors smoothed by multicolour Gauss-Seidel (oracle_smooth_gs)."""
    lib = _load()
    u, v, w = _i32(u), _i32(v), _f64(w)
    X = np.empty((n, K), np.float64)
    _check(lib.oracle_smooth_gs(n, len(u), _p(u), _p(v), _p(w), K, sweeps, float(omega), ctypes.c_uint64(seed),
                                level, ctypes.c_uint64(colour_seed), _p(X)), "smooth_gs")
    return X


# --------------------------------------------------------------------------
# Multilevel Laplacian eigensolver (Alg. 5, Sec. 4.1; Eqs. equ:lgl, equ:lgs)
# --------------------------------------------------------------------------
def shifted_jacobi(n, u, v, w, Y, lam, normalized=False, omega=0.7, iters=10):
    """`iters` weighted-Jacobi iterations on (L - lam_k B) y = 0 for every
    column k of Y (n x K), B = I or D (oracle_shifted_jacobi)."""
    Y = np.array(Y, dtype=np.float64, order="C", copy=True)
    K = Y.shape[1]
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    assert lam.shape == (K,)
    lib = _load()
    u, v, w = _i32(u), _i32(v), _f64(w)
    _check(lib.oracle_shifted_jacobi(n, len(u), _p(u), _p(v), _p(w), K, _p(lam), 1 if normalized else 0,
                                     float(omega), int(iters), _p(Y)), "shifted_jacobi")
    return Y


def shifted_jacobi_mass(n, u, v, w, Y, lam, b, omega=0.7, iters=10):
    """`iters` weighted-Jacobi iterations on (L - lam_k B) y = 0 with an
    explicit diagonal mass B = diag(b) (oracle_shifted_jacobi_mass)."""
    Y = np.array(Y, dtype=np.float64, order="C", copy=True)
    K = Y.shape[1]
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert lam.shape == (K,) and b.shape == (n,)
    lib = _load()
    u, v, w = _i32(u), _i32(v), _f64(w)
    _check(lib.oracle_shifted_jacobi_mass(n, len(u), _p(u), _p(v), _p(w), K, _p(lam), _p(b), float(omega),
                                          int(iters), _p(Y)), "shifted_jacobi_mass")
    return Y


def coarsest_eigenpairs(n, u, v, w, k, normalized=False, mass=None):
    """First k eigenpairs (ascending) of L u = lam B u on the coarsest graph
    (Alg. 5, step 2) by a dense symmetric eigensolver.  B = D (normalized) or
    an explicit positive diagonal `mass` is reduced to the standard problem
    B^-1/2 L B^-1/2 z = lam z, u = B^-1/2 z; a node of degree 0 takes
    B(i,i) = 1 in the normalised problem (the paper is silent)."""
    L = dense_laplacian(n, u, v, w)
    if mass is not None or normalized:
        if mass is not None:
            b = np.asarray(mass, np.float64)
        else:
            b = degrees(n, u, v, w).copy()
            b[b <= 0.0] = 1.0
        s = 1.0 / np.sqrt(b)
        lam, Z = np.linalg.eigh(s[:, None] * L * s[None, :])
        U = s[:, None] * Z
    else:
        lam, U = np.linalg.eigh(L)
    return lam[:k].copy(), np.ascontiguousarray(U[:, :k])


def galerkin_masses(graphs, maps, normalized=False):
    """The Galerkin-consistent masses B_l = P_l^T B_(l-1) P_l of every level:
    B_0 = I (ratio cut) or D (normalised cut; a degree-0 node takes 1) on the
    finest graph, and each coarser diagonal entry the sum of its members'
    entries, added in ascending member id (P_l^T B P_l is diagonal because
    each row of P_l holds a single 1)."""
    n0, u0, v0, w0 = graphs[0]
    if normalized:
        b = degrees(n0, u0, v0, w0).copy()
        b[b <= 0.0] = 1.0
    else:
        b = np.ones(n0, np.float64)
    out = [b]
    for j, mp in enumerate(maps):
        bc = np.zeros(graphs[j + 1][0], np.float64)
        np.add.at(bc, np.asarray(mp, np.int64), out[-1])
        out.append(bc)
    return out


def gram_schmidt(U):
    """Modified Gram-Schmidt over the columns of U, in column order."""
    U = np.array(U, dtype=np.float64, copy=True)
    for i in range(U.shape[1]):
        for j in range(i):
            U[:, i] -= (U[:, j] @ U[:, i]) * U[:, j]
        U[:, i] /= np.sqrt(U[:, i] @ U[:, i])
    return U


def multilevel_eigensolve(graphs, maps, k, normalized=False, omega=0.7, iters=10, mass="level"):
    """Alg. 5.  graphs[0] is the finest graph (n, u, v, w) and graphs[l] the
    graph coarsened from graphs[l-1] with aggregate map maps[l-1] (length
    n_{l-1}).  Coarsest eigenpairs, then for each finer level: map the block
    with H = P (U_fine[i] = U_coarse[map[i]]) and smooth every column with
    the coarsest eigenvalue as shift; orthonormalise at the finest level.
    mass = "level": every level's B is its own I or D (Alg. 5 as written);
    mass = "galerkin": B_l = P_l^T B_(l-1) P_l from the finest I or D
    (galerkin_masses), which makes the coarsest problem the Rayleigh-Ritz
    projection of the finest one onto the piecewise-constant vectors.
    Returns (U, lam) with lam the coarsest eigenvalues."""
    assert len(maps) == len(graphs) - 1 and mass in ("level", "galerkin")
    if mass == "level":
        lam, U = coarsest_eigenpairs(*graphs[-1], k, normalized)
    else:
        B = galerkin_masses(graphs, maps, normalized)
        lam, U = coarsest_eigenpairs(*graphs[-1], k, mass=B[-1])
    for j in range(len(graphs) - 2, -1, -1):
        U = U[np.asarray(maps[j], np.int64)]
        n, u, v, w = graphs[j]
        if mass == "level":
            U = shifted_jacobi(n, u, v, w, U, lam, normalized, omega, iters)
        else:
            U = shifted_jacobi_mass(n, u, v, w, U, lam, B[j], omega, iters)
    return gram_schmidt(U), lam


# --------------------------------------------------------------------------
# Reduced data set (Alg. 6, step 4): F_R = H_G^R F with H_G^R = P^T
# --------------------------------------------------------------------------
def reduce_features(agg, nc, F, mean=False):
    """F_R[A] = sum of F[i] over the fine nodes i with agg[i] = A, added in
    ascending i in FP64 (np.add.at applies the updates in index order);
    mean=True divides by the member count (empty aggregates stay 0)."""
    F = np.asarray(F, dtype=np.float64)
    agg = np.asarray(agg, np.int64)
    out = np.zeros((nc,) + F.shape[1:], np.float64)
    np.add.at(out, agg, F)
    if mean:
        cnt = np.bincount(agg, minlength=nc).astype(np.float64)
        nz = cnt > 0
        out[nz] = out[nz] / cnt[nz].reshape((-1,) + (1,) * (F.ndim - 1))
    return out


# --------------------------------------------------------------------------
# Eigenvalue check (method of the paper's eigenvalue figure for fe_tooth):
# the smallest nontrivial Laplacian eigenvalues, FP64 on the CPU.
# --------------------------------------------------------------------------
def n_components(n, u, v):
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    A = coo_matrix((np.ones(len(u)), (np.asarray(u), np.asarray(v))), shape=(n, n))
    return int(connected_components(A, directed=False)[0])


def sparse_laplacian(n, u, v, w):
    from scipy.sparse import coo_matrix
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    w = np.asarray(w, np.float64)
    deg = degrees(n, u, v, w)
    r = np.concatenate([u, v, np.arange(n)])
    c = np.concatenate([v, u, np.arange(n)])
    x = np.concatenate([-w, -w, deg])
    return coo_matrix((x, (r, c)), shape=(n, n)).tocsc()


def smallest_nontrivial_eigs(n, u, v, w, k=10, dense_max=8000):
    """The k smallest eigenvalues after skipping one zero per connected
    component.  The spectrum of L is the union of its components' spectra,
    each holding one zero, so each component is solved on its own: dense eigh
    when it has at most dense_max nodes, else shift-invert eigsh from a fixed
    start vector (one zero, so no repeated eigenvalue at the bottom); the
    components' nontrivial eigenvalues are merged and the k smallest returned."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    A = coo_matrix((np.ones(len(u)), (u, v)), shape=(n, n))
    c, lab = connected_components(A, directed=False)
    order = np.argsort(lab, kind="stable")
    starts = np.searchsorted(lab[order], np.arange(c + 1))
    local = np.empty(n, np.int64)
    local[order] = np.arange(n) - starts[lab[order]]
    elab = lab[u]
    eorder = np.argsort(elab, kind="stable")
    estarts = np.searchsorted(elab[eorder], np.arange(c + 1))
    found = []
    for comp in range(c):
        nc = int(starts[comp + 1] - starts[comp])
        if nc < 2:
            continue
        e = eorder[estarts[comp]:estarts[comp + 1]]
        cu, cv, cw = local[u[e]], local[v[e]], np.asarray(w)[e]
        if nc <= dense_max:
            ev = np.linalg.eigvalsh(sparse_laplacian(nc, cu, cv, cw).toarray())
            found.append(ev[1:1 + k])
        else:
            from scipy.sparse.linalg import eigsh
            L = sparse_laplacian(nc, cu, cv, cw)
            sigma = -1e-3 * float(np.asarray(L.diagonal()).mean())
            v0 = np.cos(np.arange(nc) * 0.7) + 0.5
            kk = min(k + 1, nc - 2)
            ev = np.sort(eigsh(L, k=kk, sigma=sigma, which="LM", v0=v0, tol=1e-12, return_eigenvectors=False))
            found.append(ev[1:1 + k])
    allev = np.sort(np.concatenate(found)) if found else np.zeros(0)
    return allev[:k]
