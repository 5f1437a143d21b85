/*
 * FP64 CPU oracle for the spectrum-preserving node-aggregation path of
 * "Nearly-Linear Time Spectral Graph Reduction for Scalable Graph Partitioning
 * and Data Visualization" (Zhao, Wang, Feng; arXiv 1812.08942), Sec. 3.2
 * (Phase A) and Alg. 3.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plainly written reference
 * that the CUDA library is checked against.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library, and the library
 * never calls it.
 *
 * Conventions shared by every function (they restate the paper's objects):
 *   - A graph is a canonical undirected edge list: u[e] < v[e], sorted
 *     lexicographically by (u, v), no duplicates, weights w[e] > 0.  The edge
 *     id of an edge is its position e in that list.
 *   - Vector blocks are row-major n x K: X[i*K + k] is entry i of column k.
 *   - Everything is IEEE binary64, evaluated in source order; the build uses
 *     -ffp-contract=off so no multiply-add is fused behind our back.
 *
 * Single-threaded, no blocking, no fusion: each function is the definition it
 * cites, written out.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

/* ------------------------------------------------------------------------ */
/* Sec. 2.1, Laplacian definition: D(i,i) = weighted degree, L = D - A.       */
/* deg[i] = sum of w[e] over edges e incident to i, in ascending edge id.     */
/* ------------------------------------------------------------------------ */
int oracle_degrees(int64_t n, int64_t m, const int32_t* u, const int32_t* v,
                   const double* w, double* deg) {
    for (int64_t i = 0; i < n; ++i) deg[i] = 0.0;
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] < 0 || v[e] < 0 || u[e] >= n || v[e] >= n) return OR_EINVAL;
        deg[u[e]] += w[e];
        deg[v[e]] += w[e];
    }
    return OR_OK;
}

/* Y = L X = D X - A X for a K-column block (Sec. 2.1). */
int oracle_laplacian_apply(int64_t n, int64_t m, const int32_t* u, const int32_t* v,
                           const double* w, int K, const double* X, double* Y) {
    double* deg = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!deg) return OR_ENOMEM;
    int st = oracle_degrees(n, m, u, v, w, deg);
    if (st != OR_OK) { free(deg); return st; }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < K; ++k) Y[i * K + k] = deg[i] * X[i * K + k];
    for (int64_t e = 0; e < m; ++e) {
        int64_t p = u[e], q = v[e];
        for (int k = 0; k < K; ++k) {
            Y[p * K + k] -= w[e] * X[q * K + k];
            Y[q * K + k] -= w[e] * X[p * K + k];
        }
    }
    free(deg);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Random test vectors (Sec. 3.2.1: K random vectors orthogonal to 1).         */
/* The paper does not name a generator.  Reading: entry (i, k) of level l is   */
/* drawn from output number c+1 of SplitMix64 (Steele, Lea, Flood, OOPSLA     */
/* 2014) seeded with `seed`, where c = l * 2^40 + i*K + k.  Output c+1 of that */
/* generator is mix(seed + (c+1) * gamma), gamma = 0x9E3779B97F4A7C15, mix the */
/* published variant-13 finaliser.  The 53 high bits give u in [0,1) and the   */
/* entry is 2u - 1, uniform on [-1, 1).                                       */
/* ------------------------------------------------------------------------ */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void oracle_test_vectors_raw(int64_t n, int K, uint64_t seed, int level, double* X) {
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < K; ++k) {
            uint64_t c = ((uint64_t)level << 40) + (uint64_t)i * (uint64_t)K + (uint64_t)k;
            uint64_t z = oracle_splitmix64(seed, c);
            double unit = (double)(z >> 11) * (1.0 / 9007199254740992.0); /* 2^-53 */
            X[i * K + k] = 2.0 * unit - 1.0;
        }
}

/* Orthogonalise each column against the all-ones vector (subtract its mean)
 * and scale it to unit 2-norm.  A column that is zero after centring is left
 * at zero.  (Sec. 3.2.1 asks for 1^T x = 0; unit norm is the normalisation the
 * smoothing applies between sweeps.) */
void oracle_center_normalize(int64_t n, int K, double* X) {
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += X[i * K + k];
        double mu = n > 0 ? s / (double)n : 0.0;
        for (int64_t i = 0; i < n; ++i) X[i * K + k] -= mu;
        double ss = 0.0;
        for (int64_t i = 0; i < n; ++i) ss += X[i * K + k] * X[i * K + k];
        double nrm = sqrt(ss);
        if (nrm > 0.0)
            for (int64_t i = 0; i < n; ++i) X[i * K + k] /= nrm;
    }
}

/* ------------------------------------------------------------------------ */
/* One weighted-Jacobi sweep of Alg. 3:  x <- (1 - theta) x + theta D^-1 A x,  */
/* applied to every column.  The neighbour sum of row i is accumulated in     */
/* ascending edge id, which for a canonical list is ascending neighbour id.   */
/* Isolated node (deg 0, the paper is silent): (D^-1 A x)_i := x_i.            */
/* ------------------------------------------------------------------------ */
int oracle_jacobi_sweep(int64_t n, int64_t m, const int32_t* u, const int32_t* v,
                        const double* w, const double* deg, int K, double omega,
                        const double* X, double* Y) {
    double* acc = (double*)calloc((size_t)(n > 0 ? n : 1) * (size_t)K, sizeof(double));
    if (!acc) return OR_ENOMEM;
    for (int64_t e = 0; e < m; ++e) {
        int64_t p = u[e], q = v[e];
        for (int k = 0; k < K; ++k) {
            acc[p * K + k] += w[e] * X[q * K + k];
            acc[q * K + k] += w[e] * X[p * K + k];
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < K; ++k) {
            double dax = deg[i] > 0.0 ? acc[i * K + k] / deg[i] : X[i * K + k];
            Y[i * K + k] = (1.0 - omega) * X[i * K + k] + omega * dax;
        }
    free(acc);
    return OR_OK;
}

/* Test-vector smoothing of Sec. 3.2.1 with the weighted-Jacobi relaxation of
 * Alg. 3: draw X0, centre + normalise, then `sweeps` times: one sweep followed
 * by centre + normalise.  Result written to X (n x K). */
int oracle_smooth(int64_t n, int64_t m, const int32_t* u, const int32_t* v,
                  const double* w, int K, int sweeps, double omega, uint64_t seed,
                  int level, double* X) {
    double* deg = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* Y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)K);
    if (!deg || !Y) { free(deg); free(Y); return OR_ENOMEM; }
    int st = oracle_degrees(n, m, u, v, w, deg);
    if (st != OR_OK) { free(deg); free(Y); return st; }
    oracle_test_vectors_raw(n, K, seed, level, X);
    oracle_center_normalize(n, K, X);
    for (int s = 0; s < sweeps; ++s) {
        st = oracle_jacobi_sweep(n, m, u, v, w, deg, K, omega, X, Y);
        if (st != OR_OK) break;
        memcpy(X, Y, sizeof(double) * (size_t)n * (size_t)K);
        oracle_center_normalize(n, K, X);
    }
    free(deg);
    free(Y);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Eq. (eqn:agg): affinity a_pq = (X_p,X_q)^2 / ((X_p,X_p)(X_q,X_q)), and the  */
/* algebraic distance d_pq = 1 - a_pq of Sec. 3.2.2.  With unit rows           */
/* h_p = X_p/|X_p|, 1 - a = 1 - cos^2 = (1 - cos)(1 + cos)                    */
/*                        = (|h_p - h_q|^2 / 2) (|h_p + h_q|^2 / 2),           */
/* which is what d is computed from (no cancellation when a is close to 1).   */
/* A zero row has no direction: a = 0, d = 1 (paper silent).                  */
/* Sums over k run in ascending k.  a_out may be NULL.                         */
/* ------------------------------------------------------------------------ */
int oracle_affinity(int64_t n, int64_t m, const int32_t* u, const int32_t* v, int K,
                    const double* X, double* d_out, double* a_out) {
    for (int64_t e = 0; e < m; ++e) {
        int64_t p = u[e], q = v[e];
        if (p < 0 || q < 0 || p >= n || q >= n) return OR_EINVAL;
        double c = 0.0, np_ = 0.0, nq = 0.0;
        for (int k = 0; k < K; ++k) {
            c += X[p * K + k] * X[q * K + k];
            np_ += X[p * K + k] * X[p * K + k];
            nq += X[q * K + k] * X[q * K + k];
        }
        double a, d;
        if (np_ == 0.0 || nq == 0.0) {
            a = 0.0;
            d = 1.0;
        } else {
            a = (c * c) / (np_ * nq);
            double rp = sqrt(np_), rq = sqrt(nq);
            double dm = 0.0, dp = 0.0;
            for (int k = 0; k < K; ++k) {
                double hp = X[p * K + k] / rp, hq = X[q * K + k] / rq;
                dm += (hp - hq) * (hp - hq);
                dp += (hp + hq) * (hp + hq);
            }
            d = 0.25 * dm * dp;
        }
        d_out[e] = d;
        if (a_out) a_out[e] = a;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Node aggregation (Sec. 3.2.2: nodes with small algebraic distance are      */
/* aggregated).  The paper gives no scheme; the reading used here:            */
/*   - edges are ordered by (d, edge id) ascending, a strict total order;     */
/*   - each pass forms the cluster graph (clusters = current aggregates; the  */
/*     key of the cluster pair {A,B} is the smallest (d, id) among the fine   */
/*     edges joining A and B; edges inside a cluster are ignored) and runs    */
/*     greedy matching on it: scan pairs in key order, merge a pair when both */
/*     clusters are still unmerged in this pass;                              */
/*   - a pass makes at most n_cur - target_nc merges (greedy stops there),    */
/*     and passes stop once n_cur <= target_nc;                               */
/*   - coarse label of an aggregate = rank of its smallest fine node id.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t a, b;   /* cluster representatives, a < b */
    double d;       /* key: distance of the fine edge ... */
    int64_t e;      /* ... and its id */
} or_qedge;

static int or_cmp_pair_then_key(const void* x, const void* y) {
    const or_qedge* P = (const or_qedge*)x;
    const or_qedge* Q = (const or_qedge*)y;
    if (P->a != Q->a) return P->a < Q->a ? -1 : 1;
    if (P->b != Q->b) return P->b < Q->b ? -1 : 1;
    if (P->d != Q->d) return P->d < Q->d ? -1 : 1;
    if (P->e != Q->e) return P->e < Q->e ? -1 : 1;
    return 0;
}

static int or_cmp_key(const void* x, const void* y) {
    const or_qedge* P = (const or_qedge*)x;
    const or_qedge* Q = (const or_qedge*)y;
    if (P->d != Q->d) return P->d < Q->d ? -1 : 1;
    if (P->e != Q->e) return P->e < Q->e ? -1 : 1;
    return 0;
}

int oracle_aggregate(int64_t n, int64_t m, const int32_t* u, const int32_t* v,
                     const double* d, int64_t target_nc, int passes,
                     int32_t* agg_out, int64_t* nc_out, int64_t* merges_out) {
    if (n < 0 || m < 0 || passes < 0) return OR_EINVAL;
    for (int64_t e = 0; e < m; ++e)
        if (u[e] < 0 || v[e] < 0 || u[e] >= n || v[e] >= n || u[e] == v[e] || !(d[e] >= 0.0))
            return OR_EINVAL;
    int64_t* rep = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* mate = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    or_qedge* qe = (or_qedge*)malloc(sizeof(or_qedge) * (size_t)(m > 0 ? m : 1));
    if (!rep || !mate || !qe) { free(rep); free(mate); free(qe); return OR_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) rep[i] = i;  /* cluster id = smallest member */
    int64_t n_cur = n;
    for (int pass = 0; pass < passes; ++pass) {
        if (n_cur <= target_nc) break;
        int64_t allowed = n_cur - (target_nc > 0 ? target_nc : 0);
        /* cluster graph: one key per cluster pair = min over joining edges */
        int64_t nq = 0;
        for (int64_t e = 0; e < m; ++e) {
            int64_t A = rep[u[e]], B = rep[v[e]];
            if (A == B) continue;
            qe[nq].a = A < B ? A : B;
            qe[nq].b = A < B ? B : A;
            qe[nq].d = d[e];
            qe[nq].e = e;
            ++nq;
        }
        qsort(qe, (size_t)nq, sizeof(or_qedge), or_cmp_pair_then_key);
        int64_t nu = 0;
        for (int64_t t = 0; t < nq; ++t)
            if (t == 0 || qe[t].a != qe[t - 1].a || qe[t].b != qe[t - 1].b) qe[nu++] = qe[t];
        /* greedy matching in ascending key order */
        qsort(qe, (size_t)nu, sizeof(or_qedge), or_cmp_key);
        for (int64_t i = 0; i < n; ++i) mate[i] = -1;
        int64_t merges = 0;
        for (int64_t t = 0; t < nu && merges < allowed; ++t) {
            int64_t A = qe[t].a, B = qe[t].b;
            if (mate[A] < 0 && mate[B] < 0) {
                mate[A] = B;
                mate[B] = A;
                ++merges;
            }
        }
        if (merges_out) merges_out[pass] = merges;
        /* merge: the new representative is the smaller of the two */
        for (int64_t i = 0; i < n; ++i) {
            int64_t A = rep[i];
            if (mate[A] >= 0 && mate[A] < A) rep[i] = mate[A];
        }
        n_cur -= merges;
        if (merges == 0) break;
    }
    /* labels: rank of each cluster's smallest member */
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (rep[i] == i) mate[i] = nc++;
    }
    for (int64_t i = 0; i < n; ++i) agg_out[i] = (int32_t)mate[rep[i]];
    *nc_out = nc;
    free(rep);
    free(mate);
    free(qe);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Galerkin reduced Laplacian L_R = H_G^R L_G H_R^G (Sec. 3.2.2), with the     */
/* reading H_R^G = P (P[i, agg i] = 1) and H_G^R = P^T.  Off-diagonal entries  */
/* of P^T L P are minus the summed weights of fine edges joining two distinct  */
/* aggregates, so the reduced graph has one edge (A<B) per joined pair, with   */
/* weight = sum of those fine weights in ascending fine edge id; fine edges    */
/* inside one aggregate vanish.  Output is canonical (sorted by (A,B)).        */
/* uc/vc/wc must hold m entries; *mc_out receives the reduced edge count.     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t a, b, e;
} or_cedge;

static int or_cmp_cedge(const void* x, const void* y) {
    const or_cedge* P = (const or_cedge*)x;
    const or_cedge* Q = (const or_cedge*)y;
    if (P->a != Q->a) return P->a < Q->a ? -1 : 1;
    if (P->b != Q->b) return P->b < Q->b ? -1 : 1;
    if (P->e != Q->e) return P->e < Q->e ? -1 : 1;
    return 0;
}

int oracle_coarsen(int64_t n, int64_t m, const int32_t* u, const int32_t* v,
                   const double* w, const int32_t* agg, int64_t nc, int64_t* mc_out,
                   int32_t* uc, int32_t* vc, double* wc) {
    for (int64_t i = 0; i < n; ++i)
        if (agg[i] < 0 || agg[i] >= nc) return OR_EINVAL;
    or_cedge* ce = (or_cedge*)malloc(sizeof(or_cedge) * (size_t)(m > 0 ? m : 1));
    if (!ce) return OR_ENOMEM;
    int64_t k = 0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t A = agg[u[e]], B = agg[v[e]];
        if (A == B) continue;
        ce[k].a = A < B ? A : B;
        ce[k].b = A < B ? B : A;
        ce[k].e = e;
        ++k;
    }
    qsort(ce, (size_t)k, sizeof(or_cedge), or_cmp_cedge);
    int64_t mc = 0;
    for (int64_t t = 0; t < k; ++t) {
        if (t == 0 || ce[t].a != ce[t - 1].a || ce[t].b != ce[t - 1].b) {
            uc[mc] = (int32_t)ce[t].a;
            vc[mc] = (int32_t)ce[t].b;
            wc[mc] = 0.0;
            ++mc;
        }
        wc[mc - 1] += w[ce[t].e];
    }
    *mc_out = mc;
    free(ce);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Spectral-mismatch loss and its gradient with respect to the reduced-graph  */
/* edge weights.  Not in the paper; it turns the edge-weight sensitivity of   */
/* Sec. 3.3 (d lambda / d w = -lambda (e_pq^T u)^2) into an exact gradient of  */
/* a smooth objective.  Definition:                                           */
/*   R_f[k] = x_k^T L_G x_k / x_k^T x_k            (fine Rayleigh quotient)    */
/*   M_A    = |aggregate A|,  y0 = M^-1 P^T X       (aggregate means)         */
/*   y_{s+1} = (1-omega) y_s + omega D_c^-1 A_c y_s, s < S  (Alg. 3 on L_c(w))  */
/*   R_c[k] = y^T L_c y / sum_A M_A (y_A - mu_k)^2,  mu_k = sum M_A y_A / sum M  */
/*   loss   = (1/K) sum_k (R_c[k]/R_f[k] - 1)^2                                */
/* The gradient is the hand-derived reverse sweep (adjoint of each Jacobi     */
/* step, then of the quotient); grad may be NULL.  Rf, Rc may be NULL.         */
/* ------------------------------------------------------------------------ */
int oracle_loss(int64_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w,
                int64_t nc, int64_t mc, const int32_t* uc, const int32_t* vc,
                const double* wc, const int32_t* agg, int K, const double* X, int sweeps,
                double omega, double* loss_out, double* grad, double* Rf_out,
                double* Rc_out) {
    size_t nK = (size_t)(nc > 0 ? nc : 1) * (size_t)K;
    size_t fK = (size_t)(n > 0 ? n : 1) * (size_t)K;
    double* LX = (double*)malloc(sizeof(double) * fK);
    double* Rf = (double*)malloc(sizeof(double) * (size_t)K);
    double* Mc = (double*)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
    double* Dc = (double*)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
    double* ys = (double*)calloc((size_t)(sweeps + 1) * nK, sizeof(double)); /* all iterates */
    double* zs = (double*)calloc((size_t)(sweeps > 0 ? sweeps : 1) * nK, sizeof(double));
    double* yb = (double*)calloc(nK, sizeof(double));   /* adjoint of y_s */
    double* yb2 = (double*)calloc(nK, sizeof(double));
    double* Ly = (double*)calloc(nK, sizeof(double));
    double* gRc = (double*)malloc(sizeof(double) * (size_t)K);
    double* Qk = (double*)malloc(sizeof(double) * (size_t)K);
    double* Nk = (double*)malloc(sizeof(double) * (size_t)K);
    double* muk = (double*)malloc(sizeof(double) * (size_t)K);
    int st = OR_OK;
    if (!LX || !Rf || !Mc || !Dc || !ys || !zs || !yb || !yb2 || !Ly || !gRc || !Qk || !Nk || !muk) {
        st = OR_ENOMEM;
        goto done;
    }
    for (int64_t i = 0; i < n; ++i)
        if (agg[i] < 0 || agg[i] >= nc) { st = OR_EINVAL; goto done; }
    /* fine Rayleigh quotients */
    st = oracle_laplacian_apply(n, m, u, v, w, K, X, LX);
    if (st != OR_OK) goto done;
    for (int k = 0; k < K; ++k) {
        double num = 0.0, den = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            num += X[i * K + k] * LX[i * K + k];
            den += X[i * K + k] * X[i * K + k];
        }
        Rf[k] = num / den;
        if (Rf_out) Rf_out[k] = Rf[k];
    }
    /* y0 = aggregate means */
    for (int64_t i = 0; i < n; ++i) Mc[agg[i]] += 1.0;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < K; ++k) ys[(size_t)agg[i] * K + k] += X[i * K + k];
    for (int64_t A = 0; A < nc; ++A)
        for (int k = 0; k < K; ++k)
            if (Mc[A] > 0.0) ys[(size_t)A * K + k] /= Mc[A];
    /* coarse degrees from the parameter weights */
    for (int64_t e = 0; e < mc; ++e) {
        Dc[uc[e]] += wc[e];
        Dc[vc[e]] += wc[e];
    }
    /* forward sweeps, keeping every iterate and z_s = D^-1 A y_s */
    for (int s = 0; s < sweeps; ++s) {
        const double* y = ys + (size_t)s * nK;
        double* z = zs + (size_t)s * nK;
        double* y1 = ys + (size_t)(s + 1) * nK;
        for (size_t t = 0; t < nK; ++t) z[t] = 0.0;
        for (int64_t e = 0; e < mc; ++e)
            for (int k = 0; k < K; ++k) {
                z[(size_t)uc[e] * K + k] += wc[e] * y[(size_t)vc[e] * K + k];
                z[(size_t)vc[e] * K + k] += wc[e] * y[(size_t)uc[e] * K + k];
            }
        for (int64_t A = 0; A < nc; ++A)
            for (int k = 0; k < K; ++k) {
                size_t t = (size_t)A * K + k;
                z[t] = Dc[A] > 0.0 ? z[t] / Dc[A] : y[t];
                y1[t] = (1.0 - omega) * y[t] + omega * z[t];
            }
    }
    /* coarse Rayleigh quotients with the M-weighted centred denominator */
    const double* yS = ys + (size_t)sweeps * nK;
    double Msum = 0.0;
    for (int64_t A = 0; A < nc; ++A) Msum += Mc[A];
    for (size_t t = 0; t < nK; ++t) Ly[t] = 0.0;
    for (int64_t e = 0; e < mc; ++e)
        for (int k = 0; k < K; ++k) {
            double diff = yS[(size_t)uc[e] * K + k] - yS[(size_t)vc[e] * K + k];
            Ly[(size_t)uc[e] * K + k] += wc[e] * diff;
            Ly[(size_t)vc[e] * K + k] -= wc[e] * diff;
        }
    double loss = 0.0;
    for (int k = 0; k < K; ++k) {
        double mu = 0.0;
        for (int64_t A = 0; A < nc; ++A) mu += Mc[A] * yS[(size_t)A * K + k];
        mu /= Msum;
        double N = 0.0, Q = 0.0;
        for (int64_t e = 0; e < mc; ++e) {
            double diff = yS[(size_t)uc[e] * K + k] - yS[(size_t)vc[e] * K + k];
            N += wc[e] * diff * diff;
        }
        for (int64_t A = 0; A < nc; ++A) {
            double c = yS[(size_t)A * K + k] - mu;
            Q += Mc[A] * c * c;
        }
        double Rc = N / Q;
        if (Rc_out) Rc_out[k] = Rc;
        double r = Rc / Rf[k] - 1.0;
        loss += r * r;
        gRc[k] = 2.0 * r / Rf[k] / (double)K;
        Nk[k] = N;
        Qk[k] = Q;
        muk[k] = mu;
    }
    loss /= (double)K;
    *loss_out = loss;
    if (!grad) goto done;
    for (int64_t e = 0; e < mc; ++e) grad[e] = 0.0;
    /* adjoint of R_c: direct weight term and d R_c / d y_S */
    for (int64_t e = 0; e < mc; ++e)
        for (int k = 0; k < K; ++k) {
            double diff = yS[(size_t)uc[e] * K + k] - yS[(size_t)vc[e] * K + k];
            grad[e] += gRc[k] * diff * diff / Qk[k];
        }
    for (int64_t A = 0; A < nc; ++A)
        for (int k = 0; k < K; ++k) {
            size_t t = (size_t)A * K + k;
            double c = yS[t] - muk[k];
            yb[t] = gRc[k] * (2.0 * Ly[t] / Qk[k] - 2.0 * Nk[k] * Mc[A] * c / (Qk[k] * Qk[k]));
        }
    /* reverse sweeps: yb holds the adjoint of y_{s+1}; produce that of y_s */
    for (int s = sweeps - 1; s >= 0; --s) {
        const double* y = ys + (size_t)s * nK;
        const double* z = zs + (size_t)s * nK;
        for (int64_t e = 0; e < mc; ++e) {
            int64_t A = uc[e], B = vc[e];
            for (int k = 0; k < K; ++k) {
                double ga = yb[(size_t)A * K + k] * omega * (y[(size_t)B * K + k] - z[(size_t)A * K + k]) / Dc[A];
                double gb = yb[(size_t)B * K + k] * omega * (y[(size_t)A * K + k] - z[(size_t)B * K + k]) / Dc[B];
                grad[e] += ga + gb;
            }
        }
        for (size_t t = 0; t < nK; ++t) yb2[t] = 0.0;
        for (int64_t e = 0; e < mc; ++e) {
            int64_t A = uc[e], B = vc[e];
            for (int k = 0; k < K; ++k) {
                yb2[(size_t)A * K + k] += wc[e] * yb[(size_t)B * K + k] / Dc[B];
                yb2[(size_t)B * K + k] += wc[e] * yb[(size_t)A * K + k] / Dc[A];
            }
        }
        for (int64_t A = 0; A < nc; ++A)
            for (int k = 0; k < K; ++k) {
                size_t t = (size_t)A * K + k;
                /* isolated aggregate: the sweep left y unchanged */
                yb2[t] = Dc[A] > 0.0 ? (1.0 - omega) * yb[t] + omega * yb2[t] : yb[t];
            }
        memcpy(yb, yb2, sizeof(double) * nK);
    }
done:
    free(LX); free(Rf); free(Mc); free(Dc); free(ys); free(zs); free(yb); free(yb2);
    free(Ly); free(gRc); free(Qk); free(Nk); free(muk);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Alg. 5 (multilevel Laplacian eigensolver), the smoothing of a mapped       */
/* eigenvector block: `iters` weighted-Jacobi iterations on                   */
/* (L - lambda_k B) y = 0 for every column k of Y (Eq. equ:lgl), with B = I   */
/* (ratio cut) or B = D (normalised cut).  Splitting L - lambda B into its    */
/* diagonal D - lambda B and off-diagonal -A, one iteration is                 */
/*   y <- (1 - theta) y + theta (D - lambda_k B)^-1 A y.                       */
/* The paper is silent on a non-positive shifted diagonal (an isolated node,  */
/* or a shift past the degree): such a row keeps its value.  Neighbour sums   */
/* in ascending edge id.                                                       */
/* ------------------------------------------------------------------------ */
int oracle_shifted_jacobi(int64_t n, int64_t m, const int32_t* u, const int32_t* v,
                          const double* w, int K, const double* lambda, int normalized,
                          double omega, int iters, double* Y) {
    double* deg = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* acc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)K);
    if (!deg || !acc) {
        free(deg);
        free(acc);
        return OR_ENOMEM;
    }
    int st = oracle_degrees(n, m, u, v, w, deg);
    for (int it = 0; st == OR_OK && it < iters; ++it) {
        memset(acc, 0, sizeof(double) * (size_t)n * (size_t)K);
        for (int64_t e = 0; e < m; ++e) {
            int64_t p = u[e], q = v[e];
            for (int k = 0; k < K; ++k) {
                acc[p * K + k] += w[e] * Y[q * K + k];
                acc[q * K + k] += w[e] * Y[p * K + k];
            }
        }
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < K; ++k) {
                double diag = deg[i] - lambda[k] * (normalized ? deg[i] : 1.0);
                if (diag > 0.0)
                    Y[i * K + k] = (1.0 - omega) * Y[i * K + k] + omega * (acc[i * K + k] / diag);
            }
    }
    free(deg);
    free(acc);
    return st;
}

/* ------------------------------------------------------------------------ */
/* The same smoothing for an explicit diagonal mass B = diag(b) (the          */
/* Galerkin-consistent mass of a coarse level, B_c = P^T B P, is diagonal):   */
/*   y <- (1 - theta) y + theta (D - lambda_k b)^-1 A y,                       */
/* a row whose shifted diagonal is not positive keeping its value; neighbour  */
/* sums in ascending edge id.                                                  */
/* ------------------------------------------------------------------------ */
int oracle_shifted_jacobi_mass(int64_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w, int K,
                               const double* lambda, const double* b, double omega, int iters, double* Y) {
    double* deg = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* acc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)K);
    if (!deg || !acc) {
        free(deg);
        free(acc);
        return OR_ENOMEM;
    }
    int st = oracle_degrees(n, m, u, v, w, deg);
    for (int it = 0; st == OR_OK && it < iters; ++it) {
        memset(acc, 0, sizeof(double) * (size_t)n * (size_t)K);
        for (int64_t e = 0; e < m; ++e) {
            int64_t p = u[e], q = v[e];
            for (int k = 0; k < K; ++k) {
                acc[p * K + k] += w[e] * Y[q * K + k];
                acc[q * K + k] += w[e] * Y[p * K + k];
            }
        }
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < K; ++k) {
                double diag = deg[i] - lambda[k] * b[i];
                if (diag > 0.0)
                    Y[i * K + k] = (1.0 - omega) * Y[i * K + k] + omega * (acc[i * K + k] / diag);
            }
    }
    free(deg);
    free(acc);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Multicolour Gauss-Seidel (the relaxation Sec. 3.2.1 names).  The paper     */
/* gives no ordering; reading: a greedy colouring in descending priority,      */
/* priority of node i = (output number c+1 of SplitMix64 seeded with `seed`,   */
/* c = 2^62 + i; then the larger id wins a tie), each node taking the smallest */
/* colour not used by its already-coloured neighbours.  A sweep then visits    */
/* the nodes in ascending (colour, id).                                        */
/* ------------------------------------------------------------------------ */
static uint64_t or_prio(uint64_t seed, int64_t i) {
    return oracle_splitmix64(seed, ((uint64_t)1 << 62) + (uint64_t)i);
}

typedef struct {
    uint64_t p;
    int64_t i;
} or_prio_node;

static int or_cmp_prio_desc(const void* x, const void* y) {
    const or_prio_node* a = (const or_prio_node*)x;
    const or_prio_node* b = (const or_prio_node*)y;
    if (a->p != b->p) return a->p > b->p ? -1 : 1;
    return a->i > b->i ? -1 : (a->i < b->i ? 1 : 0);
}

/* adjacency lists in ascending edge id (= ascending neighbour id): nbr/wt of
 * node i at [ptr[i], ptr[i+1]) */
static int or_adjacency(int64_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w, int64_t** ptr_out,
                        int32_t** nbr_out, double** wt_out) {
    int64_t* ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m > 0 ? 2 * m : 1));
    double* wt = (double*)malloc(sizeof(double) * (size_t)(2 * m > 0 ? 2 * m : 1));
    if (!ptr || !fill || !nbr || !wt) {
        free(ptr);
        free(fill);
        free(nbr);
        free(wt);
        return OR_ENOMEM;
    }
    for (int64_t e = 0; e < m; ++e) {
        ptr[u[e] + 1]++;
        ptr[v[e] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
    /* edges in ascending id; for node i the edges (q, i), q < i, come before
       the edges (i, r), and each group is in ascending id */
    for (int64_t e = 0; e < m; ++e) {
        int64_t p = u[e], q = v[e];
        int64_t sq = ptr[q] + fill[q]++;
        nbr[sq] = (int32_t)p;
        wt[sq] = w ? w[e] : 0.0;
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t p = u[e], q = v[e];
        int64_t sp = ptr[p] + fill[p]++;
        nbr[sp] = (int32_t)q;
        wt[sp] = w ? w[e] : 0.0;
    }
    free(fill);
    *ptr_out = ptr;
    *nbr_out = nbr;
    *wt_out = wt;
    return OR_OK;
}

int oracle_colour(int64_t n, int64_t m, const int32_t* u, const int32_t* v, uint64_t seed, int32_t* colour,
                  int32_t* ncolours) {
    int64_t* ptr;
    int32_t* nbr;
    double* wt;
    int st = or_adjacency(n, m, u, v, NULL, &ptr, &nbr, &wt);
    if (st != OR_OK) return st;
    or_prio_node* order = (or_prio_node*)malloc(sizeof(or_prio_node) * (size_t)(n > 0 ? n : 1));
    unsigned char* used = (unsigned char*)calloc((size_t)n + 2, 1);
    if (!order || !used) {
        free(order);
        free(used);
        free(ptr);
        free(nbr);
        free(wt);
        return OR_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i) {
        order[i].p = or_prio(seed, i);
        order[i].i = i;
        colour[i] = -1;
    }
    qsort(order, (size_t)n, sizeof(or_prio_node), or_cmp_prio_desc);
    int32_t nc = 0;
    for (int64_t t = 0; t < n; ++t) {
        int64_t i = order[t].i;
        for (int64_t j = ptr[i]; j < ptr[i + 1]; ++j)
            if (colour[nbr[j]] >= 0) used[colour[nbr[j]]] = 1;
        int32_t c = 0;
        while (used[c]) ++c;
        colour[i] = c;
        if (c + 1 > nc) nc = c + 1;
        for (int64_t j = ptr[i]; j < ptr[i + 1]; ++j)
            if (colour[nbr[j]] >= 0) used[colour[nbr[j]]] = 0;
    }
    *ncolours = nc;
    free(order);
    free(used);
    free(ptr);
    free(nbr);
    free(wt);
    return OR_OK;
}

/* One Gauss-Seidel sweep x_i <- (1 - theta) x_i + theta (sum_j w_ij x_j) / D(i,i)
 * over the nodes in the given order, each update seeing the latest values;
 * neighbour sums in ascending edge id; an isolated node keeps its value. */
static void or_gs_sweep(int64_t n, const int64_t* ptr, const int32_t* nbr, const double* wt, const double* deg,
                        const int64_t* order, int K, double omega, double* X, double* acc) {
    for (int64_t t = 0; t < n; ++t) {
        int64_t i = order[t];
        if (!(deg[i] > 0.0)) continue;
        for (int k = 0; k < K; ++k) acc[k] = 0.0;
        for (int64_t j = ptr[i]; j < ptr[i + 1]; ++j)
            for (int k = 0; k < K; ++k) acc[k] += wt[j] * X[(int64_t)nbr[j] * K + k];
        for (int k = 0; k < K; ++k) X[i * K + k] = (1.0 - omega) * X[i * K + k] + omega * (acc[k] / deg[i]);
    }
}

typedef struct {
    int32_t c;
    int64_t i;
} or_colour_node;

static int or_cmp_colour_id(const void* x, const void* y) {
    const or_colour_node* a = (const or_colour_node*)x;
    const or_colour_node* b = (const or_colour_node*)y;
    if (a->c != b->c) return a->c < b->c ? -1 : 1;
    return a->i < b->i ? -1 : (a->i > b->i ? 1 : 0);
}

/* `sweeps` Gauss-Seidel sweeps in the given node order (n entries), no
 * normalisation: the bare relaxation, for pins */
int oracle_gs_sweeps(int64_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w, int K,
                     const int64_t* order, int sweeps, double omega, double* X) {
    int64_t* ptr;
    int32_t* nbr;
    double* wt;
    int st = or_adjacency(n, m, u, v, w, &ptr, &nbr, &wt);
    if (st != OR_OK) return st;
    double* deg = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* acc = (double*)malloc(sizeof(double) * (size_t)K);
    if (!deg || !acc) st = OR_ENOMEM;
    if (st == OR_OK) st = oracle_degrees(n, m, u, v, w, deg);
    for (int s = 0; st == OR_OK && s < sweeps; ++s) or_gs_sweep(n, ptr, nbr, wt, deg, order, K, omega, X, acc);
    free(deg);
    free(acc);
    free(ptr);
    free(nbr);
    free(wt);
    return st;
}

/* Test-vector smoothing with multicolour Gauss-Seidel: X0 as for Alg. 3,
 * centre + normalise, then `sweeps` times one sweep in (colour, id) order of
 * the colouring seeded with `colour_seed`, followed by centre + normalise. */
int oracle_smooth_gs(int64_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w, int K, int sweeps,
                     double omega, uint64_t seed, int level, uint64_t colour_seed, double* X) {
    int32_t* colour = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    or_colour_node* cn = (or_colour_node*)malloc(sizeof(or_colour_node) * (size_t)(n > 0 ? n : 1));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t nc = 0;
    int st = (colour && cn && order) ? OR_OK : OR_ENOMEM;
    if (st == OR_OK) st = oracle_colour(n, m, u, v, colour_seed, colour, &nc);
    if (st == OR_OK) {
        for (int64_t i = 0; i < n; ++i) {
            cn[i].c = colour[i];
            cn[i].i = i;
        }
        qsort(cn, (size_t)n, sizeof(or_colour_node), or_cmp_colour_id);
        for (int64_t t = 0; t < n; ++t) order[t] = cn[t].i;
        oracle_test_vectors_raw(n, K, seed, level, X);
        oracle_center_normalize(n, K, X);
        for (int s = 0; st == OR_OK && s < sweeps; ++s) {
            st = oracle_gs_sweeps(n, m, u, v, w, K, order, 1, omega, X);
            oracle_center_normalize(n, K, X);
        }
    }
    free(colour);
    free(cn);
    free(order);
    return st;
}
