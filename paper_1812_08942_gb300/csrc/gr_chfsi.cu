// Coarsest eigenpairs of the multilevel eigensolver (Alg. 5 step 2, Sec. 4.1,
// Eq. equ:lgs): the k smallest eigenpairs of L u = lambda B u on the coarsest
// graph, B diagonal and positive (an entry that is not positive -- a
// degree-0 node under B = D -- counts as 1).  With S = B^-1/2 the problem is
// the standard one A x = lambda x, A = S L S, u = S x; A is never formed:
// products with it run over the coarsest graph's CSR.
//
// Method: Chebyshev-filtered subspace iteration (Zhou and Saad, "A Chebyshev-
// Davidson algorithm for large symmetric eigenproblems", SIAM J. Matrix Anal.
// Appl. 29 (2007); Zhou, Saad, Tiago and Chelikowsky, J. Comput. Phys. 219
// (2006)) on a block of p = k + max(8, k/2) columns (at most n; doubled, up
// to 64, while the block's largest Ritz value is 0 to within 1e-10 beta --
// a null space wider than the block, as on graphs of many components):
//   1. X: a seeded random block, orthonormalised, Rayleigh-Ritz'd.
//   2. Repeat: Y = T_d((A - c I) / e) X / T_d((0 - c) / e), the Chebyshev
//      polynomial of degree d that is bounded by 1 on [alpha, beta] (alpha =
//      the block's largest Ritz value, beta = a Gershgorin bound of A) and
//      equals 1 at 0, the bottom of A's spectrum (A is positive
//      semi-definite); orthonormalise Y twice by SVQB (Stathopoulos and Wu,
//      SIAM J. Sci. Comput. 23 (2002): the Gram matrix's eigenvectors scaled
//      by its eigenvalues^-1/2, after unit column scaling); Rayleigh-Ritz
//      (eigenpairs of Y^T A Y rotate Y); until the k first Ritz pairs have
//      residuals ||A x - theta x|| <= 1e-13 beta.
//   The degree is the largest (up to 4,000) for which the filter grows by at
//   most 1e6 between 0 and alpha, which bounds the filtered block's condition
//   number and keeps the SVQB steps accurate in FP64; a small alpha / beta
//   (eigenvalues clustered near 0 against a wide spectrum) thus gets a high
//   degree rather than many iterations.
// The small p x p symmetric eigenproblems (Gram and Rayleigh-Ritz matrices,
// p <= 64) run in one thread block by the cyclic Jacobi method with the
// round-robin parallel ordering (Golub and Van Loan, Matrix Computations,
// Sec. 8.5).  Every reduction is FP64 in a fixed order.
#include <math.h>
#include <string.h>

#include <vector>

#include "gr_internal.cuh"

namespace gr {

namespace {

constexpr int CT = 256;
constexpr int CF_PMAX = 64;       // block columns at most (k <= 32)
constexpr int CF_ROWS = 16;       // rows staged per step of a Gram partial
constexpr int CF_SWEEPS = 60;     // Jacobi sweeps at most
constexpr int CF_MAX_ITERS = 400; // filter iterations at most
constexpr int CF_DEG_MAX = 4000; // filter degree at most
constexpr double CF_GROWTH = 1e6; // filter growth between 0 and alpha at most
constexpr double CF_TOL = 1e-13;  // residual bar, relative to beta
constexpr double CF_DENSE_RATE = 0.05;  // per-degree rate below which small graphs go dense

// S = B^-1/2 as a vector (b = NULL: B = I)
__global__ void k_cf_scale(int64_t n, const double* __restrict__ b, double* __restrict__ sc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sc[i] = b ? 1.0 / sqrt(b[i] > 0.0 ? b[i] : 1.0) : 1.0;
}

// seeded start block: the 64-bit finaliser of MurmurHash3 over (seed, index),
// mapped to [-1, 1)
__device__ __forceinline__ double cf_uniform(uint64_t seed, uint64_t i) {
    uint64_t z = seed ^ (i * 0x9E3779B97F4A7C15ull);
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdull;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ull;
    z ^= z >> 33;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__global__ void k_cf_init(int64_t n, int p, uint64_t seed, double* __restrict__ X) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * p;
         idx += (int64_t)gridDim.x * blockDim.x)
        X[idx] = cf_uniform(seed, (uint64_t)idx);
}

// Y (n x pn) = [X (n x p) | seeded columns]
__global__ void k_cf_widen(int64_t n, int p, int pn, uint64_t seed, const double* __restrict__ X,
                           double* __restrict__ Y) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * pn;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / pn;
        const int c = (int)(idx % pn);
        Y[idx] = c < p ? X[i * p + c] : cf_uniform(seed, (uint64_t)idx);
    }
}

// Gershgorin bound of A = S L S: max_i s_i (s_i deg_i + sum_j w_ij s_j), as
// the bit pattern of a non-negative double (an integer max is exact and
// order-free).  Warp per row.
__global__ void k_cf_bound(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ eid, const double* __restrict__ ew,
                           const double* __restrict__ deg, const double* __restrict__ sc,
                           unsigned long long* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        double t = 0.0;
        for (int64_t j = rowptr[i] + lane; j < rowptr[i + 1]; j += 32) t += ew[eid[j]] * sc[col[j]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) {
            const double si = sc[i];
            const double v = si * (si * deg[i] + t);
            atomicMax(out, (unsigned long long)__double_as_longlong(v > 0.0 ? v : 0.0));
        }
    }
}

// Entries of A = S L S in the CSR's slots: off-diagonal -s_i w_ij s_j, and
// the diagonal s_i^2 deg_i per row
__global__ void k_cf_values(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ eid, const double* __restrict__ ew,
                            const double* __restrict__ deg, const double* __restrict__ sc, double* __restrict__ av,
                            double* __restrict__ ad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double si = sc[i];
        ad[i] = si * si * deg[i];
        for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) av[j] = -si * ew[eid[j]] * sc[col[j]];
    }
}

// Out = c1 (A Y) + c2 Y + c3 Yp (Yp may be NULL), n x p row-major, A from
// its slot values av and diagonal ad.  Short rows: warp per row, lanes over
// columns, the row's products in slot order.
__global__ void k_cf_apply(int64_t n, int p, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const double* __restrict__ av, const double* __restrict__ ad, double c1, double c2,
                           double c3, const double* __restrict__ Y, const double* __restrict__ Yp,
                           double* __restrict__ Out) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t j0 = rowptr[i], j1 = rowptr[i + 1];
        for (int q = lane; q < p; q += 32) {
            const double yi = Y[i * p + q];
            double acc = ad[i] * yi;
            for (int64_t j = j0; j < j1; ++j) acc += av[j] * Y[(int64_t)col[j] * p + q];
            double o = c1 * acc + c2 * yi;
            if (Yp) o += c3 * Yp[i * p + q];
            Out[i * p + q] = o;
        }
    }
}

// The same for long rows (dense coarse graphs): warp per row, lanes over the
// row's slots, 16 columns at a time in registers; each lane's partial sums in
// slot order, then a fixed butterfly over the lanes.
constexpr int CF_QC = 16;
__global__ void k_cf_apply_long(int64_t n, int p, const int64_t* __restrict__ rowptr,
                                const int32_t* __restrict__ col, const double* __restrict__ av,
                                const double* __restrict__ ad, double c1, double c2, double c3,
                                const double* __restrict__ Y, const double* __restrict__ Yp,
                                double* __restrict__ Out) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t j0 = rowptr[i], j1 = rowptr[i + 1];
        for (int q0 = 0; q0 < p; q0 += CF_QC) {
            double acc[CF_QC];
#pragma unroll
            for (int u = 0; u < CF_QC; ++u) acc[u] = 0.0;
            for (int64_t j = j0 + lane; j < j1; j += 32) {
                const double a = av[j];
                const double* yr = Y + (int64_t)col[j] * p + q0;
#pragma unroll
                for (int u = 0; u < CF_QC; ++u)
                    if (q0 + u < p) acc[u] += a * yr[u];
            }
#pragma unroll
            for (int u = 0; u < CF_QC; ++u)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
            if (lane < CF_QC && q0 + lane < p) {
                double a = 0.0;
#pragma unroll
                for (int u = 0; u < CF_QC; ++u)
                    if (u == lane) a = acc[u];
                const int q = q0 + lane;
                const double yi = Y[i * p + q];
                double o = c1 * (ad[i] * yi + a) + c2 * yi;
                if (Yp) o += c3 * Yp[i * p + q];
                Out[i * p + q] = o;
            }
        }
    }
}

// Gram partials P1^T P2 over each block's contiguous row range (rows staged
// in shared memory, summed in row order); part holds gridDim.x p x p blocks.
__global__ void __launch_bounds__(CT) k_cf_gram(int64_t n, int p, const double* __restrict__ Y1,
                                                const double* __restrict__ Y2, double* __restrict__ part) {
    __shared__ double s1[CF_ROWS * CF_PMAX], s2[CF_ROWS * CF_PMAX];
    constexpr int PER = CF_PMAX * CF_PMAX / CT;  // entries per thread at p = 64
    double acc[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) acc[u] = 0.0;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = r0 + chunk < n ? r0 + chunk : n;
    const int pp = p * p;
    for (int64_t t0 = r0; t0 < r1; t0 += CF_ROWS) {
        const int rows = (int)(r1 - t0 < CF_ROWS ? r1 - t0 : CF_ROWS);
        __syncthreads();
        for (int e = threadIdx.x; e < rows * p; e += CT) {
            s1[e] = Y1[t0 * p + e];
            s2[e] = Y2[t0 * p + e];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = threadIdx.x + u * CT;
            if (e < pp) {
                const int a = e / p, c = e % p;
                double t = acc[u];
                for (int r = 0; r < rows; ++r) t += s1[r * p + a] * s2[r * p + c];
                acc[u] = t;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * CT;
        if (e < pp) part[(int64_t)blockIdx.x * pp + e] = acc[u];
    }
}

// G = sum of the partials, block by block in order
__global__ void k_cf_gram_finish(int nb, int p, const double* __restrict__ part, double* __restrict__ G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p * p) return;
    double t = 0.0;
    for (int q = 0; q < nb; ++q) t += part[(int64_t)q * p * p + e];
    G[e] = t;
}

// Out = Y M (n x p times p x p, row-major); M staged in shared memory
__global__ void k_cf_mul(int64_t n, int p, const double* __restrict__ Y, const double* __restrict__ M,
                         double* __restrict__ Out) {
    __shared__ double sm[CF_PMAX * CF_PMAX];
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) sm[e] = M[e];
    __syncthreads();
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * p;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / p;
        const int c = (int)(idx % p);
        const double* yi = Y + i * p;
        double t = 0.0;
        for (int r = 0; r < p; ++r) t += yi[r] * sm[r * p + c];
        Out[idx] = t;
    }
}

// Squared residual norms of the first k Ritz pairs, per block over its row
// range (rows in order): part[blk * k + c] = sum_i (AX[i,c] - theta_c X[i,c])^2
__global__ void k_cf_resid(int64_t n, int p, int k, const double* __restrict__ AX, const double* __restrict__ X,
                           const double* __restrict__ theta, double* __restrict__ part) {
    const int c = threadIdx.x;
    if (c >= k) return;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = r0 + chunk < n ? r0 + chunk : n;
    const double th = theta[c];
    double t = 0.0;
    for (int64_t i = r0; i < r1; ++i) {
        const double r = AX[i * p + c] - th * X[i * p + c];
        t += r * r;
    }
    part[(int64_t)blockIdx.x * k + c] = t;
}

__global__ void k_cf_resid_finish(int nb, int k, const double* __restrict__ part, double* __restrict__ rn) {
    const int c = threadIdx.x;
    if (c >= k) return;
    double t = 0.0;
    for (int q = 0; q < nb; ++q) t += part[(int64_t)q * k + c];
    rn[c] = sqrt(t);
}

// U = S X[:, :k] (row-major n x k) and the first k Ritz values
__global__ void k_cf_take(int64_t n, int p, int k, const double* __restrict__ X, const double* __restrict__ sc,
                          double* __restrict__ U) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t i = idx / k;
    const int c = (int)(idx % k);
    U[idx] = sc[i] * X[i * p + c];
}

// Small symmetric eigenproblem in one block of CT threads, p <= 64, in
// dynamic shared memory (2 p^2 doubles + pair tables).
//   mode 0 (SVQB): in = Gram matrix G; with D = diag(G)^-1/2 the matrix
//     D G D = V diag(l) V^T; out = D V diag(max(l, 1e-15 max l))^-1/2, so that
//     Y out has orthonormal columns up to rounding.
//   mode 1 (Rayleigh-Ritz): in = Y^T A Y (symmetrised); out = its
//     eigenvectors with eigenvalues theta in ascending order.
// Cyclic Jacobi, round-robin ordering: index 0 fixed and 1 .. m-1 on a
// circle (m = p rounded up to even; index p, when present, is a dummy), so
// each step rotates m/2 disjoint pairs at once: rows, then columns and V.
__global__ void __launch_bounds__(CT) k_cf_small(int p, int mode, const double* __restrict__ in,
                                                 double* __restrict__ out, double* __restrict__ theta) {
    extern __shared__ double sh[];
    double* A = sh;          // p x p
    double* V = sh + p * p;  // p x p
    __shared__ double dsc[CF_PMAX];
    __shared__ double pc[CF_PMAX / 2], ps[CF_PMAX / 2];
    __shared__ int pa[CF_PMAX / 2], pb[CF_PMAX / 2];
    __shared__ double red[CT];
    __shared__ int rank[CF_PMAX];
    const int tid = threadIdx.x;
    const int m = p + (p & 1), half = m / 2;
    for (int a = tid; a < p; a += CT) {
        const double g = in[a * p + a];
        dsc[a] = mode == 0 ? (g > 0.0 ? 1.0 / sqrt(g) : 1.0) : 1.0;
    }
    __syncthreads();
    for (int e = tid; e < p * p; e += CT) {
        const int a = e / p, c = e % p;
        A[e] = mode == 0 ? dsc[a] * in[e] * dsc[c] : 0.5 * (in[e] + in[c * p + a]);
        V[e] = a == c ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < CF_SWEEPS; ++sweep) {
        // stop once every off-diagonal entry is at rounding level of the diagonal
        double off = 0.0, dg = 0.0;
        for (int e = tid; e < p * p; e += CT) {
            const int a = e / p, c = e % p;
            if (a == c) dg = fmax(dg, fabs(A[e]));
            else off = fmax(off, fabs(A[e]));
        }
        red[tid] = off;
        __syncthreads();
        for (int o = CT / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
            __syncthreads();
        }
        off = red[0];
        __syncthreads();
        red[tid] = dg;
        __syncthreads();
        for (int o = CT / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
            __syncthreads();
        }
        dg = red[0];
        __syncthreads();
        if (off <= 4e-16 * dg || off == 0.0) break;
        for (int t = 0; t < m - 1; ++t) {
            if (tid < half) {
                int a, c;
                if (tid == 0) {
                    a = 0;
                    c = 1 + t % (m - 1);
                } else {
                    a = 1 + (t + tid) % (m - 1);
                    c = 1 + (t - tid + (m - 1)) % (m - 1);
                }
                if (a > c) {
                    const int x = a;
                    a = c;
                    c = x;
                }
                double cs = 1.0, sn = 0.0;
                if (c < p) {
                    const double apq = A[a * p + c];
                    if (apq != 0.0) {
                        // zero the (a, c) entry: tan = sign(tau) / (|tau| + sqrt(1 + tau^2))
                        const double tau = (A[c * p + c] - A[a * p + a]) / (2.0 * apq);
                        const double at = fabs(tau);
                        const double tn = at > 1e150 ? 0.5 / at : 1.0 / (at + sqrt(1.0 + tau * tau));
                        const double tt = tau >= 0.0 ? tn : -tn;
                        cs = 1.0 / sqrt(1.0 + tt * tt);
                        sn = tt * cs;
                    }
                }
                pa[tid] = a;
                pb[tid] = c;
                pc[tid] = cs;
                ps[tid] = sn;
            }
            __syncthreads();
            for (int e = tid; e < half * p; e += CT) {  // rows a and c
                const int r = e / p, q = e % p;
                const int a = pa[r], c = pb[r];
                if (c >= p || ps[r] == 0.0) continue;
                const double x = A[a * p + q], y = A[c * p + q];
                A[a * p + q] = pc[r] * x - ps[r] * y;
                A[c * p + q] = ps[r] * x + pc[r] * y;
            }
            __syncthreads();
            for (int e = tid; e < half * p; e += CT) {  // columns a and c, and V
                const int r = e / p, q = e % p;
                const int a = pa[r], c = pb[r];
                if (c >= p || ps[r] == 0.0) continue;
                const double x = A[q * p + a], y = A[q * p + c];
                A[q * p + a] = pc[r] * x - ps[r] * y;
                A[q * p + c] = ps[r] * x + pc[r] * y;
                const double vx = V[q * p + a], vy = V[q * p + c];
                V[q * p + a] = pc[r] * vx - ps[r] * vy;
                V[q * p + c] = ps[r] * vx + pc[r] * vy;
            }
            __syncthreads();
        }
    }
    // ascending order of the eigenvalues (ties by index)
    for (int a = tid; a < p; a += CT) {
        const double la = A[a * p + a];
        int r = 0;
        for (int c = 0; c < p; ++c) {
            const double lc = A[c * p + c];
            r += (lc < la || (lc == la && c < a)) ? 1 : 0;
        }
        rank[a] = r;
    }
    __syncthreads();
    if (mode == 0) {
        double lmax = 0.0;
        for (int a = 0; a < p; ++a) lmax = fmax(lmax, A[a * p + a]);
        for (int e = tid; e < p * p; e += CT) {
            const int a = e / p, c = e % p;  // out[a, rank(c)] = d_a V[a, c] / sqrt(l_c)
            const double l = fmax(A[c * p + c], 1e-15 * lmax);
            out[a * p + rank[c]] = dsc[a] * V[e] / sqrt(l > 0.0 ? l : 1.0);
        }
    } else {
        for (int e = tid; e < p * p; e += CT) {
            const int a = e / p, c = e % p;
            out[a * p + rank[c]] = V[e];
        }
        for (int a = tid; a < p; a += CT) theta[rank[a]] = A[a * p + a];
    }
}

}  // namespace

// The k smallest eigenpairs of L u = lambda B u on graph c (b: the diagonal
// of B, NULL for B = I): lam_dev / lam_host (k ascending eigenvalues),
// U (n x k row-major, column j an eigenvector for lam[j]); scratch from the
// workspace slot WS_EIG_WORK of ws.  *iters: the filter iterations run (-1:
// handed to the dense route).
gr_status coarsest_eigenpairs(gr_ctx* c, const double* b, int k, Workspace& ws, cudaStream_t s, double* lam_dev,
                              double* lam_host, double* U, int* iters) {
    const int64_t n = c->n;
    // graphs up to DENSE_EIG_MAX nodes switch to the dense route as soon as
    // the filter would need thousands of degrees (below)
    auto go_dense = [&]() -> gr_status {
        if (iters) *iters = -1;
        return dense_eigenpairs(c, b, k, ws, s, lam_dev, lam_host, U);
    };
    int p = (int)(n < (int64_t)(k + (k / 2 > 8 ? k / 2 : 8)) ? n : (int64_t)(k + (k / 2 > 8 ? k / 2 : 8)));
    const int pcap = (int)(n < (int64_t)CF_PMAX ? n : (int64_t)CF_PMAX);
    if (k < 1 || k > 32 || p > CF_PMAX || n < k) return set_error(c, GR_EINVAL, "eigensolve: k out of range");
    const int nbg = (int)(ceil_div(n, 64) < (int64_t)c->num_sms ? ceil_div(n, 64) : (int64_t)c->num_sms);
    const int nb = nbg > 0 ? nbg : 1;
    size_t need = 0;
    auto add = [&](size_t bytes) {
        const size_t off = need;
        need += (bytes + 255) & ~size_t(255);
        return off;
    };
    // every block sized for the widest block the iteration may grow to
    const size_t blk = sizeof(double) * (size_t)n * pcap;
    const size_t o_X = add(blk), o_AX = add(blk), o_Y0 = add(blk), o_Y1 = add(blk), o_Y2 = add(blk),
                 o_part = add(sizeof(double) * (size_t)nb * pcap * pcap), o_G = add(sizeof(double) * pcap * pcap),
                 o_T = add(sizeof(double) * pcap * pcap), o_th = add(sizeof(double) * CF_PMAX),
                 o_rn = add(sizeof(double) * CF_PMAX), o_bd = add(64), o_sc = add(sizeof(double) * (size_t)n),
                 o_ad = add(sizeof(double) * (size_t)n), o_av = add(sizeof(double) * (size_t)(2 * c->m > 0 ? 2 * c->m : 1));
    void* base;
    GR_TRY_CUDA(c, ws.get(WS_EIG_WORK, need, &base), "eigensolve: scratch");
    char* Bp = (char*)base;
    double* X = (double*)(Bp + o_X);
    double* AX = (double*)(Bp + o_AX);
    double* Yb[3] = {(double*)(Bp + o_Y0), (double*)(Bp + o_Y1), (double*)(Bp + o_Y2)};
    double* part = (double*)(Bp + o_part);
    double* G = (double*)(Bp + o_G);
    double* T = (double*)(Bp + o_T);
    double* th = (double*)(Bp + o_th);
    double* rn = (double*)(Bp + o_rn);
    unsigned long long* bd = (unsigned long long*)(Bp + o_bd);
    double* sc = (double*)(Bp + o_sc);
    double* ad = (double*)(Bp + o_ad);
    double* av = (double*)(Bp + o_av);
    const bool long_rows = n > 0 && 2.0 * (double)c->m / (double)n >= 64.0;
    const unsigned wgrid = (unsigned)(ceil_div(n * 32, CT) < (int64_t)c->num_sms * 8 ? ceil_div(n * 32, CT)
                                                                                     : (int64_t)c->num_sms * 8);
    const unsigned egrid = (unsigned)(ceil_div(n * pcap, CT) < (int64_t)c->num_sms * 8 ? ceil_div(n * pcap, CT)
                                                                                        : (int64_t)c->num_sms * 8);
    GR_TRY_CUDA(c, cudaFuncSetAttribute(k_cf_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(sizeof(double) * 2 * pcap * pcap)),
                "eigensolve: smem");
    auto small_smem = [&]() { return sizeof(double) * 2 * p * p; };

    auto apply = [&](double c1, double c2, double c3, const double* Y, const double* Yp, double* Out) {
        if (long_rows)
            k_cf_apply_long<<<wgrid, CT, 0, s>>>(n, p, c->rowptr, c->col, av, ad, c1, c2, c3, Y, Yp, Out);
        else
            k_cf_apply<<<wgrid, CT, 0, s>>>(n, p, c->rowptr, c->col, av, ad, c1, c2, c3, Y, Yp, Out);
        count_launch();
    };
    auto gram = [&](const double* Y1, const double* Y2) {
        k_cf_gram<<<nb, CT, 0, s>>>(n, p, Y1, Y2, part);
        count_launch();
        k_cf_gram_finish<<<(unsigned)ceil_div(p * p, CT), CT, 0, s>>>(nb, p, part, G);
        count_launch();
    };
    auto mul = [&](const double* Y, const double* M, double* Out) {
        k_cf_mul<<<egrid, CT, 0, s>>>(n, p, Y, M, Out);
        count_launch();
    };
    // Y (in Yb[yi]) orthonormalised twice by SVQB; returns the index of the result
    auto svqb2 = [&](int yi) {
        for (int pass = 0; pass < 2; ++pass) {
            gram(Yb[yi], Yb[yi]);
            k_cf_small<<<1, CT, small_smem(), s>>>(p, 0, G, T, nullptr);
            count_launch();
            const int zi = (yi + 1) % 3;
            mul(Yb[yi], T, Yb[zi]);
            yi = zi;
        }
        return yi;
    };
    std::vector<double> hv((size_t)CF_PMAX * 2);
    // Rayleigh-Ritz of the orthonormal block Yb[yi]: X, AX, theta; residuals of
    // the first k pairs and theta read back
    auto rayleigh_ritz = [&](int yi) -> cudaError_t {
        double* AY = Yb[(yi + 1) % 3];
        apply(1.0, 0.0, 0.0, Yb[yi], nullptr, AY);
        gram(Yb[yi], AY);
        k_cf_small<<<1, CT, small_smem(), s>>>(p, 1, G, T, th);
        count_launch();
        mul(Yb[yi], T, X);
        mul(AY, T, AX);
        k_cf_resid<<<nb, 64, 0, s>>>(n, p, k, AX, X, th, part);
        count_launch();
        k_cf_resid_finish<<<1, 64, 0, s>>>(nb, k, part, rn);
        count_launch();
        GR_CUDA(cudaMemcpyAsync(hv.data(), th, sizeof(double) * p, cudaMemcpyDeviceToHost, s));
        GR_CUDA(cudaMemcpyAsync(hv.data() + CF_PMAX, rn, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
        GR_CUDA(cudaStreamSynchronize(s));
        return cudaGetLastError();
    };

    // S and the spectrum bound beta
    k_cf_scale<<<(unsigned)ceil_div(n, CT), CT, 0, s>>>(n, b, sc);
    count_launch();
    GR_TRY_CUDA(c, cudaMemsetAsync(bd, 0, sizeof(unsigned long long), s), "memset");
    k_cf_bound<<<wgrid, CT, 0, s>>>(n, c->rowptr, c->col, c->eid, c->ew, c->deg, sc, bd);
    count_launch();
    k_cf_values<<<(unsigned)ceil_div(n, CT), CT, 0, s>>>(n, c->rowptr, c->col, c->eid, c->ew, c->deg, sc, av, ad);
    count_launch();
    unsigned long long hb = 0;
    GR_TRY_CUDA(c, cudaMemcpyAsync(&hb, bd, sizeof(hb), cudaMemcpyDeviceToHost, s), "readback");
    GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
    double beta;
    memcpy(&beta, &hb, sizeof(beta));
    const double tol = CF_TOL * (beta > 0.0 ? beta : 1.0);

    // start: seeded block, orthonormalised, Rayleigh-Ritz
    k_cf_init<<<egrid, CT, 0, s>>>(n, p, 0x5EEDC0A25E5Eull, Yb[0]);
    count_launch();
    int yi = svqb2(0);
    GR_TRY_CUDA(c, rayleigh_ritz(yi), "eigensolve: Rayleigh-Ritz");
    auto converged = [&]() {
        for (int j = 0; j < k; ++j)
            if (!(hv[CF_PMAX + j] <= tol)) return false;
        return true;
    };
    int it = 0;
    // a block of all n columns spans the space: its Rayleigh-Ritz pairs are exact
    while (p < n && !converged()) {
        if (++it > CF_MAX_ITERS) return set_error(c, GR_ECUDA, "eigensolve: the coarsest eigenpairs did not converge");
        if (hv[p - 1] <= 1e-10 * beta && p < pcap && n <= DENSE_EIG_MAX) return go_dense();
        if (hv[p - 1] <= 1e-10 * beta && p < pcap) {
            // the block lies in a cluster at 0 at least p wide (a graph of many
            // components): widen it with fresh seeded columns and start over
            const int pn = 2 * p < pcap ? 2 * p : pcap;
            k_cf_widen<<<egrid, CT, 0, s>>>(n, p, pn, 0x5EEDC0A25E5Eull + (uint64_t)it, X, Yb[0]);
            count_launch();
            p = pn;
            yi = svqb2(0);
            GR_TRY_CUDA(c, rayleigh_ritz(yi), "eigensolve: Rayleigh-Ritz");
            continue;
        }
        const double alpha = hv[p - 1] > 1e-10 * beta ? hv[p - 1] : 1e-10 * beta;
        // beta bounds the spectrum from above; should the block's top Ritz value
        // reach it, damp just above that value
        const double top = beta > alpha * (1.0 + 1e-9) ? beta : alpha * (1.0 + 1e-6) + 1e-300;
        // Chebyshev filter on [alpha, top], normalised to 1 at 0
        const double e = 0.5 * (top - alpha), cc = 0.5 * (top + alpha);
        const double x0 = (0.0 - cc) / e;  // <= -1
        const double g = acosh(-x0);
        const double dmax = g > 0.0 ? acosh(CF_GROWTH) / g : (double)CF_DEG_MAX;
        const int d = dmax < 2.0 ? 2 : (dmax > (double)CF_DEG_MAX ? CF_DEG_MAX : (int)dmax);
        // after two filtered passes the Ritz values predict the rate: the
        // slowest wanted pair gains acosh(t) per degree against [alpha, top];
        // below CF_DENSE_RATE (some 600 degrees for 1e-13) the dense route is
        // cheaper, where the graph is small enough for it
        if (it > 2 && n <= DENSE_EIG_MAX) {
            const double tw = (alpha + top - 2.0 * hv[k - 1]) / (top - alpha);
            if (!(tw > 1.0) || acosh(tw) < CF_DENSE_RATE) return go_dense();
        }
        // rho_j = T_j(x0); Y_{j+1} = (2 rho_j / rho_{j+1}) x(A) Y_j - (rho_{j-1} / rho_{j+1}) Y_{j-1}
        double rm1 = 1.0, r0 = x0;
        int cur = (yi + 1) % 3, prv = yi;  // X is the current Ritz block
        apply(1.0 / (r0 * e), -cc / (r0 * e), 0.0, X, nullptr, Yb[cur]);
        const double* ym1 = X;
        for (int j = 1; j < d; ++j) {
            const double r1 = 2.0 * x0 * r0 - rm1;
            const int nxt = (cur + 1) % 3 == prv ? (cur + 2) % 3 : (cur + 1) % 3;
            apply(2.0 * r0 / (r1 * e), -2.0 * r0 * cc / (r1 * e), -rm1 / r1, Yb[cur], ym1, Yb[nxt]);
            ym1 = Yb[cur];
            prv = cur;
            cur = nxt;
            rm1 = r0;
            r0 = r1;
        }
        yi = svqb2(cur);
        GR_TRY_CUDA(c, rayleigh_ritz(yi), "eigensolve: Rayleigh-Ritz");
    }
    for (int j = 0; j < k; ++j) lam_host[j] = hv[j];
    GR_TRY_CUDA(c, cudaMemcpyAsync(lam_dev, th, sizeof(double) * k, cudaMemcpyDeviceToDevice, s), "copy");
    k_cf_take<<<(unsigned)ceil_div(n * k, CT), CT, 0, s>>>(n, p, k, X, sc, U);
    count_launch();
    GR_TRY_CUDA(c, cudaGetLastError(), "eigensolve: coarsest vectors");
    if (iters) *iters = it;
    return GR_OK;
}

}  // namespace gr
