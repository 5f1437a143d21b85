// Coarsest eigenpairs of the multilevel eigensolver (Alg. 5 step 2, Sec. 4.1,
// Eq. equ:lgs) for coarsest graphs of at most DENSE_EIG_MAX nodes: the k
// smallest eigenpairs of A = S L S (S = B^-1/2, entries of B that are not
// positive count as 1), u = S x, by the classical dense route, whose cost
// does not depend on how the eigenvalues are spread (Golub and Van Loan,
// Matrix Computations, Secs. 8.3-8.4):
//   1. Householder reduction A = Q T Q^T to a symmetric tridiagonal T: one
//      cooperative kernel; reflector j zeroes column j below the
//      subdiagonal and updates the trailing block by the symmetric rank-2
//      form A22 - u w^T - w u^T, w = p - (tau/2)(p^T u) u, p = tau A22 u;
//      the blocks meet at grid barriers (bounded waits).
//   2. The k smallest eigenvalues of T by bisection on Sturm counts
//      (multisection: a warp evaluates 32 points of the interval at once).
//   3. Their eigenvectors by inverse iteration on T - lambda I (Gaussian
//      elimination with partial pivoting on the tridiagonal), eigenvalues
//      closer than 1e-3 ||T|| treated as a cluster whose vectors are
//      re-orthogonalised (modified Gram-Schmidt, in order) after every step.
//   4. x = Q z, the reflectors applied in reverse order; U = S x.
// All FP64; every reduction in a fixed order.
#include <math.h>

#include <vector>

#include "gr_internal.cuh"

namespace gr {

namespace {

constexpr int DT = 256;                            // threads per block
constexpr int DW = DT / 32;                        // warps per block
constexpr long long DENSE_WAIT_CYCLES = 2000000000ll;  // ~1 s at 2 GHz
constexpr int INVIT_STEPS = 5;
constexpr double DEPS = 2.220446049250313e-16;

// A (column-major, n x n) = S L S
__global__ void k_dn_build(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ eid, const double* __restrict__ ew,
                           const double* __restrict__ deg, const double* __restrict__ b, double* __restrict__ A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    auto scl = [&](int64_t r) { return b ? 1.0 / sqrt(b[r] > 0.0 ? b[r] : 1.0) : 1.0; };
    const double si = scl(i);
    A[i * n + i] = si * si * deg[i];
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
        const int64_t c = col[j];
        A[c * n + i] = -si * ew[eid[j]] * scl(c);
    }
}

struct TriArgs {
    double* A;
    int n;
    double* d;
    double* e;
    double* tau;
    double* p;       // n
    double* part;    // gridDim.x
    unsigned* count; // grid barrier
    unsigned* gen;
    int* abort;
    int* err;
};

// Grid barrier for a cooperative launch: arrival counter and generation word;
// a wait gives up after about a second (sets abort and the error word), and a
// block seeing abort leaves.  Returns false once aborted (block-uniform).
__device__ bool grid_sync(const TriArgs& a) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vg = a.gen;
        volatile int* va = a.abort;
        const unsigned g = *vg;
        __threadfence();
        if (atomicAdd(a.count, 1u) == gridDim.x - 1) {
            atomicExch(a.count, 0u);
            __threadfence();
            atomicAdd(a.gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vg == g) {
                __nanosleep(32);
                if (*va) break;
                if (clock64() - t0 > DENSE_WAIT_CYCLES) {
                    atomicExch(a.abort, 1);
                    atomicExch(a.err, 1);
                    break;
                }
            }
        }
        __threadfence();
        ok = *va == 0;
    }
    __syncthreads();
    return ok != 0;
}

// warp sum in a fixed butterfly
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int COLV = DENSE_EIG_MAX / DT;  // column entries per thread of block 0

// block-wide sum in a fixed order (every thread gets the result)
__device__ double block_sum(double v) {
    __shared__ double red[DT];
    __syncthreads();
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = DT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// Block 0's share of a step: column jc (rows jc .. n-1, held in registers,
// thread t owning rows jc + t + DT q) optionally updated by the step's rank-2
// form first (u = column jc - 1's reflector, w = p - K u, at offset 1 in the
// step's indexing), then turned into its own reflector: x = A[jc+1 .., jc]
// becomes u (u_0 = 1, u_i = x_i / (x_0 - beta)) with H x = beta e_0, H = I -
// tau u u^T; d[jc], e[jc] = beta, tau[jc] recorded.
__device__ void column_reflector(const TriArgs& a, int jc, bool update, double K) {
    const int n = a.n, t = threadIdx.x;
    double* cc = a.A + (int64_t)jc * n;  // column jc, rows from 0
    double v[COLV];
    const double* uprev = a.A + (int64_t)(jc - 1) * n + jc;  // reflector of column jc - 1, from row jc
    double uc = 0.0, wc = 0.0;
    if (update) {
        uc = __ldcg(uprev);  // = 1
        wc = __ldcg(a.p) - K * uc;
    }
#pragma unroll
    for (int q = 0; q < COLV; ++q) {
        const int r = jc + t + DT * q;
        v[q] = r < n ? __ldcg(cc + r) : 0.0;
    }
    if (update) {
#pragma unroll
        for (int q = 0; q < COLV; ++q) {
            const int r = jc + t + DT * q;
            if (r < n) {
                const double ui = __ldcg(uprev + (r - jc)), wi = __ldcg(a.p + (r - jc)) - K * ui;
                v[q] -= ui * wc + wi * uc;
            }
        }
    }
    // rows jc + 2 .. : the part of x below its first entry
    double sq = 0.0;
#pragma unroll
    for (int q = 0; q < COLV; ++q) {
        const int r = jc + t + DT * q;
        if (r >= jc + 2 && r < n) sq += v[q] * v[q];
    }
    __shared__ double head[2];
    if (t == 0) head[0] = v[0];  // A[jc, jc]
    if (t == 1) head[1] = v[0];  // x_0 = A[jc + 1, jc]
    sq = block_sum(sq);          // its barriers also publish head
    const double x0 = head[1];
    double tau = 0.0, bp = x0, scale = 0.0;
    if (sq > 0.0) {
        const double mu = sqrt(x0 * x0 + sq);
        bp = x0 >= 0.0 ? -mu : mu;
        tau = (bp - x0) / bp;
        scale = 1.0 / (x0 - bp);
    }
#pragma unroll
    for (int q = 0; q < COLV; ++q) {
        const int r = jc + t + DT * q;
        if (r < n) cc[r] = r >= jc + 2 ? v[q] * scale : (r == jc + 1 ? 1.0 : v[q]);
    }
    if (t == 0) {
        a.d[jc] = head[0];
        a.e[jc] = bp;
        a.tau[jc] = tau;
    }
}

// Householder tridiagonalisation (step 1).  Cooperative launch, DT threads.
// Everything another block may have written since this kernel began is read
// through L2 (__ldcg): the SMs' L1 caches are not kept coherent.  Step j:
// p = tau A22 u (warp per row) | barrier | A22 -= u w^T + w u^T over (column,
// row chunk) items, block 0 taking the next column whole and building its
// reflector | barrier.
__global__ void __launch_bounds__(DT) k_dn_tridiag(TriArgs a) {
    const int n = a.n;
    double* A = a.A;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gwarp = blockIdx.x * DW + warp, nwarps = gridDim.x * DW;
    __shared__ double wsum[DW];
    if (n >= 3 && blockIdx.x == 0) column_reflector(a, 0, false, 0.0);
    if (!grid_sync(a)) return;
    for (int j = 0; j + 2 < n; ++j) {
        const int m = n - j - 1;
        const double* colj = A + (int64_t)j * n + (j + 1);  // u (u_0 = 1)
        const double tau = __ldcg(a.tau + j);
        // p = tau A22 u, and the block's share of p^T u
        double pu = 0.0;
        for (int r = gwarp; r < m; r += nwarps) {
            const double* cr = A + (int64_t)(j + 1 + r) * n + (j + 1);
            double t[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) t[q] = 0.0;
            int i = lane;
            for (; i + 224 < m; i += 256) {
                double av[8], uv[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    av[q] = __ldcg(cr + i + 32 * q);
                    uv[q] = __ldcg(colj + i + 32 * q);
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) t[q] += av[q] * uv[q];
            }
            for (; i < m; i += 32) t[0] += __ldcg(cr + i) * __ldcg(colj + i);
            const double tt = tau * warp_sum(((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7])));
            if (lane == 0) {
                a.p[r] = tt;
                pu += tt * __ldcg(colj + r);
            }
        }
        if (lane == 0) wsum[warp] = pu;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < DW; ++w) t += wsum[w];
            a.part[blockIdx.x] = t;
        }
        if (!grid_sync(a)) return;
        // A22 -= u w^T + w u^T, w = p - K u, K = (tau / 2) p^T u
        double ptu = 0.0;
        for (int q = 0; q < (int)gridDim.x; ++q) ptu += __ldcg(a.part + q);
        const double K = 0.5 * tau * ptu;
        if (blockIdx.x == 0) {
            if (j + 3 < n) {
                column_reflector(a, j + 1, true, K);  // the next step's column
            } else {  // last step: column j + 1 updated only
                double* cc = A + (int64_t)(j + 1) * n + (j + 1);
                const double uc = __ldcg(colj), wc = __ldcg(a.p) - K * uc;
                for (int i = threadIdx.x; i < m; i += DT) {
                    const double ui = __ldcg(colj + i), wi = __ldcg(a.p + i) - K * ui;
                    cc[i] = __ldcg(cc + i) - (ui * wc + wi * uc);
                }
            }
        }
        // the other columns in (column, 128-row chunk) items, four rows per lane
        const int nch = (m + 127) / 128;
        for (int64_t item = gwarp; item < (int64_t)(m - 1) * nch; item += nwarps) {
            const int c = 1 + (int)(item / nch), ch = (int)(item % nch);
            double* cc = A + (int64_t)(j + 1 + c) * n + (j + 1);
            const double uc = __ldcg(colj + c), wc = __ldcg(a.p + c) - K * uc;
            const int i0 = ch * 128 + lane;
            double v[4], ui[4], wi[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + 32 * q;
                if (i < m) {
                    v[q] = __ldcg(cc + i);
                    ui[q] = __ldcg(colj + i);
                    wi[q] = __ldcg(a.p + i);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + 32 * q;
                if (i < m) cc[i] = v[q] - (ui[q] * wc + (wi[q] - K * ui[q]) * uc);
            }
        }
        if (!grid_sync(a)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (n >= 2) {
            a.d[n - 2] = __ldcg(A + (int64_t)(n - 2) * n + (n - 2));
            a.e[n - 2] = __ldcg(A + (int64_t)(n - 2) * n + (n - 1));
            a.tau[n - 2] = 0.0;
        }
        a.d[n - 1] = __ldcg(A + (int64_t)(n - 1) * n + (n - 1));
        a.tau[n - 1] = 0.0;
    }
}

// Sturm count: eigenvalues of T below x = sign changes along the leading
// principal minors p_i(x) = (d_i - x) p_(i-1) - e_(i-1)^2 p_(i-2), p_0 = 1
// (no division; a zero minor takes the sign opposite to its predecessor, and
// both kept minors are rescaled by 2^-/+500 when the newer one's exponent
// leaves [-500, 500], which changes no sign)
__device__ int sturm_count(int n, const double* __restrict__ d, const double* __restrict__ e2, double x) {
    int cnt = 0;
    double pm = 1.0, pc = d[0] - x;
    if (pc == 0.0) pc = -1e-300;
    cnt += pc < 0.0;
    for (int i = 1; i < n; ++i) {
        double pn = (d[i] - x) * pc - e2[i - 1] * pm;
        if (pn == 0.0) pn = pc < 0.0 ? 1e-300 : -1e-300;
        cnt += (pn < 0.0) != (pc < 0.0);
        const int ex = ((__double2hiint(pn) >> 20) & 0x7ff) - 1023;
        if (ex > 500) {
            pn *= 0x1p-500;
            pc *= 0x1p-500;
        } else if (ex < -500) {
            pn *= 0x1p500;
            pc *= 0x1p500;
        }
        pm = pc;
        pc = pn;
    }
    return cnt;
}

// e2[i] = e[i]^2
__global__ void k_dn_square(int m, const double* __restrict__ e, double* __restrict__ e2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) e2[i] = e[i] * e[i];
}

// Gershgorin interval of T and the pivot floor, by one warp
__device__ void tri_bounds(int n, const double* __restrict__ d, const double* __restrict__ e, double* lo,
                           double* hi, double* pivmin) {
    // (pivmin: the bracket's floor width)
    const int lane = threadIdx.x & 31;
    double l = 1e308, h = -1e308, e2 = 0.0;
    for (int i = lane; i < n; i += 32) {
        const double el = i > 0 ? fabs(e[i - 1]) : 0.0, er = i + 1 < n ? fabs(e[i]) : 0.0;
        l = fmin(l, d[i] - el - er);
        h = fmax(h, d[i] + el + er);
        if (i + 1 < n) e2 = fmax(e2, e[i] * e[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
        h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
        e2 = fmax(e2, __shfl_xor_sync(0xffffffffu, e2, o));
    }
    const double tn = fmax(fabs(l), fabs(h));
    *pivmin = 1e-290 * fmax(1.0, e2);
    *lo = l - 8.0 * DEPS * tn - *pivmin;
    *hi = h + 8.0 * DEPS * tn + *pivmin;
}

// The j-th smallest eigenvalue of T (j = blockIdx.x), warp per eigenvalue:
// 32 points of the bracket per round, the bracket shrinking 33-fold
__global__ void k_dn_bisect(int n, const double* __restrict__ d, const double* __restrict__ e,
                            const double* __restrict__ e2, double* __restrict__ lam) {
    const int j = blockIdx.x, lane = threadIdx.x & 31;
    double lo, hi, pivmin;
    tri_bounds(n, d, e, &lo, &hi, &pivmin);
    for (int round = 0; round < 64; ++round) {
        if (hi - lo <= 2.0 * DEPS * fmax(fabs(lo), fabs(hi)) + pivmin) break;
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const int cnt = sturm_count(n, d, e2, x);
        const unsigned above = __ballot_sync(0xffffffffu, cnt > j);  // points with more than j below
        const double xl = __shfl_sync(0xffffffffu, x, above ? (__ffs(above) - 1) : 31);
        const double xp = __shfl_sync(0xffffffffu, x, above ? (__ffs(above) - 2 < 0 ? 0 : __ffs(above) - 2) : 31);
        if (above == 0u) {
            lo = xl;  // all 32 points hold at most j below: the last point
        } else {
            const int f = __ffs(above) - 1;
            hi = xl;
            if (f > 0) lo = xp;
        }
    }
    if (lane == 0) lam[j] = 0.5 * (lo + hi);
}

// Inverse-iteration shifts and clusters, passed by value
struct InvitParams {
    double shift[32];
    int cluster[32];  // first index of the vector's cluster
    double tiny;      // replacement of a zero pivot
};

// LU factors of T - shift_j I for every vector j (block j, one thread):
// Gaussian elimination with partial pivoting on the tridiagonal (rows i and
// i + 1 swap when |subdiagonal| > |pivot|, which creates a second
// superdiagonal).  Work per vector: 5n doubles -- reciprocal pivots, first
// and second superdiagonals, multipliers, swap flags (as 0 / 1).
__global__ void k_dn_factor(int n, const double* __restrict__ d, const double* __restrict__ e, InvitParams prm,
                            double* __restrict__ work) {
    if (threadIdx.x != 0) return;
    const int j = blockIdx.x;
    double* ra = work + (int64_t)j * 5 * n;  // pivots, then their reciprocals
    double* u1 = ra + n;
    double* u2 = u1 + n;
    double* ml = u2 + n;
    double* sw = ml + n;
    const double lam = prm.shift[j], tiny = prm.tiny;
    double ai = d[0] - lam, ui = n > 1 ? e[0] : 0.0;  // current row's pivot and superdiagonal
    for (int i = 0; i + 1 < n; ++i) {
        const double sub = e[i], an = d[i + 1] - lam, un = i + 2 < n ? e[i + 1] : 0.0;
        if (fabs(sub) > fabs(ai)) {
            // swap: row i becomes (sub, an, un); the old row i is eliminated
            const double mlt = ai / sub;
            ra[i] = sub;
            u1[i] = an;
            u2[i] = un;
            ml[i] = mlt;
            sw[i] = 1.0;
            ai = ui - mlt * an;
            ui = -mlt * un;
        } else {
            if (ai == 0.0) ai = tiny;
            const double mlt = sub / ai;
            ra[i] = ai;
            u1[i] = ui;
            u2[i] = 0.0;
            ml[i] = mlt;
            sw[i] = 0.0;
            ai = an - mlt * ui;
            ui = un;
        }
    }
    ra[n - 1] = ai != 0.0 ? ai : tiny;
    u1[n - 1] = 0.0;
    u2[n - 1] = 0.0;
    for (int i = 0; i < n; ++i) ra[i] = 1.0 / (ra[i] != 0.0 ? ra[i] : tiny);
}

// z_j <- (T - shift_j I)^-1 z_j with the stored factors (block j, one thread)
__global__ void k_dn_invit(int n, const double* __restrict__ work, double* __restrict__ Z) {
    if (threadIdx.x != 0) return;
    const int j = blockIdx.x;
    double* z = Z + (int64_t)j * n;
    const double* ra = work + (int64_t)j * 5 * n;
    const double* u1 = ra + n;
    const double* u2 = u1 + n;
    const double* ml = u2 + n;
    const double* sw = ml + n;
    double zi = z[0];
    for (int i = 0; i + 1 < n; ++i) {
        double zn = z[i + 1];
        if (sw[i] != 0.0) {
            const double t = zi;
            zi = zn;
            zn = t;
        }
        z[i] = zi;
        zi = zn - ml[i] * zi;
    }
    z[n - 1] = zi;
    double z1 = 0.0, z2 = 0.0;  // z[i + 1], z[i + 2]
    for (int i = n - 1; i >= 0; --i) {
        const double v = (z[i] - u1[i] * z1 - u2[i] * z2) * ra[i];
        z[i] = v;
        z2 = z1;
        z1 = v;
    }
}

// Normalise every vector and orthogonalise each against the earlier members
// of its cluster, in order (one block)
__global__ void __launch_bounds__(DT) k_dn_mgs(int n, int k, InvitParams prm, double* __restrict__ Z) {
    for (int j = 0; j < k; ++j) {
        double* zj = Z + (int64_t)j * n;
        for (int q = prm.cluster[j]; q < j; ++q) {
            const double* zq = Z + (int64_t)q * n;
            double t = 0.0;
            for (int i = threadIdx.x; i < n; i += DT) t += zq[i] * zj[i];
            const double dq = block_sum(t);
            for (int i = threadIdx.x; i < n; i += DT) zj[i] -= dq * zq[i];
        }
        double t = 0.0;
        for (int i = threadIdx.x; i < n; i += DT) t += zj[i] * zj[i];
        const double nr = sqrt(block_sum(t));
        const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
        for (int i = threadIdx.x; i < n; i += DT) zj[i] *= inv;
        __syncthreads();
    }
}

// x = Q z (reflectors n-3 ... 0), U[:, j] = S x; block j, z in shared memory
__global__ void __launch_bounds__(DT) k_dn_backtrans(int n, int k, const double* __restrict__ A,
                                                     const double* __restrict__ tau, const double* __restrict__ Z,
                                                     const double* __restrict__ b, double* __restrict__ U) {
    extern __shared__ double zs[];
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += DT) zs[i] = Z[(int64_t)j * n + i];
    __syncthreads();
    for (int r = n - 3; r >= 0; --r) {
        const double t = tau[r];
        if (t == 0.0) continue;  // uniform across the block
        const int m = n - r - 1;
        const double* u = A + (int64_t)r * n + (r + 1);
        double s = 0.0;
        for (int i = threadIdx.x; i < m; i += DT) s += u[i] * zs[r + 1 + i];
        const double dot = block_sum(s) * t;
        for (int i = threadIdx.x; i < m; i += DT) zs[r + 1 + i] -= dot * u[i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += DT) {
        const double sc = b ? 1.0 / sqrt(b[i] > 0.0 ? b[i] : 1.0) : 1.0;
        U[(int64_t)i * k + j] = sc * zs[i];
    }
}

}  // namespace

gr_status dense_eigenpairs(gr_ctx* c, const double* b, int k, Workspace& ws, cudaStream_t s, double* lam_dev,
                           double* lam_host, double* U) {
    const int n = (int)c->n;
    if (k < 1 || k > 32 || n < k || n > DENSE_EIG_MAX) return set_error(c, GR_EINVAL, "eigensolve: dense size");
    size_t need = 0;
    auto add = [&](size_t bytes) {
        const size_t off = need;
        need += (bytes + 255) & ~size_t(255);
        return off;
    };
    const size_t o_A = add(sizeof(double) * (size_t)n * n), o_d = add(sizeof(double) * n),
                 o_e = add(sizeof(double) * n), o_tau = add(sizeof(double) * n), o_p = add(sizeof(double) * n),
                 o_part = add(sizeof(double) * 1024), o_sig = add(64), o_bar = add(512),
                 o_Z = add(sizeof(double) * (size_t)k * n), o_work = add(sizeof(double) * 5 * (size_t)k * n),
                 o_e2 = add(sizeof(double) * n),
                 o_lam = add(sizeof(double) * 32);
    void* base;
    GR_TRY_CUDA(c, ws.get(WS_EIG_WORK, need, &base), "eigensolve: scratch");
    char* Bp = (char*)base;
    double* A = (double*)(Bp + o_A);
    double* d = (double*)(Bp + o_d);
    double* e = (double*)(Bp + o_e);
    double* tau = (double*)(Bp + o_tau);
    double* Z = (double*)(Bp + o_Z);
    double* work = (double*)(Bp + o_work);
    double* lam = (double*)(Bp + o_lam);
    unsigned* bar = (unsigned*)(Bp + o_bar);  // count, generation, abort, error: 128 bytes apart
    GR_TRY_CUDA(c, cudaMemsetAsync(A, 0, sizeof(double) * (size_t)n * n, s), "memset");
    GR_TRY_CUDA(c, cudaMemsetAsync(bar, 0, 512, s), "memset");
    k_dn_build<<<(unsigned)ceil_div(n, DT), DT, 0, s>>>(n, c->rowptr, c->col, c->eid, c->ew, c->deg, b, A);
    count_launch();

    // 1) tridiagonalisation: one cooperative launch, at most one block per SM
    int per_sm = 0;
    GR_TRY_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dn_tridiag, DT, 0), "occupancy");
    // one block per SM at most: the rank-2 update's (column, row chunk) items
    // spread over the SMs; small problems take fewer
    int grid = (int)ceil_div((int64_t)n * ((n + 127) / 128), DW);
    if (grid > c->num_sms) grid = c->num_sms;
    if (grid > per_sm * c->num_sms) grid = per_sm * c->num_sms;
    if (grid > 1024) grid = 1024;
    if (grid < 1) grid = 1;
    TriArgs ta;
    ta.A = A;
    ta.n = n;
    ta.d = d;
    ta.e = e;
    ta.tau = tau;
    ta.p = (double*)(Bp + o_p);
    ta.part = (double*)(Bp + o_part);
    ta.count = bar;
    ta.gen = bar + 32;
    ta.abort = (int*)(bar + 64);
    ta.err = (int*)(bar + 96);
    void* args[] = {&ta};
    GR_TRY_CUDA(c, cudaLaunchCooperativeKernel((void*)k_dn_tridiag, dim3(grid), dim3(DT), args, 0, s),
                "eigensolve: tridiagonalisation");
    count_launch();

    // 2) the k smallest eigenvalues of T
    double* e2 = (double*)(Bp + o_e2);
    k_dn_square<<<(unsigned)ceil_div(n, DT), DT, 0, s>>>(n - 1, e, e2);
    count_launch();
    k_dn_bisect<<<k, 32, 0, s>>>(n, d, e, e2, lam);
    count_launch();
    int herr = 0;
    GR_TRY_CUDA(c, cudaMemcpyAsync(lam_host, lam, sizeof(double) * k, cudaMemcpyDeviceToHost, s), "readback");
    GR_TRY_CUDA(c, cudaMemcpyAsync(&herr, bar + 96, sizeof(int), cudaMemcpyDeviceToHost, s), "readback");
    GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
    if (herr) return set_error(c, GR_ECUDA, "eigensolve: a grid barrier of the tridiagonalisation timed out");

    // 3) inverse iteration: clusters (eigenvalues within 1e-3 ||T|| of the
    // previous one) share a subspace; equal shifts inside a cluster are
    // separated by 10 eps ||T||
    double tn = 0.0;
    {
        std::vector<double> hd(n), he(n > 1 ? n - 1 : 1);
        GR_TRY_CUDA(c, cudaMemcpyAsync(hd.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost, s), "readback");
        if (n > 1)
            GR_TRY_CUDA(c, cudaMemcpyAsync(he.data(), e, sizeof(double) * (n - 1), cudaMemcpyDeviceToHost, s),
                        "readback");
        GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
        for (int i = 0; i < n; ++i) {
            const double el = i > 0 ? fabs(he[i - 1]) : 0.0, er = i + 1 < n ? fabs(he[i]) : 0.0;
            tn = fmax(tn, fabs(hd[i]) + el + er);
        }
    }
    InvitParams prm;
    prm.tiny = DEPS * (tn > 0.0 ? tn : 1.0);
    for (int j = 0; j < k; ++j) {
        prm.shift[j] = lam_host[j];
        prm.cluster[j] = j;
        if (j > 0 && lam_host[j] - lam_host[j - 1] <= 1e-3 * tn) {
            prm.cluster[j] = prm.cluster[j - 1];
            if (prm.shift[j] - prm.shift[j - 1] < 10.0 * prm.tiny) prm.shift[j] = prm.shift[j - 1] + 10.0 * prm.tiny;
        }
    }
    for (int j = k; j < 32; ++j) {
        prm.shift[j] = 0.0;
        prm.cluster[j] = j;
    }
    // start vectors: a smooth deterministic pattern per vector
    {
        std::vector<double> hz((size_t)k * n);
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < n; ++i) hz[(size_t)j * n + i] = cos((0.7 + 0.13 * j) * i) + 0.1;
        GR_TRY_CUDA(c, cudaMemcpyAsync(Z, hz.data(), sizeof(double) * hz.size(), cudaMemcpyHostToDevice, s),
                    "upload");
        GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
    }
    k_dn_mgs<<<1, DT, 0, s>>>(n, k, prm, Z);
    count_launch();
    k_dn_factor<<<k, 32, 0, s>>>(n, d, e, prm, work);
    count_launch();
    for (int it = 0; it < INVIT_STEPS; ++it) {
        k_dn_invit<<<k, 32, 0, s>>>(n, work, Z);
        count_launch();
        k_dn_mgs<<<1, DT, 0, s>>>(n, k, prm, Z);
        count_launch();
    }

    // 4) back to A's basis and to u = S x
    k_dn_backtrans<<<k, DT, sizeof(double) * n, s>>>(n, k, A, tau, Z, b, U);
    count_launch();
    GR_TRY_CUDA(c, cudaMemcpyAsync(lam_dev, lam, sizeof(double) * k, cudaMemcpyDeviceToDevice, s), "copy");
    GR_TRY_CUDA(c, cudaGetLastError(), "eigensolve: dense path");
    return GR_OK;
}

}  // namespace gr
