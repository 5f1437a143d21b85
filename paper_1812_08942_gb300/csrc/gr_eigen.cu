// Multilevel Laplacian eigensolver (Alg. 5, Sec. 4.1; Eqs. equ:lgl, equ:lgs).
//
// Coarsest level: the first k eigenpairs of L u = lambda B u (B = I ratio
// cut, B = D normalised cut, each level's own; or the Galerkin-consistent
// mass B_l = P^T B_(l-1) P carried from the finest I or D) from a
// Chebyshev-filtered subspace iteration on the coarsest graph
// (gr_chfsi.cu).  Then, level by level toward the finest: U_fine = P U_coarse (the parent map), and `iters` weighted-Jacobi
// iterations on (L - lambda_k B) y = 0 for every column k, the shift being the
// coarsest eigenvalue.  Finally modified Gram-Schmidt over the columns.  Every
// reduction is FP64 with a fixed summation order (per-block partials, then a
// last-block finish), so results are reproducible.
#include <vector>

#include "gr_internal.cuh"

namespace gr {

namespace {

constexpr int ET = 256;

// U_fine[i, :] = U_coarse[map[i], :]  (H = P, Alg. 5 step 5)
__global__ void k_prolong(int64_t n, int k, const int32_t* __restrict__ map, const double* __restrict__ Uc,
                          double* __restrict__ Uf) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t i = idx / k;
    const int c = (int)(idx % k);
    Uf[idx] = Uc[(int64_t)map[i] * k + c];
}

// Weighted-Jacobi iteration on (L - lambda_c B) y = 0 for every column c:
//   y <- (1 - w) y + w (A y)_r / (D_r - lambda_c B_r),
// with (A y)_r = D_r (D^-1 A y)_r from the row-scaled weights and B the
// diagonal mass b (NULL: B = I); a row whose shifted diagonal is not positive
// keeps its value.  The gain g_rc = w D_r / (D_r - lambda_c B_r) depends only
// on the level, so it is computed once per level (g = -1: the row keeps its
// value; otherwise g >= 0) and an iteration is
//   y <- (1 - w) y + g (D^-1 A y)_r:
// FP64 runs at a small fraction of the FP32 rate on this part, and the
// division, taken per entry and iteration, cost more than the row's
// products.  The keep test reads the sign bit of g with an integer compare
// (a floating compare would take the FP64 pipe too).
__global__ void k_shift_gain(int64_t n, int k, const double* __restrict__ deg, const double* __restrict__ lam,
                             const double* __restrict__ b, double omega, double* __restrict__ g) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t r = idx / k;
    const int c = (int)(idx % k);
    const double D = deg[r];
    const double diag = D - lam[c] * (b ? b[r] : 1.0);
    g[idx] = diag > 0.0 ? omega * D / diag : -1.0;
}

// One iteration, thread per (row, column).
__global__ void k_shifted_jacobi(int64_t n, int k, const int64_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ col, const double* __restrict__ wn64,
                                 const double* __restrict__ gain, double omega, const double* __restrict__ Yin,
                                 double* __restrict__ Yout) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int64_t r = idx / k;
    const int c = (int)(idx % k);
    const double y = Yin[idx];
    const double g = gain[idx];
    if (__double2hiint(g) < 0) {
        Yout[idx] = y;
        return;
    }
    double s = 0.0;
    for (int64_t j = rowptr[r]; j < rowptr[r + 1]; ++j) s += wn64[j] * Yin[(int64_t)col[j] * k + c];
    Yout[idx] = fma(g, s, (1.0 - omega) * y);
}

// The same iteration with G lanes per row, each holding one 16-byte chunk
// (two columns) of the row: the slot entries are read once per lane group and
// each neighbour row is gathered chunk-wise; rows in grid-stride order.
template <int K>
__global__ void __launch_bounds__(ET) k_shifted_jacobi_rows(int64_t n64, const int64_t* __restrict__ rowptr,
                                                           const int32_t* __restrict__ col,
                                                           const double* __restrict__ wn64,
                                                           const double* __restrict__ gain, double omega,
                                                           const double* __restrict__ Yin,
                                                           double* __restrict__ Yout) {
    constexpr int E = K >= 2 ? 2 : 1, G = K / E, RPW = 32 / G;
    const int64_t n = n64;
    const int lane = threadIdx.x & 31, seg = lane / G, q = lane % G;
    if (seg >= RPW) return;
    const int64_t stride = (((int64_t)gridDim.x * blockDim.x) >> 5) * RPW;
    for (int64_t r = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW + seg; r < n; r += stride) {
        double acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.0;
        const int64_t j1 = rowptr[r + 1];
        // two neighbour chunks in flight per step
        for (int64_t j = rowptr[r]; j < j1; j += 2) {
            const bool two = j + 1 < j1;
            const double w0 = wn64[j], w1 = two ? wn64[j + 1] : 0.0;
            const double* s0 = Yin + (int64_t)col[j] * K + q * E;
            const double* s1 = Yin + (int64_t)col[two ? j + 1 : j] * K + q * E;
            if constexpr (E == 2) {
                const double2 x0 = __ldg(reinterpret_cast<const double2*>(s0));
                const double2 x1 = __ldg(reinterpret_cast<const double2*>(s1));
                acc[0] = fma(w0, x0.x, acc[0]);
                acc[1] = fma(w0, x0.y, acc[1]);
                if (two) {
                    acc[0] = fma(w1, x1.x, acc[0]);
                    acc[1] = fma(w1, x1.y, acc[1]);
                }
            } else {
                const double x0 = __ldg(s0), x1 = __ldg(s1);
                acc[0] = fma(w0, x0, acc[0]);
                if (two) acc[0] = fma(w1, x1, acc[0]);
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int c = q * E + e;
            const double y = Yin[r * K + c];
            const double g = gain[r * K + c];
            Yout[r * K + c] = __double2hiint(g) >= 0 ? fma(g, acc[e], (1.0 - omega) * y) : y;
        }
    }
}

// finest-level mass: 1 (ratio cut) or the degree, 1 for a degree-0 node
__global__ void k_base_mass(int64_t n, const double* __restrict__ deg, int normalized, double* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = normalized ? (deg[i] > 0.0 ? deg[i] : 1.0) : 1.0;
}

// row-major n x k <-> column-major
__global__ void k_to_colmajor(int64_t n, int k, const double* __restrict__ U, double* __restrict__ V) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    V[(idx % k) * n + idx / k] = U[idx];
}
__global__ void k_to_rowmajor(int64_t n, int k, const double* __restrict__ V, double* __restrict__ U) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    U[idx] = V[(idx % k) * n + idx / k];
}

// Sum of one double per thread over the block, in a fixed order.
__device__ __forceinline__ double block_sum(double s, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < ET / 32; ++w) t += red[w];
    __syncthreads();
    return t;  // valid in thread 0
}

// Per-block partial of a grid reduction; the last block to arrive adds the
// partials (thread t takes blocks t, t + ET, ... in order, then block_sum).
__device__ __forceinline__ void grid_finish(double s, double* __restrict__ part, unsigned* __restrict__ counter,
                                            double* __restrict__ out) {
    __shared__ double red[ET / 32];
    __shared__ bool last;
    const double t = block_sum(s, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double a = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += ET) a += __ldcg(part + b);
        const double total = block_sum(a, red);
        if (threadIdx.x == 0) {
            *out = total;
            *counter = 0u;
        }
    }
}

// out = a . b over n entries: per-block partials, the last block to finish
// adds them in block order (one atomic ticket, no wait)
__global__ void __launch_bounds__(ET) k_dot(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                                            double* __restrict__ part, unsigned* __restrict__ counter,
                                            double* __restrict__ out) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    grid_finish(s, part, counter, out);
}

// y -= r x  (r = *rp)
__global__ void k_axpy(int64_t n, const double* __restrict__ rp, const double* __restrict__ x,
                       double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] -= (*rp) * x[i];
}

// y /= sqrt(*nrm2)
__global__ void k_unit(int64_t n, const double* __restrict__ nrm2, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] /= sqrt(*nrm2);
}

// per-edge sum over the canonical list of w (x_u - x_v)^2 for column x (= x' L x),
// with the same block-partial / last-block finish
__global__ void __launch_bounds__(ET) k_edge_quad(int64_t m, const int32_t* __restrict__ eu,
                                                  const int32_t* __restrict__ ev, const double* __restrict__ ew,
                                                  const double* __restrict__ x, double* __restrict__ part,
                                                  unsigned* __restrict__ counter, double* __restrict__ out) {
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const double d = x[eu[e]] - x[ev[e]];
        s += ew[e] * d * d;
    }
    grid_finish(s, part, counter, out);
}

// x' B x for B = D (x' x for B = I uses k_dot)
__global__ void k_scale_by(int64_t n, const double* __restrict__ x, const double* __restrict__ deg,
                           double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i] * deg[i];
}

}  // namespace

gr_status eigensolve_impl(gr_ctx* const* levels, int nlevels, int k, int normalized, int galerkin_mass,
                          double omega, int iters, double* U_out, double* lambda_out, double* rayleigh_out) {
    gr_ctx* f = levels[0];
    gr_ctx* c = levels[nlevels - 1];
    cudaStream_t s = f->stream;
    const int64_t n0 = f->n;
    auto blocks = [](int64_t work) { return (unsigned)ceil_div(work > 0 ? work : 1, ET); };

    // scratch: two n x k blocks at the finest size, column-major copy,
    // reduction partials, scalars
    int64_t nmax = 0;
    for (int l = 0; l < nlevels; ++l) nmax = levels[l]->n > nmax ? levels[l]->n : nmax;
    const int RB = f->num_sms * 4;  // reduction blocks
    size_t need = 0;
    auto add = [&](size_t bytes) {
        size_t off = need;
        need += (bytes + 255) & ~size_t(255);
        return off;
    };
    const size_t o_Y0 = add(sizeof(double) * (size_t)nmax * k), o_Y1 = add(sizeof(double) * (size_t)nmax * k),
                 o_G = add(sizeof(double) * (size_t)nmax * k),
                 o_V = add(sizeof(double) * (size_t)n0 * k), o_T = add(sizeof(double) * (size_t)n0),
                 o_part = add(sizeof(double) * (size_t)RB), o_sc = add(sizeof(double) * 64),
                 o_lam = add(sizeof(double) * 32), o_ctr = add(64);
    // Galerkin masses of every level: b_0 = 1 or D (degree 0 -> 1), then the
    // member sums level by level
    std::vector<size_t> o_mass;
    if (galerkin_mass)
        for (int l = 0; l < nlevels; ++l) o_mass.push_back(add(sizeof(double) * (size_t)(levels[l]->n > 0 ? levels[l]->n : 1)));
    void* base;
    GR_TRY_CUDA(f, f->ws.get(WS_EIG, need, &base), "eigensolver scratch");
    char* Bp = (char*)base;
    double* Y[2] = {(double*)(Bp + o_Y0), (double*)(Bp + o_Y1)};
    double* gain = (double*)(Bp + o_G);
    double* V = (double*)(Bp + o_V);
    double* T = (double*)(Bp + o_T);
    double* part = (double*)(Bp + o_part);
    double* sc = (double*)(Bp + o_sc);
    double* lam = (double*)(Bp + o_lam);
    unsigned* ctr = (unsigned*)(Bp + o_ctr);
    GR_TRY_CUDA(f, cudaMemsetAsync(ctr, 0, 64, s), "memset");
    // the diagonal mass of each level (NULL: B = I)
    std::vector<const double*> mass(nlevels, nullptr);
    if (galerkin_mass) {
        double* b0 = (double*)(Bp + o_mass[0]);
        k_base_mass<<<blocks(n0), ET, 0, s>>>(n0, f->deg, normalized, b0);
        count_launch();
        mass[0] = b0;
        for (int l = 1; l < nlevels; ++l) {
            double* bl = (double*)(Bp + o_mass[l]);
            gr_ctx* const one[1] = {levels[l]};
            const gr_status st = reduce_data_impl(one, 1, mass[l - 1], 1, 1, 0, bl);
            if (st != GR_OK) return set_error(f, st, "eigensolve: Galerkin mass: " + levels[l]->last_error);
            mass[l] = bl;
        }
    } else if (normalized) {
        for (int l = 0; l < nlevels; ++l) mass[l] = levels[l]->deg;
    }

    // 1) coarsest eigenpairs (Alg. 5 step 2, Eq. equ:lgs)
    int cur = 0;
    {
        const gr_status st = coarsest_eigenpairs(c, mass[nlevels - 1], k, f->ws, s, lam, lambda_out, Y[cur], nullptr);
        if (st != GR_OK) return set_error(f, st, c->last_error);
    }

    // 2) map and smooth, level by level (Alg. 5 steps 4-10)
    for (int l = nlevels - 2; l >= 0; --l) {
        gr_ctx* g = levels[l];
        const int64_t n = g->n;
        k_prolong<<<blocks(n * k), ET, 0, s>>>(n, k, levels[l + 1]->parent_map, Y[cur], Y[cur ^ 1]);
        count_launch();
        cur ^= 1;
        if (iters > 0) {
            k_shift_gain<<<blocks(n * k), ET, 0, s>>>(n, k, g->deg, lam, mass[l], omega, gain);
            count_launch();
        }
        for (int it = 0; it < iters; ++it) {
            const unsigned gr = (unsigned)(f->num_sms * 8);
#define GR_SJ_ROWS(KK)                                                                                    \
    k_shifted_jacobi_rows<KK><<<gr, ET, 0, s>>>(n, g->rowptr, g->col, g->wn64, gain, omega, Y[cur], Y[cur ^ 1])
            switch (k) {
                case 2: GR_SJ_ROWS(2); break;
                case 4: GR_SJ_ROWS(4); break;
                case 8: GR_SJ_ROWS(8); break;
                case 16: GR_SJ_ROWS(16); break;
                case 32: GR_SJ_ROWS(32); break;
                default:
                    k_shifted_jacobi<<<blocks(n * k), ET, 0, s>>>(n, k, g->rowptr, g->col, g->wn64, gain, omega,
                                                                Y[cur], Y[cur ^ 1]);
            }
#undef GR_SJ_ROWS
            count_launch();
            cur ^= 1;
        }
    }

    // 3) modified Gram-Schmidt over the columns (Alg. 5 step 11)
    k_to_colmajor<<<blocks(n0 * k), ET, 0, s>>>(n0, k, Y[cur], V);
    count_launch();
    const unsigned rb = (unsigned)(RB < ceil_div(n0, ET) ? RB : ceil_div(n0 > 0 ? n0 : 1, ET));
    for (int i = 0; i < k; ++i) {
        double* ui = V + (int64_t)i * n0;
        for (int j = 0; j < i; ++j) {
            const double* uj = V + (int64_t)j * n0;
            k_dot<<<rb, ET, 0, s>>>(n0, uj, ui, part, ctr, sc);
            count_launch();
            k_axpy<<<blocks(n0), ET, 0, s>>>(n0, sc, uj, ui);
            count_launch();
        }
        k_dot<<<rb, ET, 0, s>>>(n0, ui, ui, part, ctr, sc);
        count_launch();
        k_unit<<<blocks(n0), ET, 0, s>>>(n0, sc, ui);
        count_launch();
    }
    k_to_rowmajor<<<blocks(n0 * k), ET, 0, s>>>(n0, k, V, U_out);
    count_launch();

    // 4) Rayleigh quotients of the result, x' L x / x' B x
    if (rayleigh_out) {
        const unsigned rbm = (unsigned)(RB < ceil_div(f->m, ET) ? RB : ceil_div(f->m > 0 ? f->m : 1, ET));
        for (int i = 0; i < k; ++i) {
            const double* ui = V + (int64_t)i * n0;
            if (f->m > 0) {
                k_edge_quad<<<rbm, ET, 0, s>>>(f->m, f->eu, f->ev, f->ew, ui, part, ctr, sc + 2 * i);
                count_launch();
            } else {
                GR_TRY_CUDA(f, cudaMemsetAsync(sc + 2 * i, 0, sizeof(double), s), "memset");
            }
            const double* bu = ui;
            if (normalized) {
                k_scale_by<<<blocks(n0), ET, 0, s>>>(n0, ui, f->deg, T);
                count_launch();
                bu = T;
            }
            k_dot<<<rb, ET, 0, s>>>(n0, ui, bu, part, ctr, sc + 2 * i + 1);
            count_launch();
        }
        int64_t* hs = host_scratch();
        if (!hs) return set_error(f, GR_ENOMEM, "eigensolve: pinned scratch unavailable");
        double* hq = (double*)hs;  // 64 B: up to 4 pairs at a time
        for (int i0 = 0; i0 < k; i0 += 4) {
            const int cnt = k - i0 < 4 ? k - i0 : 4;
            GR_TRY_CUDA(f, cudaMemcpyAsync(hq, sc + 2 * i0, sizeof(double) * 2 * cnt, cudaMemcpyDeviceToHost, s),
                        "readback");
            GR_TRY_CUDA(f, cudaStreamSynchronize(s), "sync");
            for (int t = 0; t < cnt; ++t) rayleigh_out[i0 + t] = hq[2 * t] / hq[2 * t + 1];
        }
    }
    GR_TRY_CUDA(f, cudaGetLastError(), "eigensolve kernels");
    GR_TRY_CUDA(f, cudaStreamSynchronize(s), "sync");
    return GR_OK;
}

}  // namespace gr
