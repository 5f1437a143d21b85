// Spectral-mismatch loss on a reduced graph with free edge weights w_c, and
// its hand-written adjoint (reverse sweeps).  Not in the paper: it turns the
// edge-weight sensitivity of Sec. 3.3.3 (d lambda / d w = -lambda (e^T u)^2)
// into the exact gradient of a smooth objective built from the weighted
// Jacobi filter of Alg. 3 on the reduced graph.
//
//   R_f[k]  = x_k^T L_G x_k / x_k^T x_k
//   y_0     = M^-1 P^T X                            (aggregate means)
//   y_{s+1} = (1-w) y_s + w D_c^-1 A_c y_s          (isolated node: unchanged)
//   R_c[k]  = y^T L_c y / sum_A M_A (y_A - mu_k)^2,  mu_k = sum M y / sum M
//   loss    = (1/K) sum_k (R_c[k]/R_f[k] - 1)^2
// Vectors are FP32; every global sum is reduced in FP64 in a fixed order.
#include "gr_internal.cuh"

namespace gr {

constexpr int LS_THREADS = 256;

__global__ void k_i32_to_i64_n(const int32_t* a, int64_t n, int64_t* b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
    else if (i == n) b[i] = 0;
}

// one block: FP64 sum of n floats in a fixed order
__global__ void k_sum_f32(const float* a, int64_t n, double* out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)a[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < (int)blockDim.x; ++j) t += sh[j];
        *out = t;
    }
}


// Reduce K per-thread FP32 values over the block; write an FP64 partial.
template <int K>
__device__ void block_colsum(float (&v)[K], double* __restrict__ part) {
    __shared__ double ws[LS_THREADS / 32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) ws[warp][k] = (double)x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int w = 0; w < LS_THREADS / 32; ++w) s += ws[w][threadIdx.x];
        part[(int64_t)blockIdx.x * K + threadIdx.x] = s;
    }
}

// out[j] = sum over blocks of part[b*NS + j]
__global__ void k_finish_sums(const double* __restrict__ part, int nblocks, int NS,
                              double* __restrict__ out) {
    int j = threadIdx.x;
    if (j >= NS) return;
    // eight interleaved accumulators keep eight loads in flight (fixed order)
    double a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = 0.0;
    int b = 0;
    for (; b + 7 < nblocks; b += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] += part[(int64_t)(b + u) * NS + j];
    }
    for (; b < nblocks; ++b) a[0] += part[(int64_t)b * NS + j];
    out[j] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// sum_e w_e (x_u - x_v)^2 per column, over a canonical edge list
template <int K>
__global__ void __launch_bounds__(LS_THREADS) k_edge_quad(int64_t m, const int32_t* __restrict__ eu,
                                                          const int32_t* __restrict__ ev,
                                                          const double* __restrict__ w64,
                                                          const float* __restrict__ w32,
                                                          const float* __restrict__ X,
                                                          double* __restrict__ part) {
    float v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = eu[e], b = ev[e];
        const float w = w64 ? (float)w64[e] : w32[e];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float t = X[a * K + k] - X[b * K + k];
            v[k] = fmaf(w * t, t, v[k]);
        }
    }
    block_colsum<K>(v, part);
}

// sum_i mass_i * (x_i - mu)^2 per column (mass NULL: 1, mu NULL: 0)
template <int K>
__global__ void __launch_bounds__(LS_THREADS) k_row_quad(int64_t n, const float* __restrict__ X,
                                                         const float* __restrict__ mass,
                                                         const double* __restrict__ mu,
                                                         double* __restrict__ part) {
    float v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float mi = mass ? mass[i] : 1.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float t = X[i * K + k] - (mu ? (float)mu[k] : 0.f);
            v[k] = fmaf(mi * t, t, v[k]);
        }
    }
    block_colsum<K>(v, part);
}

// sum_i mass_i x_i per column
template <int K>
__global__ void __launch_bounds__(LS_THREADS) k_row_sum(int64_t n, const float* __restrict__ X,
                                                        const float* __restrict__ mass,
                                                        double* __restrict__ part) {
    float v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float mi = mass[i];
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = fmaf(mi, X[i * K + k], v[k]);
    }
    block_colsum<K>(v, part);
}

__global__ void k_agg_keys(int64_t n, const int32_t* __restrict__ agg, int64_t nc,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                           int32_t* __restrict__ cnt, int32_t* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = agg[i];
    if (a < 0 || a >= nc) {
        atomicExch(bad, 1);
        a = 0;
    }
    keys[i] = (uint32_t)a;
    vals[i] = (uint32_t)i;
    atomicAdd(&cnt[a], 1);
}

// y0[A] = mean of the member rows (members in ascending fine id), M_A = size
template <int K>
__global__ void k_aggregate_means(int64_t nc, const int64_t* __restrict__ start,
                                  const int32_t* __restrict__ cnt, const uint32_t* __restrict__ members,
                                  const float* __restrict__ X, float* __restrict__ y0,
                                  float* __restrict__ mass) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nc * K) return;
    int64_t A = idx / K;
    int k = (int)(idx % K);
    int64_t b = start[A];
    int32_t c = cnt[A];
    float s = 0.f;
    for (int32_t t = 0; t < c; ++t) s += X[(int64_t)members[b + t] * K + k];
    y0[idx] = c > 0 ? s / (float)c : 0.f;
    if (k == 0) mass[A] = (float)c;
}

// D_c[A] = sum of the parameter weights on A's row (warp per row, fixed order)
__global__ void k_param_degree(int64_t n, const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ eid, const float* __restrict__ w,
                               float* __restrict__ D) {
    const int lane = threadIdx.x & 31;
    int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= n) return;
    float s = 0.f;
    for (int64_t j = rowptr[p] + lane; j < rowptr[p + 1]; j += 32) s += w[eid[j]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) D[p] = s;
}

// forward sweep: z = D^-1 A y (or y when isolated), y1 = (1-w) y + w z
template <int K>
__global__ void k_param_sweep(int64_t n, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ col, const int32_t* __restrict__ eid,
                              const float* __restrict__ w, const float* __restrict__ D,
                              const float* __restrict__ y, float omega, float* __restrict__ z_out,
                              float* __restrict__ y1) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * K) return;
    int64_t A = idx / K;
    int k = (int)(idx % K);
    float s = 0.f;
    for (int64_t j = rowptr[A]; j < rowptr[A + 1]; ++j) s = fmaf(w[eid[j]], y[(int64_t)col[j] * K + k], s);
    float z = D[A] > 0.f ? s / D[A] : y[idx];
    if (z_out) z_out[idx] = z;
    y1[idx] = (1.f - omega) * y[idx] + omega * z;
}

// adjoint sweep: yb_s = (1-w) yb + w A D^-1 yb   (isolated: yb_s = yb)
template <int K>
__global__ void k_param_sweep_adj(int64_t n, const int64_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ col, const int32_t* __restrict__ eid,
                                  const float* __restrict__ w, const float* __restrict__ D,
                                  const float* __restrict__ yb, float omega,
                                  float* __restrict__ yb_out) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * K) return;
    int64_t A = idx / K;
    int k = (int)(idx % K);
    if (!(D[A] > 0.f)) {
        yb_out[idx] = yb[idx];
        return;
    }
    float s = 0.f;
    for (int64_t j = rowptr[A]; j < rowptr[A + 1]; ++j) {
        int64_t B = col[j];
        s = fmaf(w[eid[j]], yb[B * K + k] / D[B], s);
    }
    yb_out[idx] = (1.f - omega) * yb[idx] + omega * s;
}

// scalars: mu, Q, N, R_c, gRc from the FP64 sums
__global__ void k_loss_scalars(int K, const double* __restrict__ Nsum, const double* __restrict__ Qsum,
                               const float* __restrict__ Rf, const float* __restrict__ grad_loss,
                               float* __restrict__ loss_out, float* __restrict__ gRc,
                               float* __restrict__ Qf, float* __restrict__ Nf) {
    if (threadIdx.x != 0) return;
    double loss = 0.0;
    const double g = grad_loss ? (double)*grad_loss : 1.0;
    for (int k = 0; k < K; ++k) {
        double Rc = Nsum[k] / Qsum[k];
        double r = Rc / (double)Rf[k] - 1.0;
        loss += r * r;
        if (gRc) gRc[k] = (float)(g * 2.0 * r / (double)Rf[k] / (double)K);
        if (Qf) Qf[k] = (float)Qsum[k];
        if (Nf) Nf[k] = (float)Nsum[k];
    }
    if (loss_out) *loss_out = (float)(loss / (double)K);
}

__global__ void k_rf(int K, const double* __restrict__ num, const double* __restrict__ den,
                     float* __restrict__ Rf) {
    int k = threadIdx.x;
    if (k < K) Rf[k] = (float)(num[k] / den[k]);
}

__global__ void k_mu(int K, const double* __restrict__ s, const double* __restrict__ msum,
                     double* __restrict__ mu) {
    int k = threadIdx.x;
    if (k < K) mu[k] = s[k] / *msum;
}

// ybar_S = gRc (2 L y / Q - 2 N M (y - mu) / Q^2)
template <int K>
__global__ void k_adj_final(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ eid, const float* __restrict__ w,
                            const float* __restrict__ y, const float* __restrict__ mass,
                            const double* __restrict__ mu, const float* __restrict__ Q,
                            const float* __restrict__ N, const float* __restrict__ gRc,
                            float* __restrict__ yb) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * K) return;
    int64_t A = idx / K;
    int k = (int)(idx % K);
    const float ya = y[idx];
    float ly = 0.f;
    for (int64_t j = rowptr[A]; j < rowptr[A + 1]; ++j) ly = fmaf(w[eid[j]], ya - y[(int64_t)col[j] * K + k], ly);
    const float q = Q[k];
    yb[idx] = gRc[k] * (2.f * ly / q - 2.f * N[k] * mass[A] * (ya - (float)mu[k]) / (q * q));
}

// per coarse edge: direct term + sum over sweeps of the weight adjoint
template <int K>
__global__ void k_edge_grad(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                            int S, int64_t nK, const float* __restrict__ Y, const float* __restrict__ Z,
                            const float* __restrict__ YB, const float* __restrict__ D, float omega,
                            const float* __restrict__ Q, const float* __restrict__ gRc,
                            float* __restrict__ grad) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int64_t A = eu[e], B = ev[e];
    const float* yS = Y + (int64_t)S * nK;
    float g = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float t = yS[A * K + k] - yS[B * K + k];
        g = fmaf(gRc[k] * t / Q[k], t, g);
    }
    const float iDA = 1.f / D[A], iDB = 1.f / D[B];
    for (int s = 0; s < S; ++s) {
        const float* y = Y + (int64_t)s * nK;
        const float* z = Z + (int64_t)s * nK;
        const float* yb = YB + (int64_t)(s + 1) * nK;
        float ga = 0.f, gb = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            ga = fmaf(yb[A * K + k], y[B * K + k] - z[A * K + k], ga);
            gb = fmaf(yb[B * K + k], y[A * K + k] - z[B * K + k], gb);
        }
        g += omega * (ga * iDA + gb * iDB);
    }
    grad[e] = g;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int red_grid(const gr_ctx* c) { return c->num_sms > 0 ? 2 * c->num_sms : 64; }

template <int K>
static cudaError_t coarse_rc_parts(gr_ctx* cc, const float* y, const float* w_c, const float* mass,
                                   const double* msum, double* part, double* Nsum, double* musum,
                                   double* mu, double* Qsum) {
    cudaStream_t s = cc->stream;
    const int rg = red_grid(cc);
    // N: sum over reduced edges with the parameter weights
    k_edge_quad<K><<<rg, LS_THREADS, 0, s>>>(cc->m, cc->eu, cc->ev, nullptr, w_c, y, part); count_launch();
    k_finish_sums<<<1, 64, 0, s>>>(part, rg, K, Nsum); count_launch();
    k_row_sum<K><<<rg, LS_THREADS, 0, s>>>(cc->n, y, mass, part); count_launch();
    k_finish_sums<<<1, 64, 0, s>>>(part, rg, K, musum); count_launch();
    k_mu<<<1, 64, 0, s>>>(K, musum, msum, mu); count_launch();
    k_row_quad<K><<<rg, LS_THREADS, 0, s>>>(cc->n, y, mass, mu, part); count_launch();
    k_finish_sums<<<1, 64, 0, s>>>(part, rg, K, Qsum); count_launch();
    return cudaGetLastError();
}

template <int K>
static gr_status loss_fwd_k(gr_ctx* f, gr_ctx* cc, const int32_t* agg, const float* X,
                            const float* w_c, int S, double omega, float* loss, float* saved) {
    cudaStream_t s = f->stream;
    const int64_t n = f->n, nc = cc->n;
    const int rg = red_grid(f);
    float* y0 = saved;
    float* Rf = saved + nc * K;
    float* mass = Rf + K;
    // scratch on the coarse context
    void *pa, *pb, *pc;
    GR_TRY_CUDA(cc, cc->ws.get(WS_LOSS_A, sizeof(double) * (size_t)(rg * K + 8 * K) + 256, &pa), "ws");
    double* part = (double*)pa;
    double* Nsum = part + rg * K;
    double* den = Nsum + K;
    double* musum = den + K;
    double* mu = musum + K;
    double* Qsum = mu + K;
    GR_TRY_CUDA(cc, cc->ws.get(WS_LOSS_B, sizeof(float) * (size_t)nc * K * 2 + sizeof(float) * nc + 256, &pb), "ws");
    float* ya = (float*)pb;
    float* yb = ya + nc * K;
    float* D = yb + nc * K;
    // fine Rayleigh quotients
    k_edge_quad<K><<<rg, LS_THREADS, 0, s>>>(f->m, f->eu, f->ev, f->ew, nullptr, X, part); count_launch();
    k_finish_sums<<<1, 64, 0, s>>>(part, rg, K, Nsum); count_launch();
    k_row_quad<K><<<rg, LS_THREADS, 0, s>>>(n, X, nullptr, nullptr, part); count_launch();
    k_finish_sums<<<1, 64, 0, s>>>(part, rg, K, den); count_launch();
    k_rf<<<1, 64, 0, s>>>(K, Nsum, den, Rf); count_launch();
    // aggregate means: stable sort of fine ids by label
    GR_TRY_CUDA(cc, cc->ws.get(WS_LOSS_C, sizeof(uint32_t) * (size_t)n * 4 + sizeof(int64_t) * (nc + 1) * 2 +
                                              sizeof(int32_t) * (nc + 2) + 1024, &pc), "ws");
    uint32_t* k0 = (uint32_t*)pc;
    uint32_t* v0 = k0 + n;
    uint32_t* k1 = v0 + n;
    uint32_t* v1 = k1 + n;
    int64_t* cnt64 = (int64_t*)(v1 + n + (n & 1));
    int64_t* start = cnt64 + (nc + 1);
    int32_t* cnt = (int32_t*)(start + (nc + 1));
    int32_t* bad = cnt + nc;
    GR_TRY_CUDA(cc, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)(nc + 1), s), "memset");
    k_agg_keys<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(n, agg, nc, k0, v0, cnt, bad); count_launch();
    int alt = 0;
    GR_TRY_CUDA(cc, radix_sort_u32(k0, v0, k1, v1, n, bits_for((uint64_t)(nc - 1)), cc->ws, s, &alt), "sort");
    const uint32_t* members = alt ? v1 : v0;
    k_i32_to_i64_n<<<(unsigned)ceil_div(nc + 1, 256), 256, 0, s>>>(cnt, nc, cnt64); count_launch();
    GR_TRY_CUDA(cc, scan_exclusive_i64(cnt64, start, nc + 1, cc->ws, s), "scan");
    k_aggregate_means<K><<<(unsigned)ceil_div(nc * K, 256), 256, 0, s>>>(nc, start, cnt, members, X, y0, mass); count_launch();
    // sweeps on the reduced graph with the parameter weights
    k_param_degree<<<(unsigned)ceil_div(nc * 32, 256), 256, 0, s>>>(nc, cc->rowptr, cc->eid, w_c, D); count_launch();
    const float* y = y0;
    for (int it = 0; it < S; ++it) {
        float* out = (it & 1) ? yb : ya;
        k_param_sweep<K><<<(unsigned)ceil_div(nc * K, 256), 256, 0, s>>>(nc, cc->rowptr, cc->col, cc->eid, w_c,
                                                                         D, y, (float)omega, nullptr, out); count_launch();
        y = out;
    }
    k_sum_f32<<<1, 256, 0, s>>>(mass, nc, den); count_launch();
    GR_TRY_CUDA(cc, coarse_rc_parts<K>(cc, y, w_c, mass, den, part, Nsum, musum, mu, Qsum), "rc");
    k_loss_scalars<<<1, 32, 0, s>>>(K, Nsum, Qsum, Rf, nullptr, loss, nullptr, nullptr, nullptr); count_launch();
    GR_TRY_CUDA(cc, cudaGetLastError(), "loss fwd");
    // label check
    int32_t hbad = 0;
    GR_TRY_CUDA(cc, cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "copy");
    GR_TRY_CUDA(cc, cudaStreamSynchronize(s), "sync");
    if (hbad) return set_error(f, GR_EINVAL, "loss_fwd: agg labels must lie in [0, coarse n)");
    return GR_OK;
}

template <int K>
static gr_status loss_bwd_k(gr_ctx* cc, const float* saved, const float* w_c, int S, double omega,
                            const float* grad_loss, float* grad) {
    cudaStream_t s = cc->stream;
    const int64_t nc = cc->n;
    const int64_t nK = nc * K;
    const float* y0 = saved;
    const float* Rf = saved + nK;
    const float* mass = Rf + K;
    const int rg = red_grid(cc);
    void *pa, *pb;
    GR_TRY_CUDA(cc, cc->ws.get(WS_LOSS_A, sizeof(double) * (size_t)(rg * K + 8 * K) + 256, &pa), "ws");
    double* part = (double*)pa;
    double* Nsum = part + rg * K;
    double* den = Nsum + K;
    double* musum = den + K;
    double* mu = musum + K;
    double* Qsum = mu + K;
    // Y[0..S], Z[0..S-1], YB[0..S], D, gRc, Q, N
    size_t floats = (size_t)nK * (3 * S + 2) + nc + 4 * K + 64;
    GR_TRY_CUDA(cc, cc->ws.get(WS_LOSS_B, sizeof(float) * floats, &pb), "ws");
    float* Y = (float*)pb;
    float* Z = Y + (size_t)(S + 1) * nK;
    float* YB = Z + (size_t)(S > 0 ? S : 0) * nK;
    float* D = YB + (size_t)(S + 1) * nK;
    float* gRc = D + nc;
    float* Qf = gRc + K;
    float* Nf = Qf + K;
    GR_TRY_CUDA(cc, cudaMemcpyAsync(Y, y0, sizeof(float) * nK, cudaMemcpyDeviceToDevice, s), "copy");
    k_param_degree<<<(unsigned)ceil_div(nc * 32, 256), 256, 0, s>>>(nc, cc->rowptr, cc->eid, w_c, D); count_launch();
    for (int it = 0; it < S; ++it) {
        k_param_sweep<K><<<(unsigned)ceil_div(nK, 256), 256, 0, s>>>(nc, cc->rowptr, cc->col, cc->eid, w_c, D,
                                                                     Y + it * nK, (float)omega, Z + it * nK,
                                                                     Y + (it + 1) * nK);
        count_launch();
    }
    k_sum_f32<<<1, 256, 0, s>>>(mass, nc, den); count_launch();  // total mass, FP64
    const float* yS = Y + (size_t)S * nK;
    GR_TRY_CUDA(cc, coarse_rc_parts<K>(cc, yS, w_c, mass, den, part, Nsum, musum, mu, Qsum), "rc");
    k_loss_scalars<<<1, 32, 0, s>>>(K, Nsum, Qsum, Rf, grad_loss, nullptr, gRc, Qf, Nf); count_launch();
    k_adj_final<K><<<(unsigned)ceil_div(nK, 256), 256, 0, s>>>(nc, cc->rowptr, cc->col, cc->eid, w_c, yS, mass,
                                                               mu, Qf, Nf, gRc, YB + (size_t)S * nK); count_launch();
    for (int it = S - 1; it >= 0; --it) {
        k_param_sweep_adj<K><<<(unsigned)ceil_div(nK, 256), 256, 0, s>>>(
            nc, cc->rowptr, cc->col, cc->eid, w_c, D, YB + (size_t)(it + 1) * nK, (float)omega, YB + (size_t)it * nK);
        count_launch();
    }
    if (cc->m > 0) {
        k_edge_grad<K><<<(unsigned)ceil_div(cc->m, 256), 256, 0, s>>>(cc->m, cc->eu, cc->ev, S, nK, Y, Z, YB, D,
                                                                      (float)omega, Qf, gRc, grad);
        count_launch();
    }
    GR_TRY_CUDA(cc, cudaGetLastError(), "loss bwd");
    return GR_OK;
}

gr_status loss_fwd_impl(gr_ctx* fine, gr_ctx* coarse, const int32_t* agg, const float* X, int K,
                        const float* w_c, int sweeps, double omega, float* loss, float* saved) {
    switch (K) {
        case 4: return loss_fwd_k<4>(fine, coarse, agg, X, w_c, sweeps, omega, loss, saved);
        case 8: return loss_fwd_k<8>(fine, coarse, agg, X, w_c, sweeps, omega, loss, saved);
        case 16: return loss_fwd_k<16>(fine, coarse, agg, X, w_c, sweeps, omega, loss, saved);
        case 24: return loss_fwd_k<24>(fine, coarse, agg, X, w_c, sweeps, omega, loss, saved);
        case 32: return loss_fwd_k<32>(fine, coarse, agg, X, w_c, sweeps, omega, loss, saved);
    }
    return set_error(fine, GR_EINVAL, "loss_fwd: K must be 4, 8, 16, 24 or 32");
}

gr_status loss_bwd_impl(gr_ctx* coarse, const float* saved, int K, const float* w_c, int sweeps,
                        double omega, const float* grad_loss, float* grad_w) {
    switch (K) {
        case 4: return loss_bwd_k<4>(coarse, saved, w_c, sweeps, omega, grad_loss, grad_w);
        case 8: return loss_bwd_k<8>(coarse, saved, w_c, sweeps, omega, grad_loss, grad_w);
        case 16: return loss_bwd_k<16>(coarse, saved, w_c, sweeps, omega, grad_loss, grad_w);
        case 24: return loss_bwd_k<24>(coarse, saved, w_c, sweeps, omega, grad_loss, grad_w);
        case 32: return loss_bwd_k<32>(coarse, saved, w_c, sweeps, omega, grad_loss, grad_w);
    }
    return set_error(coarse, GR_EINVAL, "loss_bwd: K must be 4, 8, 16, 24 or 32");
}

}  // namespace gr
