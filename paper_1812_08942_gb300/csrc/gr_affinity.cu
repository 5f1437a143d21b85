// Per-edge spectral affinity (Eq. eqn:agg) and algebraic distance d = 1 - a
// (Sec. 3.2.2).  d is evaluated without cancellation:
//   1 - a = (1 - cos)(1 + cos) = (|h_p - h_q|^2 / 2)(|h_p + h_q|^2 / 2),
//   h = X_row / |X_row|.
// One thread per canonical edge; both rows are read whole (16-byte chunks).
#include <cuda_bf16.h>

#include "gr_internal.cuh"
#include "gr_vec.cuh"

namespace gr {

constexpr int AF_THREADS = 256;

template <typename T, int K>
__device__ __forceinline__ void load_row(const T* __restrict__ X, int64_t row,
                                         typename AccOf<T>::type (&x)[K]) {
    using L = RowLayout<T, K>;
#pragma unroll
    for (int q = 0; q < L::G; ++q) {
        typename AccOf<T>::type c[L::E];
        load_chunk<T, L::E>(X + row * K + q * L::E, c);
#pragma unroll
        for (int e = 0; e < L::E; ++e) x[q * L::E + e] = c[e];
    }
}

// FP32 arithmetic (FP32 and BF16 storage)
template <typename T, int K>
__global__ void __launch_bounds__(AF_THREADS) k_affinity_f32(
    int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
    const T* __restrict__ X, float* __restrict__ d_out, float* __restrict__ a_out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int64_t p = eu[e], q = ev[e];
    float xp[K], xq[K];
    load_row<T, K>(X, p, xp);
    load_row<T, K>(X, q, xq);
    float np = 0.f, nq = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        np = fmaf(xp[k], xp[k], np);
        nq = fmaf(xq[k], xq[k], nq);
        c = fmaf(xp[k], xq[k], c);
    }
    float d, a;
    if (np == 0.f || nq == 0.f) {
        d = 1.f;
        a = 0.f;
    } else {
        const float ip = rsqrtf(np), iq = rsqrtf(nq);
        float dm = 0.f, dp = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float hp = xp[k] * ip, hq = xq[k] * iq;
            float s = hp - hq, t = hp + hq;
            dm = fmaf(s, s, dm);
            dp = fmaf(t, t, dp);
        }
        d = 0.25f * dm * dp;
        a = (c * c) / (np * nq);
    }
    d_out[e] = d;
    if (a_out) a_out[e] = a;
}

// FP64, every operation rounded once in the order of the plain definition
// (no contraction), so identical inputs give identical outputs.
template <int K>
__global__ void __launch_bounds__(AF_THREADS) k_affinity_f64(
    int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
    const double* __restrict__ X, double* __restrict__ d_out, double* __restrict__ a_out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int64_t p = eu[e], q = ev[e];
    double xp[K], xq[K];
    load_row<double, K>(X, p, xp);
    load_row<double, K>(X, q, xq);
    double c = 0.0, np = 0.0, nq = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        c = __dadd_rn(c, __dmul_rn(xp[k], xq[k]));
        np = __dadd_rn(np, __dmul_rn(xp[k], xp[k]));
        nq = __dadd_rn(nq, __dmul_rn(xq[k], xq[k]));
    }
    double d, a;
    if (np == 0.0 || nq == 0.0) {
        a = 0.0;
        d = 1.0;
    } else {
        a = __ddiv_rn(__dmul_rn(c, c), __dmul_rn(np, nq));
        const double rp = __dsqrt_rn(np), rq = __dsqrt_rn(nq);
        double dm = 0.0, dp = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double hp = __ddiv_rn(xp[k], rp), hq = __ddiv_rn(xq[k], rq);
            double s = __dsub_rn(hp, hq), t = __dadd_rn(hp, hq);
            dm = __dadd_rn(dm, __dmul_rn(s, s));
            dp = __dadd_rn(dp, __dmul_rn(t, t));
        }
        d = __dmul_rn(__dmul_rn(0.25, dm), dp);
    }
    d_out[e] = d;
    if (a_out) a_out[e] = a;
}

template <int K>
static cudaError_t affinity_k(gr_ctx* c, const void* X, gr_prec prec, void* d, void* a) {
    const int64_t m = c->m;
    if (m == 0) return cudaSuccess;
    const unsigned grid = (unsigned)ceil_div(m, AF_THREADS);
    switch (prec) {
        case GR_F64:
            k_affinity_f64<K><<<grid, AF_THREADS, 0, c->stream>>>(m, c->eu, c->ev, (const double*)X,
                                                                  (double*)d, (double*)a); count_launch();
            break;
        case GR_F32:
            k_affinity_f32<float, K><<<grid, AF_THREADS, 0, c->stream>>>(
                m, c->eu, c->ev, (const float*)X, (float*)d, (float*)a); count_launch();
            break;
        case GR_BF16:
            k_affinity_f32<__nv_bfloat16, K><<<grid, AF_THREADS, 0, c->stream>>>(
                m, c->eu, c->ev, (const __nv_bfloat16*)X, (float*)d, (float*)a); count_launch();
            break;
    }
    return cudaGetLastError();
}

gr_status affinity_impl(gr_ctx* c, const void* X, int K, gr_prec prec, void* d, void* a) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (K) {
        case 4: e = affinity_k<4>(c, X, prec, d, a); break;
        case 8: e = affinity_k<8>(c, X, prec, d, a); break;
        case 16: e = affinity_k<16>(c, X, prec, d, a); break;
        case 24: e = affinity_k<24>(c, X, prec, d, a); break;
        case 32: e = affinity_k<32>(c, X, prec, d, a); break;
    }
    if (e != cudaSuccess) return cuda_error(c, e, "affinity");
    return GR_OK;
}

}  // namespace gr
