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

// A row of a block not yet normalised, normalised in registers as the
// normalising pass of the smoothing would store it: (x - mu) * (1/s) in the
// accumulator type, then rounded to the storage type.
// The statistics are read 16 bytes at a time (K is a multiple of 4).
template <typename T, int K>
__device__ __forceinline__ void normalise_row(typename AccOf<T>::type (&x)[K],
                                              const typename AccOf<T>::type* __restrict__ st) {
    using Acc = typename AccOf<T>::type;
    constexpr int V = 16 / (int)sizeof(Acc);  // statistics per 16-byte load
    static_assert(K % V == 0, "K is a multiple of 4");
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += V) {
        Acc mu[V], is[V];
        if constexpr (V == 4) {
            const float4 a = *reinterpret_cast<const float4*>(st + k0);
            const float4 b = *reinterpret_cast<const float4*>(st + K + k0);
            mu[0] = a.x; mu[1] = a.y; mu[2] = a.z; mu[3] = a.w;
            is[0] = b.x; is[1] = b.y; is[2] = b.z; is[3] = b.w;
        } else {
            const double2 a = *reinterpret_cast<const double2*>(st + k0);
            const double2 b = *reinterpret_cast<const double2*>(st + K + k0);
            mu[0] = a.x; mu[1] = a.y;
            is[0] = b.x; is[1] = b.y;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const Acc y = (x[k0 + v] - mu[v]) * is[v];
            if constexpr (sizeof(T) == 2) x[k0 + v] = __bfloat162float(__float2bfloat16_rn(y));
            else x[k0 + v] = y;
        }
    }
}

// the statistics into shared memory (NORM: the block still needs them)
template <typename Acc, int K, bool NORM>
__device__ __forceinline__ void load_stats(Acc* st, const double* __restrict__ stats) {
    if constexpr (NORM) {
        for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) st[i] = (Acc)stats[i];
        __syncthreads();
    }
}

// FP32 arithmetic (FP32 and BF16 storage)
template <typename T, int K, bool NORM>
__global__ void __launch_bounds__(AF_THREADS) k_affinity_f32(
    int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
    const T* __restrict__ X, const double* __restrict__ stats, float* __restrict__ d_out,
    float* __restrict__ a_out) {
    __shared__ __align__(16) float st[NORM ? 2 * K : 4];
    load_stats<float, K, NORM>(st, stats);
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int64_t p = eu[e], q = ev[e];
    float xp[K], xq[K];
    load_row<T, K>(X, p, xp);
    load_row<T, K>(X, q, xq);
    if constexpr (NORM) {
        normalise_row<T, K>(xp, st);
        normalise_row<T, K>(xq, st);
    }
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
template <int K, bool NORM>
__global__ void __launch_bounds__(AF_THREADS) k_affinity_f64(
    int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
    const double* __restrict__ X, const double* __restrict__ stats, double* __restrict__ d_out,
    double* __restrict__ a_out) {
    __shared__ __align__(16) double st[NORM ? 2 * K : 2];
    load_stats<double, K, NORM>(st, stats);
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int64_t p = eu[e], q = ev[e];
    double xp[K], xq[K];
    load_row<double, K>(X, p, xp);
    load_row<double, K>(X, q, xq);
    if constexpr (NORM) {
        normalise_row<double, K>(xp, st);
        normalise_row<double, K>(xq, st);
    }
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

template <int K, bool NORM>
static cudaError_t affinity_k(gr_ctx* c, const void* X, const double* stats, gr_prec prec, void* d, void* a) {
    const int64_t m = c->m;
    if (m == 0) return cudaSuccess;
    const unsigned grid = (unsigned)ceil_div(m, AF_THREADS);
    switch (prec) {
        case GR_F64:
            k_affinity_f64<K, NORM><<<grid, AF_THREADS, 0, c->stream>>>(m, c->eu, c->ev, (const double*)X, stats,
                                                                        (double*)d, (double*)a); count_launch();
            break;
        case GR_F32:
            k_affinity_f32<float, K, NORM><<<grid, AF_THREADS, 0, c->stream>>>(
                m, c->eu, c->ev, (const float*)X, stats, (float*)d, (float*)a); count_launch();
            break;
        case GR_BF16:
            k_affinity_f32<__nv_bfloat16, K, NORM><<<grid, AF_THREADS, 0, c->stream>>>(
                m, c->eu, c->ev, (const __nv_bfloat16*)X, stats, (float*)d, (float*)a); count_launch();
            break;
    }
    return cudaGetLastError();
}

template <int K>
static cudaError_t affinity_k(gr_ctx* c, const void* X, const double* stats, gr_prec prec, void* d, void* a) {
    return stats ? affinity_k<K, true>(c, X, stats, prec, d, a) : affinity_k<K, false>(c, X, stats, prec, d, a);
}

gr_status affinity_impl(gr_ctx* c, const void* X, int K, gr_prec prec, void* d, void* a, const double* stats) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (K) {
        case 4: e = affinity_k<4>(c, X, stats, prec, d, a); break;
        case 8: e = affinity_k<8>(c, X, stats, prec, d, a); break;
        case 16: e = affinity_k<16>(c, X, stats, prec, d, a); break;
        case 24: e = affinity_k<24>(c, X, stats, prec, d, a); break;
        case 32: e = affinity_k<32>(c, X, stats, prec, d, a); break;
    }
    if (e != cudaSuccess) return cuda_error(c, e, "affinity");
    return GR_OK;
}

}  // namespace gr
