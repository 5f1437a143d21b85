// Row-chunk access to row-major n x K vector blocks of double, float or
// bfloat16.  A row is split into G chunks of E elements; one lane owns one
// chunk and moves it with a single 16-byte (or 8-byte) access.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace gr {

template <typename T>
struct AccOf { using type = float; };
template <>
struct AccOf<double> { using type = double; };

constexpr int next_pow2_c(int x) { return x <= 1 ? 1 : 2 * next_pow2_c((x + 1) / 2); }

template <typename T, int K>
struct RowLayout {
    static constexpr int RB = K * (int)sizeof(T);           // row bytes
    static constexpr int CB = (RB % 16 == 0) ? 16 : 8;       // chunk bytes
    static constexpr int E = CB / (int)sizeof(T);            // elements per chunk
    static constexpr int G = K / E;                          // chunks per row
    static constexpr int GP = next_pow2_c(G);                // lanes reserved per row
    static_assert(RB % 8 == 0, "row must be a multiple of 8 bytes");
    static_assert(G <= 32, "row too wide");
};

template <typename T, int E>
__device__ __forceinline__ void load_chunk(const T* __restrict__ p, typename AccOf<T>::type (&x)[E]);

template <>
__device__ __forceinline__ void load_chunk<float, 4>(const float* __restrict__ p, float (&x)[4]) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
template <>
__device__ __forceinline__ void load_chunk<float, 2>(const float* __restrict__ p, float (&x)[2]) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    x[0] = v.x; x[1] = v.y;
}
template <>
__device__ __forceinline__ void load_chunk<double, 2>(const double* __restrict__ p, double (&x)[2]) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    x[0] = v.x; x[1] = v.y;
}
template <>
__device__ __forceinline__ void load_chunk<double, 1>(const double* __restrict__ p, double (&x)[1]) {
    x[0] = __ldg(p);
}
template <>
__device__ __forceinline__ void load_chunk<__nv_bfloat16, 8>(const __nv_bfloat16* __restrict__ p,
                                                            float (&x)[8]) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 f = __bfloat1622float2(h[i]);
        x[2 * i] = f.x;
        x[2 * i + 1] = f.y;
    }
}
template <>
__device__ __forceinline__ void load_chunk<__nv_bfloat16, 4>(const __nv_bfloat16* __restrict__ p,
                                                            float (&x)[4]) {
    uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float2 f = __bfloat1622float2(h[i]);
        x[2 * i] = f.x;
        x[2 * i + 1] = f.y;
    }
}

// Round to storage, store, and hand back the stored value in the accumulator
// type (so statistics describe exactly what the next sweep reads).
template <typename T, int E>
__device__ __forceinline__ void store_chunk(T* __restrict__ p, typename AccOf<T>::type (&x)[E]);

template <>
__device__ __forceinline__ void store_chunk<float, 4>(float* __restrict__ p, float (&x)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
template <>
__device__ __forceinline__ void store_chunk<float, 2>(float* __restrict__ p, float (&x)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
}
template <>
__device__ __forceinline__ void store_chunk<double, 2>(double* __restrict__ p, double (&x)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
}
template <>
__device__ __forceinline__ void store_chunk<double, 1>(double* __restrict__ p, double (&x)[1]) {
    *p = x[0];
}
template <>
__device__ __forceinline__ void store_chunk<__nv_bfloat16, 8>(__nv_bfloat16* __restrict__ p,
                                                             float (&x)[8]) {
    uint4 v;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
        float2 f = __bfloat1622float2(h[i]);
        x[2 * i] = f.x;
        x[2 * i + 1] = f.y;
    }
    *reinterpret_cast<uint4*>(p) = v;
}
template <>
__device__ __forceinline__ void store_chunk<__nv_bfloat16, 4>(__nv_bfloat16* __restrict__ p,
                                                             float (&x)[4]) {
    uint2 v;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        h[i] = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
        float2 f = __bfloat1622float2(h[i]);
        x[2 * i] = f.x;
        x[2 * i + 1] = f.y;
    }
    *reinterpret_cast<uint2*>(p) = v;
}

}  // namespace gr
