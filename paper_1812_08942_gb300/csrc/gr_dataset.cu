// Reduced data set F_R = H_G^R F (Alg. 6, step 4) with H_G^R = P^T composed
// over the levels: row A of F_R is the sum (or, on request, the mean) of the
// rows of the fine nodes that end in coarsest aggregate A.  The fine node ids
// are stably sorted by their coarsest label, so each aggregate's members come
// out in ascending id and are added in that order (FP64 accumulation).
#include "gr_internal.cuh"

namespace gr {

namespace {

constexpr int DT = 256;

__global__ void k_label_keys(int64_t n, const int32_t* __restrict__ map, int64_t nc, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ vals, int32_t* __restrict__ cnt, int32_t* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t a = map[i];
    if (a < 0 || a >= nc) {
        atomicExch(bad, 1);
        keys[i] = 0u;
    } else {
        keys[i] = (uint32_t)a;
        atomicAdd(&cnt[a], 1);
    }
    vals[i] = (uint32_t)i;
}

// thread per (aggregate, column)
template <typename T>
__global__ void k_segment_rows(int64_t nc, int d, const int32_t* __restrict__ start, const uint32_t* __restrict__ mem,
                               const T* __restrict__ F, int mean, T* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nc * d) return;
    const int64_t A = idx / d;
    const int j = (int)(idx % d);
    const int32_t b = start[A], e = start[A + 1];
    double s = 0.0;
    for (int32_t t = b; t < e; ++t) s += (double)F[(int64_t)mem[t] * d + j];
    if (mean && e > b) s = s / (double)(e - b);
    out[idx] = (T)s;
}

}  // namespace

gr_status reduce_data_impl(gr_ctx* const* levels, int nlevels, const void* F, int d, int f64, int mean,
                           void* F_out) {
    gr_ctx* c0 = levels[0];
    cudaStream_t s = c0->stream;
    const int64_t n = c0->parent_n, nc = levels[nlevels - 1]->n;
    size_t need = 0;
    auto add = [&](size_t bytes) {
        size_t off = need;
        need += (bytes + 255) & ~size_t(255);
        return off;
    };
    const size_t o_map = add(4 * (size_t)n), o_k0 = add(4 * (size_t)n), o_v0 = add(4 * (size_t)n),
                 o_k1 = add(4 * (size_t)n), o_v1 = add(4 * (size_t)n), o_cnt = add(4 * (size_t)(nc + 1)),
                 o_start = add(4 * (size_t)(nc + 1)), o_bad = add(16);
    void* base;
    GR_TRY_CUDA(c0, c0->ws.get(WS_DATASET, need, &base), "reduce_data scratch");
    char* B = (char*)base;
    int32_t* map = (int32_t*)(B + o_map);
    uint32_t* k0 = (uint32_t*)(B + o_k0);
    uint32_t* v0 = (uint32_t*)(B + o_v0);
    uint32_t* k1 = (uint32_t*)(B + o_k1);
    uint32_t* v1 = (uint32_t*)(B + o_v1);
    int32_t* cnt = (int32_t*)(B + o_cnt);
    int32_t* start = (int32_t*)(B + o_start);
    int32_t* bad = (int32_t*)(B + o_bad);

    gr_status st = compose_impl(levels, nlevels, map);
    if (st != GR_OK) return st;
    GR_TRY_CUDA(c0, cudaMemsetAsync(cnt, 0, 4 * (size_t)(nc + 1), s), "memset");
    GR_TRY_CUDA(c0, cudaMemsetAsync(bad, 0, 4, s), "memset");
    if (n > 0) {
        k_label_keys<<<(unsigned)ceil_div(n, DT), DT, 0, s>>>(n, map, nc, k0, v0, cnt, bad);
        count_launch();
    }
    int alt = 0;
    GR_TRY_CUDA(c0, radix_sort_u32(k0, v0, k1, v1, n, bits_for((uint64_t)(nc > 1 ? nc - 1 : 1)), c0->ws, s, &alt),
                "sort by label");
    const uint32_t* mem = alt ? v1 : v0;
    GR_TRY_CUDA(c0, scan_exclusive_i32(cnt, start, nc + 1, c0->ws, s), "scan");
    if (nc > 0 && d > 0) {
        if (f64) {
            k_segment_rows<double><<<(unsigned)ceil_div(nc * d, DT), DT, 0, s>>>(nc, d, start, mem, (const double*)F,
                                                                               mean, (double*)F_out);
        } else {
            k_segment_rows<float><<<(unsigned)ceil_div(nc * d, DT), DT, 0, s>>>(nc, d, start, mem, (const float*)F,
                                                                              mean, (float*)F_out);
        }
        count_launch();
    }
    GR_TRY_CUDA(c0, cudaGetLastError(), "reduce_data kernels");
    int64_t* hs = host_scratch();
    if (!hs) return set_error(c0, GR_ENOMEM, "reduce_data: pinned scratch unavailable");
    GR_TRY_CUDA(c0, cudaMemcpyAsync(hs, bad, 4, cudaMemcpyDeviceToHost, s), "readback");
    GR_TRY_CUDA(c0, cudaStreamSynchronize(s), "sync");
    if (((int32_t*)hs)[0]) return set_error(c0, GR_ECUDA, "reduce_data: composed map out of range");
    return GR_OK;
}

}  // namespace gr
