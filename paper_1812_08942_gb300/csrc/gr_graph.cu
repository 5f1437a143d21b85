// Graph construction: the symmetric CSR of A_G and the degrees D_G (Sec. 2.1),
// and Galerkin coarsening L_R = P^T L_G P (Sec. 3.2.2): row by row in shared
// memory (gr_galerkin.cu), or by a global sort + segmented sum when a coarse
// row is too long for that.
#include "gr_internal.cuh"

namespace gr {

constexpr int TB = 256;

// ---------------------------------------------------------------------------
// CSR construction from a canonical edge list
// ---------------------------------------------------------------------------
// eptr[p] = first edge with u >= p (u is sorted), for p in [0, n]
__global__ void k_upper_ptr(const int32_t* __restrict__ eu, int64_t m, int64_t n,
                            int64_t* __restrict__ eptr) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > m) return;
    int64_t prev = e == 0 ? -1 : (int64_t)eu[e - 1];
    int64_t cur = e == m ? n : (int64_t)eu[e];
    for (int64_t p = prev + 1; p <= cur; ++p) eptr[p] = e;
}

// rowcnt[p] = lower count + upper count (entry n is 0); lc64 = lower count as int64
__global__ void k_row_count(const int32_t* __restrict__ lcnt, const int64_t* __restrict__ eptr,
                            int64_t n, int64_t* __restrict__ rowcnt, int64_t* __restrict__ lc64) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) {
        rowcnt[p] = (int64_t)lcnt[p] + (eptr[p + 1] - eptr[p]);
        lc64[p] = lcnt[p];
    } else if (p == n) {
        rowcnt[p] = 0;
        lc64[p] = 0;
    }
}

__global__ void k_keys_from_v(const int32_t* __restrict__ ev, int64_t m, uint32_t* __restrict__ keys,
                              uint32_t* __restrict__ vals) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) {
        keys[e] = (uint32_t)ev[e];
        vals[e] = (uint32_t)e;
    }
}

// lower part of row p: edges (q, p), q < p, in ascending q (= ascending id);
// position t of the stable sort by v holds the t-th such edge overall.
__global__ void k_fill_lower(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sval,
                             int64_t m, const int64_t* __restrict__ lstart,
                             const int64_t* __restrict__ rowptr, const int32_t* __restrict__ eu,
                             const double* __restrict__ ew, int32_t* __restrict__ col,
                             int32_t* __restrict__ eid, double* __restrict__ wslot) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int64_t p = skey[t];
    int64_t e = sval[t];
    int64_t slot = rowptr[p] + (t - lstart[p]);
    col[slot] = eu[e];
    eid[slot] = (int32_t)e;
    wslot[slot] = ew[e];
}

// upper part of row p: edges (p, v), v > p, after the lower part
__global__ void k_fill_upper(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                             const double* __restrict__ ew, int64_t m,
                             const int64_t* __restrict__ eptr, const int32_t* __restrict__ lcnt,
                             const int64_t* __restrict__ rowptr, int32_t* __restrict__ col,
                             int32_t* __restrict__ eid, double* __restrict__ wslot) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    int64_t p = eu[e];
    int64_t slot = rowptr[p] + lcnt[p] + (e - eptr[p]);
    col[slot] = ev[e];
    eid[slot] = (int32_t)e;
    wslot[slot] = ew[e];
}

// warp per row: D(p,p) = sum of the row's weights (fixed shuffle-tree order),
// then the row-scaled weights w / D(p,p) that D^-1 A uses.
__global__ void k_degree_scale(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               int64_t n, double* __restrict__ wn64, int2* __restrict__ cw32,
                               double* __restrict__ deg) {
    const int lane = threadIdx.x & 31;
    int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= n) return;
    int64_t b = rowptr[p], e = rowptr[p + 1];
    double s = 0.0;
    for (int64_t j = b + lane; j < e; j += 32) s += wn64[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) deg[p] = s;
    double inv = s > 0.0 ? 1.0 / s : 0.0;
    for (int64_t j = b + lane; j < e; j += 32) {
        double x = wn64[j] * inv;
        wn64[j] = x;
        cw32[j] = make_int2(col[j], __float_as_int((float)x));
    }
}

// thread per row (short rows): D(p,p) summed sequentially in slot order,
// which is ascending edge id -- the plain definition's order.  A warp's 32
// rows are consecutive: when their slots fit the warp's shared-memory buffer
// the warp reads the weights and columns in whole lines, each thread sums and
// scales its row there, and the warp writes both slot arrays in whole lines.
constexpr int DS_CAP = 512;  // slots a warp stages

__global__ void __launch_bounds__(TB, 4) k_degree_scale_rows(const int64_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col, int64_t n,
                                                          double* __restrict__ wn64, int2* __restrict__ cw32,
                                                          double* __restrict__ deg) {
    __shared__ double s_w[TB / 32][DS_CAP];
    __shared__ int32_t s_c[TB / 32][DS_CAP];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t pw = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    if (pw >= n) return;  // whole warp
    const int64_t p = pw + lane;
    const int lv = (int)((n - pw < 32 ? n - pw : 32) - 1);
    const int64_t R0 = rowptr[pw], R1 = rowptr[pw + lv + 1];
    if (R1 - R0 <= DS_CAP) {
        double* W = s_w[wp];
        int32_t* C = s_c[wp];
        const int ns = (int)(R1 - R0);
        for (int j = lane; j < ns; j += 32) {
            W[j] = wn64[R0 + j];
            C[j] = col[R0 + j];
        }
        __syncwarp();
        if (p < n) {
            const int b = (int)(rowptr[p] - R0), e = (int)(rowptr[p + 1] - R0);
            double s = 0.0;
            for (int j = b; j < e; ++j) s += W[j];
            deg[p] = s;
            const double inv = s > 0.0 ? 1.0 / s : 0.0;
            for (int j = b; j < e; ++j) W[j] = W[j] * inv;
        }
        __syncwarp();
        for (int j = lane; j < ns; j += 32) {
            const double x = W[j];
            wn64[R0 + j] = x;
            cw32[R0 + j] = make_int2(C[j], __float_as_int((float)x));
        }
        return;
    }
    if (p >= n) return;
    const int64_t b = rowptr[p], e = rowptr[p + 1];
    double s = 0.0;
    for (int64_t j = b; j < e; ++j) s += wn64[j];
    deg[p] = s;
    const double inv = s > 0.0 ? 1.0 / s : 0.0;
    for (int64_t j = b; j < e; ++j) {
        const double x = wn64[j] * inv;
        wn64[j] = x;
        cw32[j] = make_int2(col[j], __float_as_int((float)x));
    }
}

// ---------------------------------------------------------------------------
// CSR of a sparse graph by lower-part sorting.  The upper part of row p
// (edges (p, v), v > p) is a contiguous, sorted run of the canonical list; the
// lower part (edges (q, p), q < p) is gathered by atomic slot claims and then
// sorted per row by edge id, which for a fixed p is ascending q.  One pass per
// row then writes both parts, the degree and the row-scaled weights.
// ---------------------------------------------------------------------------
constexpr int LOWER_THREAD = 32;   // lower parts up to this long: sorted by the row's own thread
constexpr int LOWER_WARP = 2048;   // up to this long: by a warp in shared memory; longer: global sort
constexpr int FW = 4;              // warps per block of the warp kernel

// per edge: canonical-input check (when asked) and the lower count of v;
// the block maximum of the counts reached goes to lmax
__global__ void k_csr_count(int64_t n, int64_t m, const int32_t* __restrict__ u, const int32_t* __restrict__ v,
                            const double* __restrict__ w, int check, int32_t* __restrict__ lcnt,
                            int32_t* __restrict__ bad, int32_t* __restrict__ lmax) {
    __shared__ int32_t bmax;
    if (threadIdx.x == 0) bmax = 0;
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) {
        const int32_t a = u[e], b = v[e];
        if (check) {
            bool ok = a >= 0 && b < n && a < b && w[e] > 0.0 && isfinite(w[e]);
            if (e > 0) {
                const int32_t pa = u[e - 1], pb = v[e - 1];
                ok = ok && (pa < a || (pa == a && pb < b));
            }
            if (!ok) atomicExch(bad, 1);
        }
        if (b >= 0 && b < n) atomicMax(&bmax, atomicAdd(&lcnt[b], 1) + 1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && bmax) atomicMax(lmax, bmax);
}

__global__ void k_row_total(const int32_t* __restrict__ lcnt, const int64_t* __restrict__ eptr, int64_t n,
                            int64_t* __restrict__ rowcnt) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) rowcnt[p] = (int64_t)lcnt[p] + (eptr[p + 1] - eptr[p]);
    else if (p == n) rowcnt[p] = 0;
}

// lower part of row v: edge ids in claim order (sorted by the row pass)
__global__ void k_lower_claim(const int32_t* __restrict__ ev, int64_t m, const int64_t* __restrict__ rowptr,
                              int32_t* __restrict__ lfill, int32_t* __restrict__ eid) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t b = ev[e];
    eid[rowptr[b] + atomicAdd(&lfill[b], 1)] = (int32_t)e;
}

// thread per row (graphs of mean degree below 32): insertion-sort the lower ids, write
// the row, D(p,p) summed sequentially in slot order (= ascending edge id),
// then w / D(p,p).  Rows with longer lower parts go to the warp kernel's list.
//
// A warp's 32 rows are consecutive, so their slots and their upper edges are
// two contiguous ranges.  When both fit the warp's shared-memory buffers (and
// no row of the warp is listed), the warp reads the claimed lower ids and the
// upper edges' ends and weights in whole lines, each thread builds its row in
// the buffers, and the warp writes the four slot arrays in whole lines; only
// the lower edges' own ends and weights are gathered.  Other warps write each
// row from its thread (the same values in the same order).
constexpr int FIN_CAP = 256;   // slots a warp stages
constexpr int FIN_ECAP = 160;  // upper edges a warp stages

__global__ void __launch_bounds__(TB, 4) k_row_finish_thread(int64_t n, const int64_t* __restrict__ rowptr,
                                                          const int64_t* __restrict__ eptr,
                                                          const int32_t* __restrict__ lcnt,
                                                          const int32_t* __restrict__ eu,
                                                          const int32_t* __restrict__ ev,
                                                          const double* __restrict__ ew, int32_t* __restrict__ col,
                                                          int32_t* __restrict__ eid, double* __restrict__ wn64,
                                                          int2* __restrict__ cw32, double* __restrict__ deg,
                                                          int32_t* __restrict__ list, int32_t* __restrict__ nlist) {
    __shared__ int32_t s_col[TB / 32][FIN_CAP];
    __shared__ int32_t s_eid[TB / 32][FIN_CAP];
    __shared__ double s_w[TB / 32][FIN_CAP];
    __shared__ int32_t s_ev[TB / 32][FIN_ECAP];
    __shared__ double s_ew[TB / 32][FIN_ECAP];
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t pw = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);  // the warp's first row
    if (pw >= n) return;                                                       // whole warp
    const int64_t p = pw + lane;
    const bool in = p < n;
    const int L = in ? lcnt[p] : 0;
    const bool listed = L > LOWER_THREAD;
    const int32_t k = warp_slot(listed, nlist);
    if (k >= 0) list[k] = (int32_t)p;
    int64_t r0 = 0, e0 = 0, e1 = 0;
    if (in) {
        r0 = rowptr[p];
        e0 = eptr[p];
        e1 = eptr[p + 1];
    }
    const int lv = (int)((n - pw < 32 ? n - pw : 32) - 1);  // the warp's last row
    const int64_t R0 = __shfl_sync(FULL, r0, 0), E0 = __shfl_sync(FULL, e0, 0);
    const int64_t E1 = __shfl_sync(FULL, e1, lv);
    const int64_t R1 = __shfl_sync(FULL, r0 + L + (e1 - e0), lv);
    const bool staged = !__any_sync(FULL, listed) && R1 - R0 <= FIN_CAP && E1 - E0 <= FIN_ECAP;
    if (staged) {
        int32_t* S_col = s_col[wp];
        int32_t* S_eid = s_eid[wp];
        double* S_w = s_w[wp];
        int32_t* S_ev = s_ev[wp];
        double* S_ew = s_ew[wp];
        const int ns = (int)(R1 - R0), ne = (int)(E1 - E0);
        for (int j = lane; j < ns; j += 32) S_eid[j] = eid[R0 + j];  // lower parts: ids in claim order
        for (int j = lane; j < ne; j += 32) {
            S_ev[j] = ev[E0 + j];
            S_ew[j] = ew[E0 + j];
        }
        __syncwarp();
        if (in) {
            const int b = (int)(r0 - R0), u0 = (int)(e0 - E0), U = (int)(e1 - e0);
            for (int i = 1; i < L; ++i) {
                const int32_t x = S_eid[b + i];
                int j = i;
                while (j > 0 && S_eid[b + j - 1] > x) {
                    S_eid[b + j] = S_eid[b + j - 1];
                    --j;
                }
                S_eid[b + j] = x;
            }
            double sum = 0.0;
            for (int i0 = 0; i0 < L; i0 += 4) {  // four lower edges' ends and weights in flight
                int32_t e4[4], c4[4];
                double w4[4];
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (i0 + t < L) {
                        e4[t] = S_eid[b + i0 + t];
                        w4[t] = ew[e4[t]];
                        c4[t] = eu[e4[t]];
                    }
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (i0 + t < L) {
                        S_col[b + i0 + t] = c4[t];
                        S_w[b + i0 + t] = w4[t];
                        sum += w4[t];
                    }
            }
            for (int i = 0; i < U; ++i) {
                const double w = S_ew[u0 + i];
                S_col[b + L + i] = S_ev[u0 + i];
                S_eid[b + L + i] = (int32_t)(e0 + i);
                S_w[b + L + i] = w;
                sum += w;
            }
            deg[p] = sum;
            const double inv = sum > 0.0 ? 1.0 / sum : 0.0;
            for (int i = 0; i < L + U; ++i) S_w[b + i] = S_w[b + i] * inv;
        }
        __syncwarp();
        for (int j = lane; j < ns; j += 32) {
            const int32_t cj = S_col[j];
            const double x = S_w[j];
            col[R0 + j] = cj;
            eid[R0 + j] = S_eid[j];
            wn64[R0 + j] = x;
            cw32[R0 + j] = make_int2(cj, __float_as_int((float)x));
        }
        return;
    }
    if (!in || listed) return;
    int32_t le[LOWER_THREAD];
    for (int i = 0; i < L; ++i) {
        const int32_t x = eid[r0 + i];
        int j = i;
        while (j > 0 && le[j - 1] > x) {
            le[j] = le[j - 1];
            --j;
        }
        le[j] = x;
    }
    double sum = 0.0;
    for (int i = 0; i < L; ++i) {
        const int32_t e = le[i];
        const double w = ew[e];
        col[r0 + i] = eu[e];
        eid[r0 + i] = e;
        wn64[r0 + i] = w;
        sum += w;
    }
    for (int64_t e = e0; e < e1; ++e) {
        const int64_t j = r0 + L + (e - e0);
        const double w = ew[e];
        col[j] = ev[e];
        eid[j] = (int32_t)e;
        wn64[j] = w;
        sum += w;
    }
    deg[p] = sum;
    const double inv = sum > 0.0 ? 1.0 / sum : 0.0;
    const int64_t r1 = r0 + L + (e1 - e0);
    for (int64_t j = r0; j < r1; ++j) {
        const double x = wn64[j] * inv;
        wn64[j] = x;
        cw32[j] = make_int2(col[j], __float_as_int((float)x));
    }
}

// warp per listed row (lower part longer than a thread sorts): lower ids
// bitonic-sorted in shared memory; D(p,p) as lane-strided sums in slot order
// combined by a fixed shuffle tree
__global__ void __launch_bounds__(FW * 32) k_row_finish_warp(
    const int32_t* __restrict__ list, const int32_t* __restrict__ nlist,
    const int64_t* __restrict__ rowptr, const int64_t* __restrict__ eptr, const int32_t* __restrict__ lcnt,
    const int32_t* __restrict__ eu, const int32_t* __restrict__ ev, const double* __restrict__ ew,
    int32_t* __restrict__ col, int32_t* __restrict__ eid, double* __restrict__ wn64, int2* __restrict__ cw32,
    double* __restrict__ deg) {
    __shared__ int32_t sh[FW][LOWER_WARP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t* S = sh[w];
    const int64_t count = *nlist;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < count;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t p = list[r];
        const int L = lcnt[p];
        const int64_t r0 = rowptr[p], e0 = eptr[p], e1 = eptr[p + 1];
        const int P = L <= 1 ? 1 : 1 << (32 - __clz(L - 1));
        for (int t = lane; t < P; t += 32) S[t] = t < L ? eid[r0 + t] : 0x7fffffff;
        __syncwarp();
        for (int kk = 2; kk <= P; kk <<= 1)
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int t = lane; t < P; t += 32) {
                    const int u2 = t ^ j;
                    if (u2 > t) {
                        const int32_t x = S[t], y = S[u2];
                        if ((x > y) == ((t & kk) == 0)) {
                            S[t] = y;
                            S[u2] = x;
                        }
                    }
                }
                __syncwarp();
            }
        const int64_t len = L + (e1 - e0);
        double sum = 0.0;
        for (int64_t i = lane; i < len; i += 32) {
            int32_t e, q;
            if (i < L) {
                e = S[i];
                q = eu[e];
            } else {
                e = (int32_t)(e0 + (i - L));
                q = ev[e];
            }
            const double wv = ew[e];
            col[r0 + i] = q;
            eid[r0 + i] = e;
            wn64[r0 + i] = wv;
            sum += wv;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) deg[p] = sum;
        const double inv = sum > 0.0 ? 1.0 / sum : 0.0;
        for (int64_t i = lane; i < len; i += 32) {
            const double x = wn64[r0 + i] * inv;
            wn64[r0 + i] = x;
            cw32[r0 + i] = make_int2(col[r0 + i], __float_as_int((float)x));
        }
        __syncwarp();
    }
}

gr_status build_csr(gr_ctx* c, bool check, bool* invalid) {
    const int64_t n = c->n, m = c->m;
    cudaStream_t s = c->stream;
    if (invalid) *invalid = false;
    int64_t* hs = host_scratch();
    if (!hs) return set_error(c, GR_ENOMEM, "csr: pinned scratch unavailable");
    GR_TRY_CUDA(c, cudaMallocAsync(&c->eptr, sizeof(int64_t) * (n + 1), s), "alloc eptr");
    GR_TRY_CUDA(c, cudaMallocAsync(&c->rowptr, sizeof(int64_t) * (n + 1 + CSR_PAD_ROWS), s), "alloc rowptr");
    GR_TRY_CUDA(c, cudaMallocAsync(&c->deg, sizeof(double) * (n > 0 ? n : 1), s), "alloc deg");
    size_t slots = (size_t)(2 * m > 0 ? 2 * m : 1) + CSR_PAD_SLOTS;
    GR_TRY_CUDA(c, cudaMallocAsync(&c->col, sizeof(int32_t) * slots, s), "alloc col");
    GR_TRY_CUDA(c, cudaMallocAsync(&c->eid, sizeof(int32_t) * slots, s), "alloc eid");
    GR_TRY_CUDA(c, cudaMallocAsync(&c->cw32, sizeof(int2) * slots, s), "alloc cw32");
    GR_TRY_CUDA(c, cudaMallocAsync(&c->wn64, sizeof(double) * slots, s), "alloc wn64");

    // lcnt (n+1), lfill (n+1), list (n+1), flags (16 B); rowcnt (n+1, int64)
    void *p_i32, *p_i64;
    const size_t R = (size_t)(n + 1);
    GR_TRY_CUDA(c, c->ws.get(WS_COARSE_TMP, sizeof(int32_t) * (3 * R + 4), &p_i32), "ws");
    GR_TRY_CUDA(c, c->ws.get(WS_SORT_C, sizeof(int64_t) * R * 3, &p_i64), "ws");
    int32_t* lcnt = (int32_t*)p_i32;
    int32_t* lfill = lcnt + R;
    int32_t* list = lfill + R;
    int32_t* flags = list + R;  // [0] not canonical, [1] longest lower part, [2] listed rows
    int64_t* rowcnt = (int64_t*)p_i64;

    GR_TRY_CUDA(c, cudaMemsetAsync(lcnt, 0, sizeof(int32_t) * (2 * R), s), "memset");
    GR_TRY_CUDA(c, cudaMemsetAsync(flags, 0, 16, s), "memset");
    if (m > 0) {
        k_csr_count<<<(unsigned)ceil_div(m, TB), TB, 0, s>>>(n, m, c->eu, c->ev, c->ew, check ? 1 : 0, lcnt, flags,
                                                            flags + 1);
        count_launch();
    }
    // dense graphs (mean degree 32 or more): the global sort of the lower
    // parts beats per-row sorting of long lower parts
    const bool sparse = 2 * m < 32 * n;
    int32_t lmax = 0;
    if (check || sparse) {
        GR_TRY_CUDA(c, cudaMemcpyAsync(hs, flags, 16, cudaMemcpyDeviceToHost, s), "readback");
        GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
        const int32_t* hf = (const int32_t*)hs;
        if (hf[0]) {
            if (invalid) *invalid = true;
            return set_error(c, GR_EINVAL, "csr: the edge list is not canonical");
        }
        lmax = hf[1];
    }
    k_upper_ptr<<<(unsigned)ceil_div(m + 1, TB), TB, 0, s>>>(c->eu, m, n, c->eptr); count_launch();
    if (!sparse || lmax > LOWER_WARP) return build_csr_sorted(c, lcnt, rowcnt);
    k_row_total<<<(unsigned)ceil_div(n + 1, TB), TB, 0, s>>>(lcnt, c->eptr, n, rowcnt); count_launch();
    GR_TRY_CUDA(c, scan_exclusive_i64(rowcnt, c->rowptr, n + 1, c->ws, s), "scan rowptr");
    if (m > 0) {
        k_lower_claim<<<(unsigned)ceil_div(m, TB), TB, 0, s>>>(c->ev, m, c->rowptr, lfill, c->eid);
        count_launch();
    }
    if (n > 0) {
        k_row_finish_thread<<<(unsigned)ceil_div(n, TB), TB, 0, s>>>(n, c->rowptr, c->eptr, lcnt, c->eu, c->ev,
                                                                   c->ew, c->col, c->eid, c->wn64, c->cw32, c->deg,
                                                                   list, flags + 2);
        count_launch();
        if (lmax > LOWER_THREAD) {
            k_row_finish_warp<<<(unsigned)(c->num_sms * 16), FW * 32, 0, s>>>(list, flags + 2, c->rowptr, c->eptr,
                                                                              lcnt, c->eu, c->ev, c->ew, c->col,
                                                                              c->eid, c->wn64, c->cw32, c->deg);
            count_launch();
        }
    }
    GR_TRY_CUDA(c, cudaGetLastError(), "csr kernels");
    return GR_OK;
}

// Rows with a lower part too long for one warp's shared memory: a stable
// radix sort of the edge ids by v lists every row's lower part in order.
gr_status build_csr_sorted(gr_ctx* c, const int32_t* lcnt, int64_t* rowcnt) {
    const int64_t n = c->n, m = c->m;
    cudaStream_t s = c->stream;
    int64_t* lc64 = rowcnt + (n + 1);
    int64_t* lstart = lc64 + (n + 1);
    k_row_count<<<(unsigned)ceil_div(n + 1, TB), TB, 0, s>>>(lcnt, c->eptr, n, rowcnt, lc64); count_launch();
    GR_TRY_CUDA(c, scan_exclusive_i64(rowcnt, c->rowptr, n + 1, c->ws, s), "scan rowptr");
    GR_TRY_CUDA(c, scan_exclusive_i64(lc64, lstart, n + 1, c->ws, s), "scan lstart");
    if (m > 0) {
        void *p_k0, *p_v0, *p_alt;
        GR_TRY_CUDA(c, c->ws.get(WS_SORT_A, sizeof(uint32_t) * (size_t)m, &p_k0), "ws");
        GR_TRY_CUDA(c, c->ws.get(WS_SORT_B, sizeof(uint32_t) * (size_t)m, &p_v0), "ws");
        GR_TRY_CUDA(c, c->ws.get(WS_SORT_D, sizeof(uint32_t) * (size_t)m * 2, &p_alt), "ws");
        uint32_t* k0 = (uint32_t*)p_k0;
        uint32_t* v0 = (uint32_t*)p_v0;
        uint32_t* k1 = (uint32_t*)p_alt;
        uint32_t* v1 = k1 + m;
        k_keys_from_v<<<(unsigned)ceil_div(m, TB), TB, 0, s>>>(c->ev, m, k0, v0); count_launch();
        int alt = 0;
        GR_TRY_CUDA(c, radix_sort_u32(k0, v0, k1, v1, m, bits_for((uint64_t)(n - 1)), c->ws, s, &alt),
                    "sort by v");
        const uint32_t* sk = alt ? k1 : k0;
        const uint32_t* sv = alt ? v1 : v0;
        k_fill_lower<<<(unsigned)ceil_div(m, TB), TB, 0, s>>>(sk, sv, m, lstart, c->rowptr, c->eu,
                                                              c->ew, c->col, c->eid, c->wn64); count_launch();
        k_fill_upper<<<(unsigned)ceil_div(m, TB), TB, 0, s>>>(c->eu, c->ev, c->ew, m, c->eptr, lcnt,
                                                              c->rowptr, c->col, c->eid, c->wn64); count_launch();
    }
    GR_TRY_CUDA(c, degree_scale(c), "degree scale");
    return GR_OK;
}

cudaError_t degree_scale(gr_ctx* c) {
    const int64_t n = c->n, m = c->m;
    if (n > 0) {
        if (2 * m < 32 * n) {  // mean degree below 32: a thread per row
            k_degree_scale_rows<<<(unsigned)ceil_div(n, TB), TB, 0, c->stream>>>(c->rowptr, c->col, n, c->wn64,
                                                                                 c->cw32, c->deg);
        } else {
            k_degree_scale<<<(unsigned)ceil_div(n * 32, TB), TB, 0, c->stream>>>(c->rowptr, c->col, n, c->wn64,
                                                                                c->cw32, c->deg);
        }
        count_launch();
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Galerkin coarsening
// ---------------------------------------------------------------------------
// key of fine edge e = (min(A,B), max(A,B)) packed as min*nc + max; an edge
// inside one aggregate gets the sentinel nc*nc, which sorts after every pair.
__global__ void k_galerkin_keys(const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                                const int32_t* __restrict__ agg, int64_t m, uint64_t nc,
                                uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    uint64_t A = (uint64_t)agg[eu[e]], B = (uint64_t)agg[ev[e]];
    uint64_t lo = A < B ? A : B, hi = A < B ? B : A;
    keys[e] = A == B ? nc * nc : lo * nc + hi;
    vals[e] = (uint32_t)e;
}

__global__ void k_segment_heads(const uint64_t* __restrict__ keys, int64_t m, uint64_t sentinel,
                                int32_t* __restrict__ head) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    uint64_t k = keys[t];
    head[t] = (k != sentinel && (t == 0 || keys[t - 1] != k)) ? 1 : 0;
}

// one thread per segment head: sum the segment's fine weights in sorted order
// (ascending fine edge id, the sort being stable) into the reduced edge.
__global__ void k_segment_sum(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                              const int32_t* __restrict__ head, const int32_t* __restrict__ hpos,
                              int64_t m, uint64_t nc, const double* __restrict__ ew,
                              int32_t* __restrict__ uc, int32_t* __restrict__ vc,
                              double* __restrict__ wc) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m || !head[t]) return;
    uint64_t k = keys[t];
    double sum = 0.0;
    for (int64_t j = t; j < m && keys[j] == k; ++j) sum += ew[vals[j]];
    int64_t r = hpos[t];
    uc[r] = (int32_t)(k / nc);
    vc[r] = (int32_t)(k % nc);
    wc[r] = sum;
}

__global__ void k_total_i32(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                            int64_t m, int64_t* __restrict__ out) {
    *out = m > 0 ? (int64_t)pos[m - 1] + flag[m - 1] : 0;
}

__global__ void k_check_labels(const int32_t* __restrict__ agg, int64_t n, int64_t nc,
                               int32_t* __restrict__ used, int32_t* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t a = agg[i];
    if (a < 0 || a >= nc) atomicExch(bad, 1);
    else used[a] = 1;
}

__global__ void k_check_used(const int32_t* __restrict__ used, int64_t nc, int32_t* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc && !used[i]) atomicExch(bad, 1);
}

gr_status coarsen_impl(gr_ctx* c, const int32_t* agg, int64_t nc, gr_ctx** out) {
    const int64_t n = c->n, m = c->m;
    cudaStream_t s = c->stream;
    int64_t* hs = host_scratch();
    if (!hs) return set_error(c, GR_ENOMEM, "coarsen: pinned scratch unavailable");
    if (nc < 1 || nc > n) return set_error(c, GR_EINVAL, "coarsen: nc must be in [1, n]");
    if ((uint64_t)nc > (1ull << 31)) return set_error(c, GR_EINVAL, "coarsen: nc too large");

    gr_ctx* cc = new gr_ctx();
    cc->stream = s;
    cc->device = c->device;
    cc->num_sms = c->num_sms;
    cc->ws.stream = s;
    cc->n = nc;
    auto fail = [&](gr_status st) {
        graph_reduce_destroy(cc);
        return st;
    };
    // row-by-row assembly unless a coarse row is too long for shared memory
    bool too_long = false;
    {
        gr_status st = galerkin_rows(c, agg, nc, cc, &too_long);
        if (st != GR_OK) return fail(st);
        if (!too_long) {
            if (cudaMallocAsync(&cc->parent_map, sizeof(int32_t) * (size_t)(n > 0 ? n : 1), s) != cudaSuccess) {
                set_error(c, GR_ENOMEM, "coarsen: allocation failed");
                return fail(GR_ENOMEM);
            }
            GR_TRY_CUDA(c, cudaMemcpyAsync(cc->parent_map, agg, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice,
                                           s), "copy map");
            cc->parent_n = n;
            *out = cc;
            return GR_OK;
        }
    }
    // global sort path: labels must lie in [0, nc) and all be used
    void* p_chk;
    GR_TRY_CUDA(c, c->ws.get(WS_COARSE_TMP, sizeof(int32_t) * (size_t)(nc + 2), &p_chk), "ws");
    int32_t* used = (int32_t*)p_chk;
    int32_t* bad = used + nc;
    GR_TRY_CUDA(c, cudaMemsetAsync(used, 0, sizeof(int32_t) * (size_t)(nc + 1), s), "memset");
    k_check_labels<<<(unsigned)ceil_div(n, TB), TB, 0, s>>>(agg, n, nc, used, bad); count_launch();
    k_check_used<<<(unsigned)ceil_div(nc, TB), TB, 0, s>>>(used, nc, bad); count_launch();
    int64_t mc = 0;
    if (m > 0) {
        void *p_k, *p_v, *p_head;
        GR_TRY_CUDA(c, c->ws.get(WS_COARSE_KEYS, sizeof(uint64_t) * (size_t)m * 2, &p_k), "ws");
        GR_TRY_CUDA(c, c->ws.get(WS_COARSE_VALS, sizeof(uint32_t) * (size_t)m * 2, &p_v), "ws");
        GR_TRY_CUDA(c, c->ws.get(WS_SORT_A, sizeof(int32_t) * (size_t)m * 2, &p_head), "ws");
        uint64_t* k0 = (uint64_t*)p_k;
        uint64_t* k1 = k0 + m;
        uint32_t* v0 = (uint32_t*)p_v;
        uint32_t* v1 = v0 + m;
        int32_t* head = (int32_t*)p_head;
        int32_t* hpos = head + m;
        const uint64_t sentinel = (uint64_t)nc * (uint64_t)nc;
        k_galerkin_keys<<<(unsigned)ceil_div(m, TB), TB, 0, s>>>(c->eu, c->ev, agg, m, (uint64_t)nc, k0, v0); count_launch();
        int alt = 0;
        GR_TRY_CUDA(c, radix_sort_u64(k0, v0, k1, v1, m, bits_for(sentinel), c->ws, s, &alt), "sort keys");
        const uint64_t* sk = alt ? k1 : k0;
        const uint32_t* sv = alt ? v1 : v0;
        k_segment_heads<<<(unsigned)ceil_div(m, TB), TB, 0, s>>>(sk, m, sentinel, head); count_launch();
        GR_TRY_CUDA(c, scan_exclusive_i32(head, hpos, m, c->ws, s), "scan heads");
        k_total_i32<<<1, 1, 0, s>>>(head, hpos, m, hs); count_launch();
        GR_TRY_CUDA(c, cudaGetLastError(), "galerkin kernels");
        GR_TRY_CUDA(c, cudaMemcpyAsync(hs + 1, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                    "copy");
        GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
        mc = hs[0];
        if (((int32_t*)(hs + 1))[0]) {
            delete cc;
            return set_error(c, GR_EINVAL, "coarsen: labels must lie in [0, nc) and all be used");
        }
        cc->m = mc;
        cudaError_t e1 = cudaMallocAsync(&cc->eu, sizeof(int32_t) * (size_t)(mc > 0 ? mc : 1), s);
        cudaError_t e2 = cudaMallocAsync(&cc->ev, sizeof(int32_t) * (size_t)(mc > 0 ? mc : 1), s);
        cudaError_t e3 = cudaMallocAsync(&cc->ew, sizeof(double) * (size_t)(mc > 0 ? mc : 1), s);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
            set_error(c, GR_ENOMEM, "coarsen: allocation failed");
            return fail(GR_ENOMEM);
        }
        k_segment_sum<<<(unsigned)ceil_div(m, TB), TB, 0, s>>>(sk, sv, head, hpos, m, (uint64_t)nc,
                                                               c->ew, cc->eu, cc->ev, cc->ew); count_launch();
        GR_TRY_CUDA(c, cudaGetLastError(), "segment sum");
    } else {
        hs[1] = 0;
        GR_TRY_CUDA(c, cudaMemcpyAsync(hs + 1, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                    "copy");
        GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
        if (((int32_t*)(hs + 1))[0]) {
            delete cc;
            return set_error(c, GR_EINVAL, "coarsen: labels must lie in [0, nc) and all be used");
        }
        cc->m = 0;
        cudaMallocAsync(&cc->eu, 4, s);
        cudaMallocAsync(&cc->ev, 4, s);
        cudaMallocAsync(&cc->ew, 8, s);
    }
    gr_status st = build_csr(cc, false, nullptr);
    if (st != GR_OK) {
        set_error(c, st, "coarsen: " + cc->last_error);
        return fail(st);
    }
    if (cudaMallocAsync(&cc->parent_map, sizeof(int32_t) * (size_t)(n > 0 ? n : 1), s) != cudaSuccess) {
        set_error(c, GR_ENOMEM, "coarsen: allocation failed");
        return fail(GR_ENOMEM);
    }
    GR_TRY_CUDA(c, cudaMemcpyAsync(cc->parent_map, agg, sizeof(int32_t) * (size_t)n,
                                   cudaMemcpyDeviceToDevice, s), "copy map");
    cc->parent_n = n;
    *out = cc;
    return GR_OK;
}

// ---------------------------------------------------------------------------
// Map composition (fine -> coarsest)
// ---------------------------------------------------------------------------
struct MapChain {
    const int32_t* map[64];
    int count;
};

__global__ void k_compose(MapChain chain, int64_t n, int32_t* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t x = (int32_t)i;
    for (int l = 0; l < chain.count; ++l) x = chain.map[l][x];
    out[i] = x;
}

gr_status compose_impl(gr_ctx* const* levels, int nlevels, int32_t* out) {
    gr_ctx* c0 = levels[0];
    if (nlevels > 64) return set_error(c0, GR_EINVAL, "compose: at most 64 levels");
    MapChain ch;
    ch.count = nlevels;
    for (int l = 0; l < nlevels; ++l) {
        if (!levels[l] || !levels[l]->parent_map)
            return set_error(c0, GR_ESTATE, "compose: every level must come from coarsen");
        if (l > 0 && levels[l]->parent_n != levels[l - 1]->n)
            return set_error(c0, GR_EINVAL, "compose: levels do not chain");
        ch.map[l] = levels[l]->parent_map;
    }
    int64_t n = c0->parent_n;
    if (n > 0) {
        k_compose<<<(unsigned)ceil_div(n, TB), TB, 0, c0->stream>>>(ch, n, out);
        count_launch();
    }
    GR_TRY_CUDA(c0, cudaGetLastError(), "compose");
    return GR_OK;
}

}  // namespace gr
