// Galerkin reduced graph L_R = P^T L_G P (Sec. 3.2.2), assembled row by row.
//
// Coarse row A owns the CSR slots of its member nodes.  Each slot becomes the
// key (B << 32 | fine edge id) with B the aggregate of the slot's neighbour
// (slots of edges inside A become NOKEY), written into A's segment of a
// scratch array.  Sorting a segment groups equal B in ascending fine edge id,
// so summing each run in order gives w_R(A, B) exactly as the plain
// definition adds the crossing fine weights (ascending edge id), and the runs
// in order are A's coarse row with ascending neighbours -- the coarse CSR and
// the canonical coarse edge list come out directly, with no global sort.
//
// Segments are sorted by one warp each: up to 32 slots in registers, up to
// 128 in a small shared-memory buffer, up to 1,024 in a larger one.  A
// sorting network costs O(s log^2 s) per row, so graphs whose coarse rows are
// mostly long (more than 1/16 of them above 128 slots, or any above 1,024)
// use the global sort instead.
#include "gr_internal.cuh"

namespace gr {

namespace {

constexpr int GT = 256;
constexpr int SMALL_P = 128;      // rows up to this many slots: the small-row kernel
constexpr int MEDIUM_P = 1024;    // up to this many: a warp with a 16 KB buffer
constexpr int MEDIUM_WARPS = 4;   // warps per block in the medium kernel
constexpr uint64_t NOKEY = ~0ull;

__device__ __forceinline__ int32_t key_col(uint64_t k) { return (int32_t)(k >> 32); }
__device__ __forceinline__ int32_t key_edge(uint64_t k) { return (int32_t)(uint32_t)k; }

// member and slot counts per aggregate; labels outside [0, nc) raise `bad`
__global__ void k_gal_count(const int32_t* __restrict__ agg, const int64_t* __restrict__ rowptr, int64_t n,
                            int64_t nc, int32_t* __restrict__ mcnt, unsigned long long* __restrict__ scnt,
                            int32_t* __restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t a = agg[i];
    if (a < 0 || a >= nc) {
        atomicExch(bad, 1);
        return;
    }
    atomicAdd(&mcnt[a], 1);
    const int64_t len = rowptr[i + 1] - rowptr[i];
    if (len) atomicAdd(&scnt[a], (unsigned long long)len);
}

// every label used; the longest row; rows past the small kernel listed
__global__ void k_gal_check(const int32_t* __restrict__ mcnt, const unsigned long long* __restrict__ scnt,
                            int64_t nc, int32_t* __restrict__ bad, unsigned long long* __restrict__ smax,
                            int32_t* __restrict__ med, int32_t* __restrict__ nmed) {
    const int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long s = 0;
    if (A < nc) {
        if (mcnt[A] == 0) atomicExch(bad, 1);
        s = scnt[A];
    }
    const int32_t km = warp_slot(s > SMALL_P && s <= MEDIUM_P, nmed);
    if (km >= 0) med[km] = (int32_t)A;
    unsigned long long w = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, w, o);
        w = x > w ? x : w;
    }
    if ((threadIdx.x & 31) == 0 && w) atomicMax(smax, w);
}

// each fine node's slots into its aggregate's key segment; LPN lanes per node
template <int LPN>
__global__ void k_gal_scatter(const int32_t* __restrict__ agg, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ col, const int32_t* __restrict__ eid, int64_t n,
                              const int64_t* __restrict__ sptr, unsigned long long* __restrict__ sfill,
                              uint64_t* __restrict__ keys) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPN;
    const int l = threadIdx.x % LPN;
    if (i >= n) return;
    const int32_t a = agg[i];
    const int64_t b0 = rowptr[i], len = rowptr[i + 1] - b0;
    if (len == 0) return;
    int64_t off = 0;
    if (l == 0) off = sptr[a] + (int64_t)atomicAdd(&sfill[a], (unsigned long long)len);
    if (LPN > 1) {
        const unsigned gmask = LPN == 32 ? 0xffffffffu : (((1u << LPN) - 1u) << ((threadIdx.x & 31) / LPN * LPN));
        off = __shfl_sync(gmask, off, 0, LPN);
    }
    for (int64_t k = l; k < len; k += LPN) {
        const int64_t j = b0 + k;
        const int32_t B = __ldg(agg + col[j]);
        keys[off + k] = B == a ? NOKEY : (((uint64_t)(uint32_t)B << 32) | (uint64_t)(uint32_t)eid[j]);
    }
}

// Each fine node's slots into its aggregate's key segment, a warp per 32
// consecutive nodes: each lane claims its node's place in the segment, then
// the warp runs over the nodes' slots -- one contiguous range -- a slot per
// lane, so the column and edge-id reads come in whole lines.  Ranges longer
// than SC_CAP slots are written by each node's own lane.
constexpr int SC_CAP = 1024;

__global__ void __launch_bounds__(GT) k_gal_scatter_warp(const int32_t* __restrict__ agg,
                                                         const int64_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col,
                                                         const int32_t* __restrict__ eid, int64_t n,
                                                         const int64_t* __restrict__ sptr,
                                                         unsigned long long* __restrict__ sfill,
                                                         uint64_t* __restrict__ keys) {
    __shared__ uint8_t s_row[GT / 32][SC_CAP];
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int64_t pw = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    if (pw >= n) return;  // whole warp
    const int64_t p = pw + lane;
    const bool in = p < n;
    const int32_t a = in ? agg[p] : 0;
    const int64_t b0 = in ? rowptr[p] : 0;
    const int64_t len = in ? rowptr[p + 1] - b0 : 0;
    int64_t off = 0;
    if (len) off = sptr[a] + (int64_t)atomicAdd(&sfill[a], (unsigned long long)len);
    const int lv = (int)((n - pw < 32 ? n - pw : 32) - 1);
    const int64_t R0 = __shfl_sync(FULL, b0, 0);
    const int64_t R1 = __shfl_sync(FULL, b0 + len, lv);
    if (R1 - R0 > SC_CAP) {
        for (int64_t k = 0; k < len; ++k) {
            const int64_t j = b0 + k;
            const int32_t B = __ldg(agg + col[j]);
            keys[off + k] = B == a ? NOKEY : (((uint64_t)(uint32_t)B << 32) | (uint64_t)(uint32_t)eid[j]);
        }
        return;
    }
    uint8_t* S = s_row[wp];
    for (int64_t k = 0; k < len; ++k) S[b0 - R0 + k] = (uint8_t)lane;
    __syncwarp();
    const int ns = (int)(R1 - R0);
    for (int j0 = 0; j0 < ns; j0 += 32) {
        const int j = j0 + lane;
        const int r = j < ns ? S[j] : 0;
        const int32_t ar = __shfl_sync(FULL, a, r);
        const int64_t offr = __shfl_sync(FULL, off, r);
        const int64_t br = __shfl_sync(FULL, b0, r);
        if (j < ns) {
            const int64_t g = R0 + j;
            const int32_t B = __ldg(agg + col[g]);
            keys[offr + (g - br)] = B == ar ? NOKEY : (((uint64_t)(uint32_t)B << 32) | (uint64_t)(uint32_t)eid[g]);
        }
    }
}

// ascending bitonic sort of P (power of two, at least 64) keys in shared
// memory by one warp; the lanes take the stage's P / 2 compare-exchange
// pairs (t, t + j), t with bit j clear, so none idles
__device__ __forceinline__ void warp_bitonic(uint64_t* K, int P, int lane) {
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = lane; p < (P >> 1); p += 32) {
                const int t = ((p & ~(j - 1)) << 1) | (p & (j - 1));
                const int u = t | j;
                const uint64_t a = K[t], b = K[u];
                if ((a > b) == ((t & k) == 0)) {
                    K[t] = b;
                    K[u] = a;
                }
            }
            __syncwarp();
        }
}

__device__ __forceinline__ int next_pow2_dev(int x) { return x <= 1 ? 1 : 1 << (32 - __clz(x - 1)); }

// Runs of equal B in the sorted segment K[0, s) -> the coarse row of A, by one
// warp: weights gathered in parallel into Wt, each run summed in order by the
// lane holding its first slot.
__device__ __forceinline__ void warp_emit(const uint64_t* K, double* Wt, int s, int32_t A, int lane,
                                          const double* __restrict__ ew, int64_t base,
                                          int32_t* __restrict__ ucol, double* __restrict__ uw,
                                          int64_t* __restrict__ ucnt, int64_t* __restrict__ upcnt) {
    int valid = 0;
    for (int b = 0; b < s; b += 32) {
        const int t = b + lane;
        const bool ok = t < s && K[t] != NOKEY;
        if (ok) Wt[t] = __ldg(ew + key_edge(K[t]));
        valid += __popc(__ballot_sync(0xffffffffu, ok));
    }
    __syncwarp();
    int run = 0, up = 0;
    for (int b = 0; b < valid; b += 32) {
        const int t = b + lane;
        const bool h = t < valid && (t == 0 || key_col(K[t]) != key_col(K[t - 1]));
        const unsigned bal = __ballot_sync(0xffffffffu, h);
        const bool hu = h && key_col(K[t]) > A;
        if (h) {
            const int32_t B = key_col(K[t]);
            double sum = Wt[t];
            for (int u = t + 1; u < valid && key_col(K[u]) == B; ++u) sum += Wt[u];
            const int64_t r = base + run + __popc(bal & ((1u << lane) - 1u));
            ucol[r] = B;
            uw[r] = sum;
        }
        run += __popc(bal);
        up += __popc(__ballot_sync(0xffffffffu, hu));
    }
    if (lane == 0) {
        ucnt[A] = run;
        upcnt[A] = up;
    }
}

// A row of at most 32 slots, one slot per lane, without shared memory: the
// lanes sort 32-bit keys (B << 5 | slot) -- runs of equal B come out
// contiguous -- then rank the slots of each run by fine edge id, and the
// run's first lane adds the run's weights in that order.  Needs B < 2^27.
__device__ __forceinline__ void row32(const uint64_t* __restrict__ keys, int64_t base, int s, int32_t A, int lane,
                                      const double* __restrict__ ew, int32_t* __restrict__ ucol,
                                      double* __restrict__ uw, int64_t* __restrict__ ucnt,
                                      int64_t* __restrict__ upcnt) {
    constexpr unsigned FULL = 0xffffffffu;
    const uint64_t k = lane < s ? keys[base + lane] : NOKEY;
    const bool ok = k != NOKEY;
    const int32_t e = key_edge(k);
    const double w = ok ? __ldg(ew + e) : 0.0;
    uint32_t sk = ok ? (((uint32_t)key_col(k) << 5) | (uint32_t)lane) : 0xffffffffu;
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1)
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            const uint32_t o = __shfl_xor_sync(FULL, sk, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & kk) == 0);
            sk = keep_min ? min(sk, o) : max(sk, o);
        }
    const bool v = sk != 0xffffffffu;
    const int src = (int)(sk & 31u);
    const int32_t B = (int32_t)(sk >> 5);
    const int32_t ee = __shfl_sync(FULL, e, src);
    const double ww = __shfl_sync(FULL, w, src);
    const int32_t Bp = __shfl_up_sync(FULL, B, 1);
    const bool head = v && (lane == 0 || Bp != B);
    const unsigned hb = __ballot_sync(FULL, head);
    const unsigned vb = __ballot_sync(FULL, v);
    // this lane's run [start, end): from the last head at or below it to the
    // next head or the first empty lane after it
    const int start = 31 - __clz(hb & (FULL >> (31 - lane)));
    const unsigned after = lane == 31 ? 0u : ((hb | ~vb) & (FULL << (lane + 1)));
    const int end = after ? __ffs(after) - 1 : 32;
    const int len = v ? end - start : 0;
    int R = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) R = max(R, __shfl_xor_sync(FULL, R, o));
    int rank = 0;
    for (int d = 1; d < R; ++d) {
        const int32_t eu_ = __shfl_up_sync(FULL, ee, d);
        const int32_t ed_ = __shfl_down_sync(FULL, ee, d);
        if (v && lane - d >= start && eu_ < ee) ++rank;
        if (v && lane + d < end && ed_ < ee) ++rank;
    }
    const unsigned runmask = v ? ((end == 32 ? FULL : ((1u << end) - 1u)) & ~((1u << start) - 1u)) : 0u;
    double sum = 0.0;
    for (int r = 0; r < R; ++r) {
        const unsigned pick = __ballot_sync(FULL, v && rank == r) & runmask;
        const double x = __shfl_sync(FULL, ww, pick ? __ffs(pick) - 1 : lane);
        if (head && r < len) sum = r == 0 ? x : sum + x;
    }
    const unsigned ub = __ballot_sync(FULL, head && B > A);
    if (head) {
        const int64_t r = base + __popc(hb & ((1u << lane) - 1u));
        ucol[r] = B;
        uw[r] = sum;
    }
    if (lane == 0) {
        ucnt[A] = __popc(hb);
        upcnt[A] = __popc(ub);
    }
}

// rows of at most SMALL_P slots, a warp each (all rows visited, longer ones skipped)
__global__ void __launch_bounds__(GT) k_gal_rows_small(int64_t nc, const int64_t* __restrict__ sptr,
                                                       const uint64_t* __restrict__ keys,
                                                       const double* __restrict__ ew, int32_t* __restrict__ ucol,
                                                       double* __restrict__ uw, int64_t* __restrict__ ucnt,
                                                       int64_t* __restrict__ upcnt) {
    __shared__ uint64_t sk[GT / 32][SMALL_P];
    __shared__ double sw[GT / 32][SMALL_P];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t A = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (A >= nc) return;
    const int64_t base = sptr[A];
    const int s = (int)(sptr[A + 1] - base > SMALL_P ? SMALL_P + 1 : sptr[A + 1] - base);
    if (s > SMALL_P) return;
    if (s <= 32) {
        row32(keys, base, s, (int32_t)A, lane, ew, ucol, uw, ucnt, upcnt);
        return;
    }
    uint64_t* K = sk[w];
    const int P = next_pow2_dev(s);
    for (int t = lane; t < P; t += 32) K[t] = t < s ? keys[base + t] : NOKEY;
    __syncwarp();
    warp_bitonic(K, P, lane);
    warp_emit(K, sw[w], s, (int32_t)A, lane, ew, base, ucol, uw, ucnt, upcnt);
}

// listed rows of SMALL_P < s <= MEDIUM_P slots, a warp each, 16 KB of shared memory per warp
__global__ void __launch_bounds__(MEDIUM_WARPS * 32) k_gal_rows_medium(
    const int32_t* __restrict__ list, const int32_t* __restrict__ count, const int64_t* __restrict__ sptr,
    const uint64_t* __restrict__ keys, const double* __restrict__ ew, int32_t* __restrict__ ucol,
    double* __restrict__ uw, int64_t* __restrict__ ucnt, int64_t* __restrict__ upcnt) {
    extern __shared__ uint64_t smem_med[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t* K = smem_med + (size_t)w * 2 * MEDIUM_P;
    double* Wt = reinterpret_cast<double*>(K + MEDIUM_P);
    const int total = *count;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < total;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t A = list[r];
        const int64_t base = sptr[A];
        const int s = (int)(sptr[A + 1] - base);
        const int P = next_pow2_dev(s);
        for (int t = lane; t < P; t += 32) K[t] = t < s ? keys[base + t] : NOKEY;
        __syncwarp();
        warp_bitonic(K, P, lane);
        warp_emit(K, Wt, s, A, lane, ew, base, ucol, uw, ucnt, upcnt);
        __syncwarp();
    }
}

// Coarse CSR and canonical edge list from the per-row runs.  Lower entries
// (B < A) take the id of edge (B, A): A's position among B's upper entries.
template <int G>
__global__ void k_gal_fill(int64_t nc, const int64_t* __restrict__ sptr, const int32_t* __restrict__ ucol,
                           const double* __restrict__ uw, const int64_t* __restrict__ ucnt,
                           const int64_t* __restrict__ upcnt, const int64_t* __restrict__ rowptr,
                           const int64_t* __restrict__ eptr, int32_t* __restrict__ col, int32_t* __restrict__ eid,
                           double* __restrict__ wslot, int32_t* __restrict__ eu, int32_t* __restrict__ ev,
                           double* __restrict__ ew) {
    const int64_t A = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int l = threadIdx.x % G;
    if (A >= nc) return;
    const int64_t base = sptr[A], U = ucnt[A], low = U - upcnt[A], r0 = rowptr[A], e0 = eptr[A];
    for (int64_t i = l; i < U; i += G) {
        const int32_t B = ucol[base + i];
        const double w = uw[base + i];
        col[r0 + i] = B;
        wslot[r0 + i] = w;
        int64_t e;
        if (i >= low) {
            e = e0 + (i - low);
            eu[e] = (int32_t)A;
            ev[e] = B;
            ew[e] = w;
        } else {
            const int64_t bb = sptr[B], bu = ucnt[B], blow = bu - upcnt[B];
            int64_t lo = blow, hi = bu;  // A is among B's upper entries
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (ucol[bb + mid] < (int32_t)A) lo = mid + 1;
                else hi = mid;
            }
            e = eptr[B] + (lo - blow);
        }
        eid[r0 + i] = (int32_t)e;
    }
}

}  // namespace

gr_status galerkin_rows(gr_ctx* c, const int32_t* agg, int64_t nc, gr_ctx* cc, bool* too_long) {
    const int64_t n = c->n, m = c->m, slots = 2 * m;
    cudaStream_t s = c->stream;
    *too_long = false;
    int64_t* hs = host_scratch();
    if (!hs) return set_error(c, GR_ENOMEM, "coarsen: pinned scratch unavailable");

    // per-row arrays
    size_t need = 0;
    auto add = [&](size_t bytes) {
        size_t off = need;
        need += (bytes + 255) & ~size_t(255);
        return off;
    };
    const size_t R = (size_t)nc + 1;
    const size_t o_mcnt = add(4 * R), o_scnt = add(8 * R), o_sfill = add(8 * R), o_sptr = add(8 * R),
                 o_ucnt = add(8 * R), o_upcnt = add(8 * R), o_med = add(4 * R), o_ctr = add(64);
    void* pr;
    GR_TRY_CUDA(c, c->ws.get(WS_GAL_ROWS, need, &pr), "coarsen scratch");
    char* Bp = (char*)pr;
    int32_t* mcnt = (int32_t*)(Bp + o_mcnt);
    unsigned long long* scnt = (unsigned long long*)(Bp + o_scnt);
    unsigned long long* sfill = (unsigned long long*)(Bp + o_sfill);
    int64_t* sptr = (int64_t*)(Bp + o_sptr);
    int64_t* ucnt = (int64_t*)(Bp + o_ucnt);
    int64_t* upcnt = (int64_t*)(Bp + o_upcnt);
    int32_t* med = (int32_t*)(Bp + o_med);
    int32_t* ctr = (int32_t*)(Bp + o_ctr);  // [0] bad, [1] medium rows, [4..5] longest row
    // mcnt .. sfill are contiguous: one memset clears counts, slot sums and fills
    GR_TRY_CUDA(c, cudaMemsetAsync(Bp + o_mcnt, 0, o_sptr - o_mcnt, s), "memset");
    GR_TRY_CUDA(c, cudaMemsetAsync(ctr, 0, 64, s), "memset");
    if (n > 0) {
        k_gal_count<<<(unsigned)ceil_div(n, GT), GT, 0, s>>>(agg, c->rowptr, n, nc, mcnt, scnt, ctr);
        count_launch();
    }
    k_gal_check<<<(unsigned)ceil_div(nc, GT), GT, 0, s>>>(mcnt, scnt, nc, ctr, (unsigned long long*)(ctr + 4), med,
                                                          ctr + 1);
    count_launch();
    GR_TRY_CUDA(c, scan_exclusive_i64((const int64_t*)scnt, sptr, (int64_t)R, c->ws, s), "scan slots");
    GR_TRY_CUDA(c, cudaMemcpyAsync(hs, ctr, 32, cudaMemcpyDeviceToHost, s), "readback");
    GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
    const int32_t* hc = (const int32_t*)hs;
    if (hc[0]) return set_error(c, GR_EINVAL, "coarsen: labels must lie in [0, nc) and all be used");
    const int32_t nmed = hc[1];
    const unsigned long long smax = ((const unsigned long long*)hs)[2];
    // (the register path packs B into 27 bits)
    if (smax > (unsigned long long)MEDIUM_P || nc >= (int64_t(1) << 27)) {
        *too_long = true;
        return GR_OK;
    }

    void *pk, *pc, *pw;
    GR_TRY_CUDA(c, c->ws.get(WS_GAL_KEYS, sizeof(uint64_t) * (size_t)(slots > 0 ? slots : 1), &pk), "ws");
    GR_TRY_CUDA(c, c->ws.get(WS_GAL_UCOL, sizeof(int32_t) * (size_t)(slots > 0 ? slots : 1), &pc), "ws");
    GR_TRY_CUDA(c, c->ws.get(WS_GAL_UW, sizeof(double) * (size_t)(slots > 0 ? slots : 1), &pw), "ws");
    uint64_t* keys = (uint64_t*)pk;
    int32_t* ucol = (int32_t*)pc;
    double* uw = (double*)pw;

    if (slots > 0) {
        if (slots >= 32 * n) {
            k_gal_scatter<32><<<(unsigned)ceil_div(n * 32, GT), GT, 0, s>>>(agg, c->rowptr, c->col, c->eid, n, sptr,
                                                                           sfill, keys);
        } else {
            k_gal_scatter_warp<<<(unsigned)ceil_div(n, GT), GT, 0, s>>>(agg, c->rowptr, c->col, c->eid, n, sptr,
                                                                       sfill, keys);
        }
        count_launch();
    }
    k_gal_rows_small<<<(unsigned)ceil_div(nc * 32, GT), GT, 0, s>>>(nc, sptr, keys, c->ew, ucol, uw, ucnt, upcnt);
    count_launch();
    if (nmed > 0) {
        const size_t dyn = (size_t)MEDIUM_WARPS * 2 * MEDIUM_P * sizeof(uint64_t);
        GR_TRY_CUDA(c, cudaFuncSetAttribute(k_gal_rows_medium, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn),
                    "smem attribute");
        const int64_t want = ceil_div(nmed, MEDIUM_WARPS), cap = (int64_t)c->num_sms * 3;
        k_gal_rows_medium<<<(unsigned)(want < cap ? want : cap), MEDIUM_WARPS * 32, dyn, s>>>(
            med, ctr + 1, sptr, keys, c->ew, ucol, uw, ucnt, upcnt);
        count_launch();
    }
    GR_TRY_CUDA(c, cudaGetLastError(), "galerkin rows");

    // coarse row pointers and edge-id bases
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->eptr, sizeof(int64_t) * R, s), "alloc eptr");
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->rowptr, sizeof(int64_t) * (R + CSR_PAD_ROWS), s), "alloc rowptr");
    GR_TRY_CUDA(c, cudaMemsetAsync(ucnt + nc, 0, sizeof(int64_t), s), "memset");
    GR_TRY_CUDA(c, cudaMemsetAsync(upcnt + nc, 0, sizeof(int64_t), s), "memset");
    GR_TRY_CUDA(c, scan_exclusive_i64(ucnt, cc->rowptr, (int64_t)R, c->ws, s), "scan rows");
    GR_TRY_CUDA(c, scan_exclusive_i64(upcnt, cc->eptr, (int64_t)R, c->ws, s), "scan edges");
    GR_TRY_CUDA(c, cudaMemcpyAsync(hs, cc->eptr + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "readback");
    GR_TRY_CUDA(c, cudaMemcpyAsync(hs + 1, cc->rowptr + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "readback");
    GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
    const int64_t mc = hs[0];
    if (hs[1] != 2 * mc) return set_error(c, GR_ECUDA, "coarsen: coarse rows are not symmetric");
    cc->m = mc;
    const size_t cs = (size_t)(2 * mc > 0 ? 2 * mc : 1) + CSR_PAD_SLOTS, ce = (size_t)(mc > 0 ? mc : 1);
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->eu, sizeof(int32_t) * ce, s), "alloc");
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->ev, sizeof(int32_t) * ce, s), "alloc");
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->ew, sizeof(double) * ce, s), "alloc");
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->deg, sizeof(double) * (size_t)(nc > 0 ? nc : 1), s), "alloc");
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->col, sizeof(int32_t) * cs, s), "alloc");
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->eid, sizeof(int32_t) * cs, s), "alloc");
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->cw32, sizeof(int2) * cs, s), "alloc");
    GR_TRY_CUDA(c, cudaMallocAsync(&cc->wn64, sizeof(double) * cs, s), "alloc");
    if (mc > 0) {
        if (2 * mc >= 32 * nc) {
            k_gal_fill<32><<<(unsigned)ceil_div(nc * 32, GT), GT, 0, s>>>(nc, sptr, ucol, uw, ucnt, upcnt, cc->rowptr,
                                                                        cc->eptr, cc->col, cc->eid, cc->wn64, cc->eu,
                                                                        cc->ev, cc->ew);
        } else {
            k_gal_fill<4><<<(unsigned)ceil_div(nc * 4, GT), GT, 0, s>>>(nc, sptr, ucol, uw, ucnt, upcnt, cc->rowptr,
                                                                      cc->eptr, cc->col, cc->eid, cc->wn64, cc->eu,
                                                                      cc->ev, cc->ew);
        }
        count_launch();
    }
    GR_TRY_CUDA(c, cudaGetLastError(), "galerkin fill");
    GR_TRY_CUDA(c, degree_scale(cc), "degree scale");
    return GR_OK;
}

}  // namespace gr
