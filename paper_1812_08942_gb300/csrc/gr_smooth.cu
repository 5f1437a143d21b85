// Test-vector smoothing (Sec. 3.2.1, weighted Jacobi of Alg. 3).
//
// Storage scheme.  The stored block A_t is the un-normalised iterate; the
// FP64 statistics (mu_t, 1/s_t) of its columns define the normalised iterate
// X_t = (A_t - mu_t) / s_t.  Because J = (1-w) I + w D^-1 A maps the all-ones
// vector to itself (an isolated node keeps its value, so this holds there
// too), J X_t = (J A_t - mu_t) / s_t: a sweep gathers the raw A_t, applies the
// previous statistics once per output row in its epilogue, and accumulates the
// statistics of what it stores.  A final pass writes (A_S - mu_S) / s_S.
#include <cuda_bf16.h>

#include "gr_internal.cuh"
#include "gr_sweep.cuh"
#include "gr_vec.cuh"

namespace gr {

constexpr int SM_THREADS = 256;
constexpr int SM_WARPS = SM_THREADS / 32;

// ---------------------------------------------------------------------------
// Column statistics: per-block partial sums (FP64) and a last-block finish
// that turns them into (mu, 1/s) for every column, in fixed order.
// ---------------------------------------------------------------------------
// Block-level combine of per-lane column sums; lane l of segment 0 with
// t == 0 holds chunk l.  Writes the block partial and, in the last block to
// finish, the final statistics.
template <typename Acc, int K, int E, int G, int LPR>
__device__ void block_stats(Acc (&s1)[E], Acc (&s2)[E], double* __restrict__ part,
                            unsigned* __restrict__ counter, int64_t n,
                            double* __restrict__ stats_out) {
    __shared__ double wst[SM_WARPS][2 * K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < E; ++e) {
#pragma unroll
        for (int o = LPR; o < 32; o <<= 1) {
            s1[e] += __shfl_xor_sync(0xffffffffu, s1[e], o);
            s2[e] += __shfl_xor_sync(0xffffffffu, s2[e], o);
        }
    }
    if (lane < G) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            wst[warp][lane * E + e] = (double)s1[e];
            wst[warp][K + lane * E + e] = (double)s2[e];
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        double s = 0.0;
        for (int w = 0; w < SM_WARPS; ++w) s += wst[w][threadIdx.x];
        part[(int64_t)blockIdx.x * 2 * K + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    finish_stats<K, SM_THREADS>(part, gridDim.x, counter, n, stats_out);
}

// Column sums of a stored block, per lane in the accumulator type (FP32 for
// FP32 / BF16 blocks): a lane sums a few hundred entries at most, then lanes
// are combined in FP32 within a warp and in FP64 from the warp level up.
// Compensated FP32 sums per lane were measured 13-74 % slower on the
// latency-bound sweep, and FP64 arithmetic runs at a small fraction of the
// FP32 rate on this part, so the per-lane sums stay plain FP32.
template <typename Acc, int E>
__device__ __forceinline__ void add_sums(Acc (&s1)[E], Acc (&s2)[E], const Acc (&y)[E]) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
        s1[e] += y[e];
        s2[e] += y[e] * y[e];
    }
}

// ---------------------------------------------------------------------------
// Initial test vectors: SplitMix64 output c+1 for counter c (Steele, Lea,
// Flood 2014), top 53 bits -> u in [0,1), entry 2u - 1, rounded once to the
// storage type (bfloat16: rounded from the FP32 value).
// ---------------------------------------------------------------------------
constexpr uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ull;

// the generator's output for state z = seed + (c + 1) * gamma
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    return splitmix64_mix(seed + (c + 1ull) * SM_GAMMA);
}

// 2u - 1 with u = (z>>11) 2^-53 equals t 2^-52 for the integer
// t = (z>>11) - 2^52, |t| <= 2^52.  This part's FP64 and 64-bit conversion
// units are slow, so neither conversion below uses them.
__device__ __forceinline__ int64_t uniform_pm1_int(uint64_t z) { return (int64_t)(z >> 11) - (1ll << 52); }

// FP64: exact, the IEEE bit pattern built with integer operations
__device__ __forceinline__ double scaled_int_to_f64(int64_t t) {
    if (t == 0) return 0.0;
    const uint64_t sign = t < 0 ? (1ull << 63) : 0ull;
    const uint64_t a = t < 0 ? (uint64_t)(-t) : (uint64_t)t;
    const int p = 63 - __clzll((long long)a);  // a in [2^p, 2^(p+1)), p <= 52
    const uint64_t frac = (a << (52 - p)) & ((1ull << 52) - 1ull);
    return __longlong_as_double((long long)(sign | ((uint64_t)(p - 52 + 1023) << 52) | frac));
}

// FP32: rounded once to nearest, ties to even, by rounding to odd (Boldo and
// Melquiond, IEEE Trans. Computers 57(4), 2008).  t = hi 2^29 + lo with
// 0 <= lo < 2^29; hi 2^29 is exact in FP32, and so is lo rounded to odd on
// the grid 2^5 (24 significant bits at most).  Their FP32 sum is the nearest
// even rounding of t whenever that grid lies two bits below t's last kept
// bit, i.e. |t| >= 2^30; smaller |t| fit in 32 bits and take the 32-bit
// conversion, which rounds to nearest even itself.
// hi = t >> 29 = (z >> 40) - 2^23 and lo = bits 11..39 of z come straight
// from the generator output's two 32-bit halves.
__device__ __forceinline__ float uniform_pm1_f32(uint64_t z) {
    const uint32_t zh = (uint32_t)(z >> 32), zl = (uint32_t)z;
    const int32_t hi = (int32_t)(zh >> 8) - (1 << 23);
    const uint32_t lo = __funnelshift_r(zl, zh, 11) & 0x1fffffffu;
    if ((uint32_t)(hi + 2) > 3u) {  // hi >= 2 or hi <= -3: |t| >= 2^30
        const uint32_t lo_odd = (lo & ~31u) | ((lo & 31u) ? 32u : 0u);
        return (__int2float_rn(hi) * 0x1p29f + __uint2float_rn(lo_odd)) * 0x1p-52f;
    }
    return __int2float_rn((int32_t)((uint32_t)hi << 29) + (int32_t)lo) * 0x1p-52f;  // |t| < 2^30
}

template <typename T>
__device__ __forceinline__ typename AccOf<T>::type uniform_pm1(uint64_t z);
template <>
__device__ __forceinline__ double uniform_pm1<double>(uint64_t z) {
    return scaled_int_to_f64(uniform_pm1_int(z));
}
template <>
__device__ __forceinline__ float uniform_pm1<float>(uint64_t z) {
    return uniform_pm1_f32(z);
}
template <>
__device__ __forceinline__ float uniform_pm1<__nv_bfloat16>(uint64_t z) {
    return uniform_pm1<float>(z);
}

// Block-level combine when thread t of the grid holds the sums of column
// chunk (t mod G) -- the grid's thread count is a multiple of G, so lane l of
// a warp holds chunk (c + l) mod G with c the warp's first thread: lane l < G
// adds the lanes l + r G (all 32 lanes carry data) and writes its chunk's
// sums.  Then as block_stats.
template <typename Acc, int K, int E, int G>
__device__ void block_stats_chunks(Acc (&s1)[E], Acc (&s2)[E], int q, double* __restrict__ part,
                                   unsigned* __restrict__ counter, int64_t n, double* __restrict__ stats_out) {
    __shared__ double wst[SM_WARPS][2 * K];
    constexpr int RW = (32 + G - 1) / G;  // lane groups per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
        for (int r = 1; r < RW; ++r) {
            const int src = lane + r * G;
            const Acc a1 = __shfl_sync(0xffffffffu, s1[e], src & 31);
            const Acc a2 = __shfl_sync(0xffffffffu, s2[e], src & 31);
            if (lane < G && src < 32) {
                s1[e] += a1;
                s2[e] += a2;
            }
        }
    if (lane < G) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            wst[warp][q * E + e] = (double)s1[e];
            wst[warp][K + q * E + e] = (double)s2[e];
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        double t = 0.0;
        for (int w = 0; w < SM_WARPS; ++w) t += wst[w][threadIdx.x];
        part[(int64_t)blockIdx.x * 2 * K + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    finish_stats<K, SM_THREADS>(part, gridDim.x, counter, n, stats_out);
}

// X0 and its statistics.  Chunk c (entries c E ... c E + E - 1 of the
// row-major block, row c / G) goes to thread c mod T of the grid, T threads in
// all, a multiple of G (init_grid): every lane of a warp works, and each
// thread keeps one chunk column.
template <typename T, int K>
__global__ void __launch_bounds__(SM_THREADS) k_init(int64_t n, uint64_t seed, uint64_t level,
                                                     T* __restrict__ A, double* __restrict__ part,
                                                     unsigned* __restrict__ counter,
                                                     double* __restrict__ stats_out) {
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t c0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t total = (uint64_t)n * G;
    const int q = (int)(c0 % G);
    Acc s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) s1[e] = s2[e] = Acc(0);
    for (uint64_t c = c0; c < total; c += nthreads) {
        Acc x[E];
        // generator state of this chunk's first entry (entry index c E); the
        // next entries follow by one gamma each
        uint64_t zs = seed + ((level << 40) + c * E + 1ull) * SM_GAMMA;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            x[e] = uniform_pm1<T>(splitmix64_mix(zs));
            zs += SM_GAMMA;
        }
        store_chunk<T, E>(A + c * E, x);
        add_sums<Acc, E>(s1, s2, x);
    }
    block_stats_chunks<Acc, K, E, G>(s1, s2, q, part, counter, n, stats_out);
}

// k_init's grid: one full wave of resident blocks (a larger grid would leave
// a ragged second wave), fewer when there are few rows
template <typename T, int K>
static int init_grid(const gr_ctx* c, int64_t n) {
    static int occ = 0;
    if (!occ) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_init<T, K>, SM_THREADS, 0) != cudaSuccess || occ < 1)
            occ = 1;
        if (occ > 8) occ = 8;
    }
    // the grid's thread count must be a multiple of G: of 3 blocks when 3 | G
    constexpr int G = RowLayout<T, K>::G;
    constexpr int64_t step = G % 3 == 0 ? 3 : 1;
    const int64_t want = ceil_div(n * G, (int64_t)SM_THREADS);
    int64_t cap = (int64_t)c->num_sms * occ;
    if (cap > STATS_GROUP * STATS_MAX_GROUPS) cap = STATS_GROUP * STATS_MAX_GROUPS;
    int64_t g = want < cap ? want : cap;
    g = (g + step - 1) / step * step;
    if (g > cap) g -= step;
    return (int)(g > 0 ? g : step);
}

// ---------------------------------------------------------------------------
// Streaming sweep.
//
// Each warp owns a contiguous row range holding about the same number of
// slots (+ ST_ROW_COST per row), so its slot list is one contiguous stream.
// The warp keeps ST_D batches of 32 slots in flight into a private shared-
// memory ring with cp.async (16 B per lane, L2 only), so the DRAM latency of
// the slot stream overlaps the L2 gathers of the neighbour rows.
// The warp takes one row at a time, 32 slots per step (LPR = 32): GP lanes
// own a 16-byte chunk of the vector row and TS = 32 / GP neighbours are
// gathered per round.
// Slots: (column, FP32 weight) for FP32 / BF16 blocks, (column, pad, FP64
// weight) for FP64 blocks.
// ---------------------------------------------------------------------------
constexpr int ST_NB = 16;              // ring batches per warp
constexpr int ST_D = 8;                // batches kept in flight ahead of use
constexpr int ST_RING = ST_NB * 32;    // ring slots per warp
constexpr int ST_SPAN = ST_NB - ST_D;  // batches one window may span
static_assert(ST_SPAN >= 1, "a window must fit the ring");
constexpr int ST_ROW_COST = 8;         // partition weight of a row, in slots

template <typename T>
struct SlotOf { using type = int2; };
template <>
struct SlotOf<double> { using type = int4; };
__device__ __forceinline__ int slot_col(const int2& v) { return v.x; }
__device__ __forceinline__ int slot_col(const int4& v) { return v.x; }
__device__ __forceinline__ float slot_w(const int2& v, float) { return __int_as_float(v.y); }
__device__ __forceinline__ double slot_w(const int4& v, double) { return __hiloint2double(v.w, v.z); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// wpart[w] = first row r with rowptr[r] + ST_ROW_COST * r >= w * C / W
__global__ void k_warp_partition(int64_t n, const int64_t* __restrict__ rowptr, int64_t W,
                                 int32_t* __restrict__ wpart) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w > W) return;
    const double C = (double)rowptr[n] + (double)ST_ROW_COST * (double)n;
    const double target = C * (double)w / (double)W;
    int64_t lo = 0, hi = n;  // answer in [0, n]
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((double)rowptr[mid] + (double)ST_ROW_COST * (double)mid >= target) hi = mid;
        else lo = mid + 1;
    }
    wpart[w] = (int32_t)(w == W ? n : lo);
}

// (col, 0, w) packed slots for the FP64 stream
__global__ void k_pack64(int64_t slots, const int32_t* __restrict__ col, const double* __restrict__ wn64,
                         int4* __restrict__ cw64) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < slots) {
        double w = wn64[j];
        cw64[j] = make_int4(col[j], 0, __double2loint(w), __double2hiint(w));
    }
}

template <typename T, int K, int LPR>
__global__ void __launch_bounds__(SM_THREADS) k_sweep_stream(
    int64_t n, const int64_t* __restrict__ rowptr, const typename SlotOf<T>::type* __restrict__ slots,
    int64_t total_slots, const int32_t* __restrict__ wpart, const T* __restrict__ Ain, T* __restrict__ Aout,
    double omega_d, const double* __restrict__ stats_in, double* __restrict__ part,
    unsigned* __restrict__ counter, double* __restrict__ stats_out) {
    using Slot = typename SlotOf<T>::type;
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G, GP = L::GP;
    static_assert(LPR == 32, "one row per warp");
    constexpr int TS = 32 / GP;                  // neighbours per round
    constexpr int PER_LANE = 16 / (int)sizeof(Slot);  // slots one 16-byte copy moves
    constexpr int COPY_LANES = 32 / PER_LANE;
    extern __shared__ __align__(16) unsigned char st_dyn[];
    __shared__ Acc st_sh[2 * K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane % GP, t = lane / GP;
    const bool chunk_ok = q < G;
    const Acc omega = (Acc)omega_d, one_m = (Acc)(1.0 - omega_d);
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) st_sh[i] = (Acc)stats_in[i];
    __syncthreads();
    Slot* ring = reinterpret_cast<Slot*>(st_dyn) + warp * ST_RING;
    Acc s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) s1[e] = s2[e] = Acc(0);

    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int32_t r0 = wpart[wg], r1 = wpart[wg + 1];
    if (r0 < r1) {
        // stream positions are 32-bit offsets from B0 (a warp's range is < 2^31 slots)
        const int64_t S0 = rowptr[r0];
        const int64_t B0 = S0 & ~(int64_t)31;
        const int32_t o_s0 = (int32_t)(S0 - B0);
        const int32_t o_s1 = (int32_t)(rowptr[r1] - B0);
        const int32_t o_tot = (int32_t)((total_slots - B0) < 0x7fffffff ? (total_slots - B0) : 0x7fffffff);
        const Slot* src = slots + B0;
        // batch k: offsets [32k, 32k + 32); COPY_LANES lanes move 16 bytes each
        auto issue = [&](int32_t k) {
            const int32_t o = 32 * k + PER_LANE * lane;
            if (lane < COPY_LANES && o < o_s1 && o + PER_LANE > o_s0 && o < o_tot)
                cp_async16(&ring[o & (ST_RING - 1)], src + o);
            cp_async_commit();
        };
#pragma unroll 1
        for (int k = 0; k < ST_D; ++k) issue(k);
        int32_t ready = 0;  // batches [0, ready) have landed
        // the window [lo, hi] of batches must fit the ring: hi - lo < ST_SPAN
        auto ensure = [&](int32_t kb_hi) {
            while (ready <= kb_hi) {
                cp_async_wait<ST_D - 1>();
                __syncwarp();
                issue(ready + ST_D);
                ++ready;
            }
        };
        int32_t rp_base = r0;  // lane l caches rowptr[rp_base + 1 + l] - B0
        int32_t rp_next = (r0 + 1 + lane <= n) ? (int32_t)(rowptr[r0 + 1 + lane] - B0) : 0;
        int32_t gb = o_s0;     // start of the current row
        {
            for (int32_t row = r0; row < r1; ++row) {
                if (row - rp_base >= 32) {
                    rp_base = row;
                    rp_next = (row + 1 + lane <= n) ? (int32_t)(rowptr[row + 1 + lane] - B0) : 0;
                }
                const int32_t e_end = __shfl_sync(0xffffffffu, rp_next, row - rp_base);
                Acc xi[E];
                if (t == 0 && chunk_ok) load_chunk<T, E>(Ain + (int64_t)row * K + q * E, xi);
                Acc acc[E];
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] = Acc(0);
                for (int32_t base = gb; base < e_end; base += 32) {
                    const int32_t cnt = e_end - base < 32 ? e_end - base : 32;
                    ensure((base + cnt - 1) >> 5);
#pragma unroll
                    for (int r = 0; r < GP; ++r) {
                        const int sidx = r * TS + t;
                        if (sidx < cnt && chunk_ok) {
                            const Slot v = ring[(base + sidx) & (ST_RING - 1)];
                            Acc x[E];
                            load_chunk<T, E>(Ain + (int64_t)slot_col(v) * K + q * E, x);
                            const Acc w = slot_w(v, Acc(0));
#pragma unroll
                            for (int e = 0; e < E; ++e) acc[e] = fma(w, x[e], acc[e]);
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < E; ++e)
#pragma unroll
                    for (int o = GP; o < 32; o <<= 1) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
                if (t == 0 && chunk_ok) {
                    const bool isolated = gb == e_end;
                    Acc y[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int k = q * E + e;
                        Acc z = isolated ? xi[e] : one_m * xi[e] + omega * acc[e];
                        y[e] = (z - st_sh[k]) * st_sh[K + k];
                    }
                    store_chunk<T, E>(Aout + (int64_t)row * K + q * E, y);
                    add_sums<Acc, E>(s1, s2, y);
                }
                        gb = e_end;
            }
        }
        cp_async_wait_all();
    }
    block_stats<Acc, K, E, G, LPR>(s1, s2, part, counter, n, stats_out);
}

// ---------------------------------------------------------------------------
// Row-group sweep (the default sweep kernel).
//
// G lanes serve one row (one 16-byte chunk of the K-wide vector row each), so
// a warp runs RPW = floor(32 / G) consecutive rows at once (for K = 24 FP32:
// 5 rows x 6 lanes, 30 of 32 lanes busy); row groups go in grid-stride order,
// so all warps work on one band of rows at a time and the neighbour rows of
// banded graphs stay in L2.  Every lane reads the slot entries of its row
// itself (the G lanes of a row hit the same address, an L1 broadcast), then
// gathers U neighbour chunks at once: no shuffles, no predicated empty
// rounds.  The row pointers of the next two groups are loaded ahead; keeping
// registers low buys resident warps, which hides the gather latency better
// than deeper per-warp prefetch did.  Slot indices are 32-bit (2m < 2^32) and
// rows 32-bit (n < 2^31).
// ---------------------------------------------------------------------------
template <typename Acc, int K, int E, int G>
__device__ void block_stats_rows(Acc (&s1)[E], Acc (&s2)[E], double* __restrict__ part,
                                 unsigned* __restrict__ counter, int64_t n, double* __restrict__ stats_out) {
    __shared__ double wst[SM_WARPS][2 * K];
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // lanes q < G collect the sums of lanes q + r G (same chunk, other rows)
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
        for (int r = 1; r < RPW; ++r) {
            const Acc a1 = __shfl_sync(0xffffffffu, s1[e], (lane + r * G) & 31);
            const Acc a2 = __shfl_sync(0xffffffffu, s2[e], (lane + r * G) & 31);
            if (lane < G) {
                s1[e] += a1;
                s2[e] += a2;
            }
        }
    if (lane < G) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            wst[warp][lane * E + e] = (double)s1[e];
            wst[warp][K + lane * E + e] = (double)s2[e];
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        double t = 0.0;
        for (int w = 0; w < SM_WARPS; ++w) t += wst[w][threadIdx.x];
        part[(int64_t)blockIdx.x * 2 * K + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    finish_stats<K, SM_THREADS>(part, gridDim.x, counter, n, stats_out);
}


template <typename T, int K, int U>
__device__ __forceinline__ void sweep_row_body(
    int64_t n64, const int64_t* __restrict__ rowptr, const typename SlotOf<T>::type* __restrict__ slots,
    const T* __restrict__ Ain, T* __restrict__ Aout, double omega_d, const double* __restrict__ stats_in,
    double* __restrict__ part, unsigned* __restrict__ counter, double* __restrict__ stats_out) {
    using Slot = typename SlotOf<T>::type;
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G;
    constexpr int RPW = 32 / G;
    __shared__ Acc st_sh[2 * K];
    const int n = (int)n64;
    const int lane = threadIdx.x & 31;
    const int seg = lane / G, q = lane % G;
    const bool lane_ok = seg < RPW;  // the last 32 mod G lanes idle
    const Acc omega = (Acc)omega_d, one_m = (Acc)(1.0 - omega_d);
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) st_sh[i] = (Acc)stats_in[i];
    __syncthreads();
    Acc s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) s1[e] = s2[e] = Acc(0);
    const int stride = ((gridDim.x * blockDim.x) >> 5) * RPW;
    int row = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW + (lane_ok ? seg : 0);
    const T* Aq = Ain + q * E;
    auto rp = [&](int r, unsigned& b, unsigned& e) {
        if (r < n && lane_ok) {
            b = (unsigned)__ldg(rowptr + r);
            e = (unsigned)__ldg(rowptr + r + 1);
        } else {
            b = e = 0u;
        }
    };
    unsigned b0, e0, b1, e1;
    rp(row, b0, e0);
    rp(row + stride, b1, e1);
    const int gend = n + (lane_ok ? seg : 0);  // the loop runs while this warp's group start is < n
    for (; row < gend; row += stride) {
        unsigned b2, e2;
        rp(row + 2 * stride, b2, e2);
        if (lane_ok) {
            Acc xi[E];
            if (row < n) load_chunk<T, E>(Aq + (size_t)row * K, xi);
            Acc acc[E];
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = Acc(0);
            for (unsigned j = b0; j < e0; j += U) {
                Slot v[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (j + u < e0) v[u] = __ldg(slots + j + u);
                Acc x[U][E];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (j + u < e0) load_chunk<T, E>(Aq + (size_t)slot_col(v[u]) * K, x[u]);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (j + u < e0) {
                        const Acc w = slot_w(v[u], Acc(0));
#pragma unroll
                        for (int e = 0; e < E; ++e) acc[e] = fma(w, x[u][e], acc[e]);
                    }
            }
            if (q == 0 && e1 > b1) {
                // the next group's slot lines into L1 (its row pointers have
                // arrived by now): its slot loads then wait on L1, not on
                // memory, and no register is held for them
                const char* p0 = reinterpret_cast<const char*>(slots + b1);
                const char* p1 = reinterpret_cast<const char*>(slots + e1) - 1;
                asm volatile("prefetch.global.L1 [%0];" ::"l"(p0));
                if (((uintptr_t)p0 >> 7) != ((uintptr_t)p1 >> 7)) asm volatile("prefetch.global.L1 [%0];" ::"l"(p1));
            }
            if (row < n) {
                const bool isolated = b0 == e0;
                Acc y[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int k = q * E + e;
                    Acc z = isolated ? xi[e] : one_m * xi[e] + omega * acc[e];
                    y[e] = (z - st_sh[k]) * st_sh[K + k];
                }
                store_chunk<T, E>(Aout + (size_t)row * K + q * E, y);
                add_sums<Acc, E>(s1, s2, y);
            }
        }
        b0 = b1;
        e0 = e1;
        b1 = b2;
        e1 = e2;
    }
    block_stats_rows<Acc, K, E, G>(s1, s2, part, counter, n64, stats_out);
}

// the registers as the compiler fits them (three blocks per SM for FP32
// rows of 24 columns) ...
template <typename T, int K, int U>
__global__ void __launch_bounds__(SM_THREADS) k_sweep_row(
    int64_t n64, const int64_t* __restrict__ rowptr, const typename SlotOf<T>::type* __restrict__ slots,
    const T* __restrict__ Ain, T* __restrict__ Aout, double omega_d, const double* __restrict__ stats_in,
    double* __restrict__ part, unsigned* __restrict__ counter, double* __restrict__ stats_out) {
    sweep_row_body<T, K, U>(n64, rowptr, slots, Ain, Aout, omega_d, stats_in, part, counter, stats_out);
}

// ... or fitted to four blocks per SM (four slots in flight)
template <typename T, int K>
__global__ void __launch_bounds__(SM_THREADS, 4) k_sweep_row_fit4(
    int64_t n64, const int64_t* __restrict__ rowptr, const typename SlotOf<T>::type* __restrict__ slots,
    const T* __restrict__ Ain, T* __restrict__ Aout, double omega_d, const double* __restrict__ stats_in,
    double* __restrict__ part, unsigned* __restrict__ counter, double* __restrict__ stats_out) {
    sweep_row_body<T, K, 4>(n64, rowptr, slots, Ain, Aout, omega_d, stats_in, part, counter, stats_out);
}

// X = (A - mu) * inv_s, chunk-parallel; A may be X itself (each entry is read
// and written by the same thread).  The statistics are converted to the
// accumulator type once per block; chunk indices are 32-bit when they fit.
template <typename T, int K>
__global__ void k_apply(int64_t n, const T* A, T* X, const double* __restrict__ stats) {
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G;
    __shared__ Acc st[2 * K];
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) st[i] = (Acc)stats[i];
    __syncthreads();
    const uint64_t total = (uint64_t)n * G;
    auto one = [&](int64_t row, int q) {
        Acc x[E];
        load_chunk<T, E>(A + row * K + q * E, x);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = q * E + e;
            x[e] = (x[e] - st[k]) * st[K + k];
        }
        store_chunk<T, E>(X + row * K + q * E, x);
    };
    if (total <= 0xffffffffull) {
        const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
        if (idx < (uint32_t)total) one((int64_t)(idx / G), (int)(idx % G));
    } else {
        const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (idx < total) one((int64_t)(idx / G), (int)(idx % G));
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Scratch the sweep launchers keep in the context between calls (the packed
// FP64 slots, the streaming kernel's row partition).  graph_reduce_smooth
// allocates it in the context on first use; the allocation-free entry point
// passes a region of its fixed array instead, and whatever the context does
// not hold already is rebuilt there on every call.
struct SweepScratch {
    char* base = nullptr;  // nullptr: allocate in the context
    size_t bytes = 0, used = 0;
    bool fixed() const { return base != nullptr; }
    void* take(size_t n) {
        const size_t off = (used + 255) & ~size_t(255);
        if (off + n > bytes) return nullptr;
        used = off + n;
        return base + off;
    }
};

// Streaming sweep when a group of 32 / GP rows would hold more slots than
// four ring batches (long rows).
template <typename T, int K>
static bool stream_wide(const gr_ctx* c) {
    constexpr int GP = RowLayout<T, K>::GP;
    const double avg = c->n > 0 ? 2.0 * (double)c->m / (double)c->n : 0.0;
    return GP < 32 && (32.0 / GP) * avg > 128.0;
}

template <typename T>
constexpr int prec_of() {
    return sizeof(T) == 8 ? GR_F64 : (sizeof(T) == 4 ? GR_F32 : GR_BF16);
}

// the kernel every sweep of one smoothing call runs, and its inputs
struct SweepPlan {
    int kind = GR_SWEEP_ROW;     // GR_SWEEP_ROW / GR_SWEEP_STREAM / GR_SWEEP_BAND
    const int4* cw64 = nullptr;  // FP64 slots of the row-group and streaming kernels
    const int32_t* wpart = nullptr;
    int grid = 0;
    size_t dyn = 0;
    BandPlan band;               // band kernel: its shape, far runs and slot rows
    const int4* runs = nullptr;
    const void* bslots = nullptr;
};

// packed (column, 0, FP64 weight) slots
static cudaError_t prepare_slots64(gr_ctx* c, SweepScratch& sc, const int4** out) {
    if (c->cw64) {
        *out = c->cw64;
        return cudaSuccess;
    }
    const size_t bytes = sizeof(int4) * (size_t)(2 * c->m > 0 ? 2 * c->m : 1);
    int4* p = nullptr;
    if (sc.fixed()) {
        p = (int4*)sc.take(bytes);
        if (!p) return cudaErrorMemoryAllocation;
    } else {
        GR_CUDA(cudaMallocAsync(&c->cw64, bytes, c->stream));
        p = c->cw64;
    }
    if (c->m > 0) {
        k_pack64<<<(unsigned)ceil_div(2 * c->m, 256), 256, 0, c->stream>>>(2 * c->m, c->col, c->wn64, p);
        count_launch();
    }
    *out = p;
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t prepare_stream(gr_ctx* c, SweepScratch& sc, int part_cap, SweepPlan* P) {
    using Slot = typename SlotOf<T>::type;
    static int bps = 0;
    P->dyn = sizeof(Slot) * (size_t)ST_RING * SM_WARPS;
    if (!bps) {
        auto kern = k_sweep_stream<T, K, 32>;
        GR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->dyn));
        GR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, SM_THREADS, P->dyn));
        if (bps < 1) bps = 1;
    }
    int grid = c->num_sms * bps;
    if (grid > part_cap) grid = part_cap;
    P->grid = grid;
    const int64_t W = (int64_t)grid * SM_WARPS;
    if (c->wpart_W == W) {
        P->wpart = c->wpart;
    } else {
        int32_t* wp = nullptr;
        if (sc.fixed()) {
            wp = (int32_t*)sc.take(sizeof(int32_t) * (size_t)(W + 1));
            if (!wp) return cudaErrorMemoryAllocation;
        } else {
            if (c->wpart) GR_CUDA(cudaFreeAsync(c->wpart, c->stream));
            c->wpart = nullptr;
            c->wpart_W = 0;
            GR_CUDA(cudaMallocAsync(&c->wpart, sizeof(int32_t) * (size_t)(W + 1), c->stream));
            c->wpart_W = W;
            wp = c->wpart;
        }
        k_warp_partition<<<(unsigned)ceil_div(W + 1, 256), 256, 0, c->stream>>>(c->n, c->rowptr, W, wp);
        count_launch();
        P->wpart = wp;
    }
    if constexpr (sizeof(T) == 8) GR_CUDA(prepare_slots64(c, sc, &P->cw64));
    return cudaGetLastError();
}

// Band kernel: when forced, wherever a band fits shared memory; in the
// automatic choice, for rows that are not long (the streaming kernel's case)
// on graphs large enough to give every SM a chunk of bands (smaller ones skip
// the locality profile and its synchronisation), whose locality profile
// admits a band and whose tables place at least BAND_AUTO_SHARED of the
// neighbours in shared memory (the verdict is kept in the context per plan).  `tmp` (at least 264 bytes of device memory
// the stream does not use yet) holds the locality profile's counts on the
// first call.  *chosen tells whether P now runs the band kernel.
constexpr double BAND_AUTO_SHARED = 0.95;

template <typename T, int K>
static cudaError_t choose_band(gr_ctx* c, SweepScratch& sc, void* tmp, SweepPlan* P, bool* chosen) {
    *chosen = false;
    const int want = c->sweep_kind;
    constexpr bool f64 = sizeof(T) == 8;
    if (want != GR_SWEEP_BAND && !(want == GR_SWEEP_AUTO && !stream_wide<T, K>(c))) return cudaSuccess;
    // FP32 / BF16 bands hold 80 rows or more and a chunk 8 bands: smaller
    // graphs could not give every SM a chunk
    if (want == GR_SWEEP_AUTO && c->n < (int64_t)c->num_sms * 8 * 80) return cudaSuccess;
    GR_CUDA(ensure_locality(c, tmp));
    BandPlan bp;
    if (!band_usable(c, prec_of<T>(), K, want == GR_SWEEP_BAND, &bp)) return cudaSuccess;
    if (want == GR_SWEEP_AUTO && bp.grid < c->num_sms) return cudaSuccess;
    const bool known = c->band_auto_ok >= 0 && c->band_auto_R == bp.R && c->band_auto_H == bp.H &&
                       c->band_auto_grid == bp.grid && c->band_auto_f64 == (int)f64;
    if (want == GR_SWEEP_AUTO && known && c->band_auto_ok == 0) return cudaSuccess;
    void* scr = nullptr;
    size_t scr_bytes = 0;
    if (sc.fixed()) {  // what the context does not hold is built in the rest of the fixed array
        const size_t off = (sc.used + 255) & ~size_t(255);
        scr_bytes = off < sc.bytes ? sc.bytes - off : 0;
        scr = scr_bytes ? sc.take(scr_bytes) : nullptr;
    }
    int64_t nglobal = -1;
    const bool decide = want == GR_SWEEP_AUTO && !known;
    GR_CUDA(band_prepare(c, bp, f64, sc.fixed(), scr, scr_bytes, &P->runs, &P->bslots, decide ? &nglobal : nullptr));
    if (decide) {
        c->band_auto_R = bp.R;
        c->band_auto_H = bp.H;
        c->band_auto_grid = bp.grid;
        c->band_auto_f64 = (int)f64;
        c->band_auto_ok = (double)nglobal <= (1.0 - BAND_AUTO_SHARED) * 2.0 * (double)c->m ? 1 : 0;
        if (!c->band_auto_ok) {
            if (!sc.fixed()) band_release(c);
            return cudaSuccess;
        }
    }
    P->kind = GR_SWEEP_BAND;
    P->band = bp;
    *chosen = true;
    return cudaSuccess;
}

// Kernel choice: forced by graph_reduce_set_sweep_kernel; automatically the
// streaming kernel for long rows, the band kernel on banded graphs (above),
// otherwise the row-group kernel.
template <typename T, int K>
static cudaError_t sweep_prepare(gr_ctx* c, SweepScratch& sc, int part_cap, void* tmp, SweepPlan* P) {
    const int want = c->sweep_kind;
    bool band = false;
    GR_CUDA((choose_band<T, K>(c, sc, tmp, P, &band)));
    if (band) return cudaSuccess;
    if (want == GR_SWEEP_STREAM || (want == GR_SWEEP_AUTO && stream_wide<T, K>(c))) {
        P->kind = GR_SWEEP_STREAM;
        return prepare_stream<T, K>(c, sc, part_cap, P);
    }
    P->kind = GR_SWEEP_ROW;
    if constexpr (sizeof(T) == 8) GR_CUDA(prepare_slots64(c, sc, &P->cw64));
    return cudaSuccess;
}

template <typename T, int K>
static cudaError_t launch_sweep_row(gr_ctx* c, const SweepPlan& P, const T* Ain, T* Aout, double omega,
                                    const double* st_in, double* part, int part_cap, unsigned* counter,
                                    double* st_out) {
    // two slots in flight per lane; four on rows of mean degree >= 10 in
    // FP32/BF16 storage (measured: 13-19 % faster there, slower in FP64 and
    // on shorter rows).  The products are added in slot order either way.
    // Large FP32 blocks that stay in L2 (at least ROW_DENSE_MIN_ROWS rows, at
    // most ROW_DENSE_MAX_BYTES) are gather-latency bound: there the four-slot
    // kernel runs with its registers fitted to four blocks per SM (level 1 of
    // the 128^3 mesh, 605k rows: 86 against 96 us per sweep; smaller levels
    // ran slower with more, smaller blocks).
    constexpr int64_t ROW_DENSE_MIN_ROWS = 400000;
    constexpr size_t ROW_DENSE_MAX_BYTES = size_t(96) << 20;
    static int bps2 = 0, bps4 = 0, bps4d = 0;
    if (!bps2) {
        GR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps2, k_sweep_row<T, K, 2>, SM_THREADS, 0));
        GR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps4, k_sweep_row<T, K, 4>, SM_THREADS, 0));
        if constexpr (sizeof(T) == 4)
            GR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps4d, k_sweep_row_fit4<T, K>, SM_THREADS, 0));
        if (bps2 < 1) bps2 = 1;
        if (bps4 < 1) bps4 = 1;
        if (bps4d < 1) bps4d = 1;
    }
    const bool four = sizeof(T) < 8 && c->n > 0 && 2.0 * (double)c->m / (double)c->n >= 10.0;
    const bool dense = four && sizeof(T) == 4 && c->n >= ROW_DENSE_MIN_ROWS &&
                       (size_t)c->n * K * sizeof(T) <= ROW_DENSE_MAX_BYTES;
    int grid = c->num_sms * (dense ? bps4d : (four ? bps4 : bps2));
    if (grid > part_cap) grid = part_cap;
    const typename SlotOf<T>::type* slots;
    if constexpr (sizeof(T) == 8) slots = P.cw64;
    else slots = c->cw32;
    if constexpr (sizeof(T) == 4) {
        if (dense) {
            k_sweep_row_fit4<T, K><<<grid, SM_THREADS, 0, c->stream>>>(c->n, c->rowptr, slots, Ain, Aout, omega,
                                                                       st_in, part, counter, st_out);
            count_launch();
            return cudaGetLastError();
        }
    }
    if (four)
        k_sweep_row<T, K, 4><<<grid, SM_THREADS, 0, c->stream>>>(c->n, c->rowptr, slots, Ain, Aout, omega, st_in, part,
                                                                 counter, st_out);
    else
        k_sweep_row<T, K, 2><<<grid, SM_THREADS, 0, c->stream>>>(c->n, c->rowptr, slots, Ain, Aout, omega, st_in, part,
                                                                 counter, st_out);
    count_launch();
    return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t launch_sweep(gr_ctx* c, const SweepPlan& P, const T* Ain, T* Aout, double omega,
                                const double* st_in, double* part, int part_cap, unsigned* counter, double* st_out) {
    if (P.kind == GR_SWEEP_BAND)  // the error word follows the counter
        return sweep_band(c, prec_of<T>(), K, P.band, P.runs, P.bslots, Ain, Aout, omega, st_in, part, part_cap,
                          counter, st_out, (int*)(counter + 1));
    if (P.kind == GR_SWEEP_STREAM) {
        const typename SlotOf<T>::type* slots;
        if constexpr (sizeof(T) == 8) slots = P.cw64;
        else slots = c->cw32;
        k_sweep_stream<T, K, 32><<<P.grid, SM_THREADS, P.dyn, c->stream>>>(c->n, c->rowptr, slots, 2 * c->m, P.wpart,
                                                                          Ain, Aout, omega, st_in, part, counter,
                                                                          st_out);
        count_launch();
        return cudaGetLastError();
    }
    return launch_sweep_row<T, K>(c, P, Ain, Aout, omega, st_in, part, part_cap, counter, st_out);
}

// Bytes of the statistics region: two 2K-double statistics sets, then the
// counter words (the kernel and group tickets of the statistics finish and
// the band kernel's error word).
template <int K>
constexpr size_t stats_bytes() {
    return sizeof(double) * 4 * K + STATS_COUNTER_BYTES;
}

// X0, `sweeps` sweeps and the final centring + scaling into X.  buf is the
// second n x K block; stats has stats_bytes<K>(); part holds 2K doubles for
// each of up to part_cap blocks.
template <typename T, int K>
static cudaError_t run_sweeps(gr_ctx* c, SweepScratch& sc, int sweeps, double omega, uint64_t seed, int level,
                              T* X, T* buf, double* stats, double* part, int part_cap, cudaEvent_t ev0,
                              cudaEvent_t ev1, SmoothRaw* raw = nullptr) {
    cudaStream_t s = c->stream;
    const int64_t n = c->n;
    double* st0 = stats;
    double* st1 = st0 + 2 * K;
    unsigned* counter = (unsigned*)(st1 + 2 * K);
    // the tickets and the error word start at zero: the region may hold an earlier call's values
    GR_CUDA(cudaMemsetAsync(counter, 0, STATS_COUNTER_BYTES, s));
    SweepPlan P;
    // the partials are free until k_init: scratch for the locality profile
    if (sweeps > 0) GR_CUDA((sweep_prepare<T, K>(c, sc, part_cap, part, &P)));
    const int igrid = init_grid<T, K>(c, n);
    k_init<T, K><<<igrid, SM_THREADS, 0, s>>>(n, seed, (uint64_t)level, X, part, counter, st0); count_launch();
    GR_CUDA(cudaGetLastError());
    const T* cur = X;
    T* nxt = buf;
    if (ev0) GR_CUDA(cudaEventRecord(ev0, s));
    double* sin = st0;
    double* sout = st1;
    for (int it = 0; it < sweeps; ++it) {
        GR_CUDA((launch_sweep<T, K>(c, P, cur, nxt, omega, sin, part, part_cap, counter, sout)));
        const T* tmp = cur;
        cur = nxt;
        nxt = (T*)tmp;
        double* ts = sin;
        sin = sout;
        sout = ts;
    }
    if (ev1) GR_CUDA(cudaEventRecord(ev1, s));
    if (raw) {  // the caller applies the statistics
        raw->A = cur;
        raw->stats = sin;
        return cudaSuccess;
    }
    constexpr int G = RowLayout<T, K>::G;
    if (n > 0) {
        k_apply<T, K><<<(unsigned)ceil_div(n * G, 256), 256, 0, s>>>(n, cur, X, sin);
        count_launch();
    }
    return cudaGetLastError();
}

// blocks any sweep or k_init grid may have (the statistics partials)
static int part_capacity(const gr_ctx* c) {
    const int cap = c->num_sms * 8;
    return cap < STATS_GROUP * STATS_MAX_GROUPS ? cap : STATS_GROUP * STATS_MAX_GROUPS;
}

template <typename T, int K>
static cudaError_t run_smooth(gr_ctx* c, int sweeps, double omega, uint64_t seed, int level,
                              T* X, cudaEvent_t ev0, cudaEvent_t ev1, SmoothRaw* raw) {
    const int64_t n = c->n;
    void *p_buf, *p_st, *p_part;
    const int cap = part_capacity(c);
    GR_CUDA(c->ws.get(WS_SMOOTH_BUF, sizeof(T) * (size_t)n * K, &p_buf));
    GR_CUDA(c->ws.get(WS_SMOOTH_STATS, stats_bytes<K>(), &p_st));
    GR_CUDA(c->ws.get(WS_SMOOTH_PART, sizeof(double) * 2 * K * (size_t)cap, &p_part));
    SweepScratch sc;
    return run_sweeps<T, K>(c, sc, sweeps, omega, seed, level, X, (T*)p_buf, (double*)p_st, (double*)p_part, cap,
                            ev0, ev1, raw);
}

template <typename T>
static cudaError_t smooth_typed(gr_ctx* c, int K, int sweeps, double omega, uint64_t seed,
                                int level, void* X, cudaEvent_t e0, cudaEvent_t e1, SmoothRaw* raw) {
    switch (K) {
        case 4: return run_smooth<T, 4>(c, sweeps, omega, seed, level, (T*)X, e0, e1, raw);
        case 8: return run_smooth<T, 8>(c, sweeps, omega, seed, level, (T*)X, e0, e1, raw);
        case 16: return run_smooth<T, 16>(c, sweeps, omega, seed, level, (T*)X, e0, e1, raw);
        case 24: return run_smooth<T, 24>(c, sweeps, omega, seed, level, (T*)X, e0, e1, raw);
        case 32: return run_smooth<T, 32>(c, sweeps, omega, seed, level, (T*)X, e0, e1, raw);
    }
    return cudaErrorInvalidValue;
}

// the raw block X0 alone (one launch of k_init; its statistics go to scratch)
template <typename T, int K>
static cudaError_t run_test_vectors(gr_ctx* c, uint64_t seed, int level, T* X) {
    cudaStream_t s = c->stream;
    const int64_t n = c->n;
    void *p_st, *p_part;
    GR_CUDA(c->ws.get(WS_SMOOTH_STATS, stats_bytes<K>(), &p_st));
    double* st0 = (double*)p_st;
    unsigned* counter = (unsigned*)(st0 + 4 * K);
    const int64_t cap = part_capacity(c);
    const int igrid = init_grid<T, K>(c, n);
    GR_CUDA(c->ws.get(WS_SMOOTH_PART, sizeof(double) * 2 * K * (size_t)cap, &p_part));
    GR_CUDA(cudaMemsetAsync(counter, 0, STATS_COUNTER_BYTES, s));
    k_init<T, K><<<igrid, SM_THREADS, 0, s>>>(n, seed, (uint64_t)level, X, (double*)p_part, counter, st0);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
static cudaError_t test_vectors_typed(gr_ctx* c, int K, uint64_t seed, int level, void* X) {
    switch (K) {
        case 4: return run_test_vectors<T, 4>(c, seed, level, (T*)X);
        case 8: return run_test_vectors<T, 8>(c, seed, level, (T*)X);
        case 16: return run_test_vectors<T, 16>(c, seed, level, (T*)X);
        case 24: return run_test_vectors<T, 24>(c, seed, level, (T*)X);
        case 32: return run_test_vectors<T, 32>(c, seed, level, (T*)X);
    }
    return cudaErrorInvalidValue;
}

gr_status test_vectors_impl(gr_ctx* c, int K, uint64_t seed, int level, gr_prec prec, void* X) {
    cudaError_t e;
    switch (prec) {
        case GR_F64: e = test_vectors_typed<double>(c, K, seed, level, X); break;
        case GR_F32: e = test_vectors_typed<float>(c, K, seed, level, X); break;
        case GR_BF16: e = test_vectors_typed<__nv_bfloat16>(c, K, seed, level, X); break;
        default: return set_error(c, GR_EINVAL, "test_vectors: unknown precision");
    }
    if (e != cudaSuccess) return cuda_error(c, e, "test_vectors");
    return GR_OK;
}

gr_status smooth_impl(gr_ctx* c, int K, int sweeps, double omega, uint64_t seed, int level,
                      gr_prec prec, void* X, cudaEvent_t e0, cudaEvent_t e1, SmoothRaw* raw) {
    cudaError_t e;
    switch (prec) {
        case GR_F64: e = smooth_typed<double>(c, K, sweeps, omega, seed, level, X, e0, e1, raw); break;
        case GR_F32: e = smooth_typed<float>(c, K, sweeps, omega, seed, level, X, e0, e1, raw); break;
        case GR_BF16: e = smooth_typed<__nv_bfloat16>(c, K, sweeps, omega, seed, level, X, e0, e1, raw); break;
        default: return set_error(c, GR_EINVAL, "smooth: unknown precision");
    }
    if (e != cudaSuccess) return cuda_error(c, e, "smooth");
    return GR_OK;
}

// The kernel choice of sweep_prepare, without launching a sweep (the band
// kernel's tables and verdict are built on first use, as a smoothing call
// would).
template <typename T, int K>
static cudaError_t sweep_plan_typed(gr_ctx* c, int32_t* kind) {
    const int want = c->sweep_kind;
    void* tmp = nullptr;
    GR_CUDA(c->ws.get(WS_SMOOTH_PART, sizeof(double) * 2 * K * (size_t)part_capacity(c), &tmp));
    SweepScratch sc;
    SweepPlan P;
    bool band = false;
    GR_CUDA((choose_band<T, K>(c, sc, tmp, &P, &band)));
    if (band) {
        *kind = GR_SWEEP_BAND;
        return cudaSuccess;
    }
    *kind = (want == GR_SWEEP_STREAM || (want == GR_SWEEP_AUTO && stream_wide<T, K>(c))) ? GR_SWEEP_STREAM
                                                                                         : GR_SWEEP_ROW;
    return cudaSuccess;
}

template <typename T>
static cudaError_t sweep_plan_k(gr_ctx* c, int K, int32_t* info) {
    switch (K) {
        case 4: return sweep_plan_typed<T, 4>(c, info);
        case 8: return sweep_plan_typed<T, 8>(c, info);
        case 16: return sweep_plan_typed<T, 16>(c, info);
        case 24: return sweep_plan_typed<T, 24>(c, info);
        case 32: return sweep_plan_typed<T, 32>(c, info);
    }
    return cudaErrorInvalidValue;
}

gr_status sweep_plan_impl(gr_ctx* c, int K, gr_prec prec, int32_t* info) {
    cudaError_t e;
    switch (prec) {
        case GR_F64: e = sweep_plan_k<double>(c, K, info); break;
        case GR_F32: e = sweep_plan_k<float>(c, K, info); break;
        case GR_BF16: e = sweep_plan_k<__nv_bfloat16>(c, K, info); break;
        default: return set_error(c, GR_EINVAL, "sweep_plan: unknown precision");
    }
    if (e != cudaSuccess) return cuda_error(c, e, "sweep_plan");
    return GR_OK;
}

// ---------------------------------------------------------------------------
// Multicolour Gauss-Seidel (the relaxation Sec. 3.2.1 names).  Ordering: the
// greedy colouring in descending priority, computed by Jones-Plassmann rounds
// (an uncoloured node whose priority beats all its uncoloured neighbours takes
// the smallest colour its coloured neighbours leave free).  Adjacent nodes
// never colour in the same round, and a node's coloured neighbours when it
// colours are exactly its higher-priority ones, so the result is the greedy
// colouring whatever the order of the updates within a round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t gs_prio(uint64_t seed, int64_t i) {
    return splitmix64_at(seed, (1ull << 62) + (uint64_t)i);
}

__global__ void k_jp_round(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           uint64_t seed, int32_t* colour, int32_t* __restrict__ left, int32_t* __restrict__ maxc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || __ldcg(colour + i) >= 0) return;
    const uint64_t pi = gs_prio(seed, i);
    const int64_t b = rowptr[i], e = rowptr[i + 1];
    for (int64_t j = b; j < e; ++j) {
        const int32_t q = col[j];
        if (__ldcg(colour + q) < 0) {
            const uint64_t pq = gs_prio(seed, q);
            if (pq > pi || (pq == pi && q > i)) {
                atomicAdd(left, 1);
                return;
            }
        }
    }
    // smallest colour not used by a coloured neighbour, 64 candidates at a time
    int32_t c = 0;
    for (int32_t base = 0;; base += 64) {
        unsigned long long used = 0;
        for (int64_t j = b; j < e; ++j) {
            const int32_t cq = __ldcg(colour + col[j]);
            if (cq >= base && cq < base + 64) used |= 1ull << (cq - base);
        }
        if (~used) {
            c = base + __ffsll((long long)~used) - 1;
            break;
        }
    }
    colour[i] = c;
    atomicMax(maxc, c);
}

__global__ void k_colour_keys(int64_t n, const int32_t* __restrict__ colour, uint32_t* __restrict__ keys,
                              uint32_t* __restrict__ vals, int32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = (uint32_t)colour[i];
    vals[i] = (uint32_t)i;
    atomicAdd(&cnt[colour[i]], 1);
}

// Colouring for colour_seed: colour (device, n) and, in the context, the node
// list in ascending (colour, id) with each colour's range.
static gr_status gs_prepare(gr_ctx* c, uint64_t colour_seed, int32_t* colour_out) {
    const int64_t n = c->n;
    cudaStream_t s = c->stream;
    size_t need = 0;
    auto add = [&](size_t bytes) {
        size_t off = need;
        need += (bytes + 255) & ~size_t(255);
        return off;
    };
    const size_t o_col = add(4 * (size_t)n), o_k0 = add(4 * (size_t)n), o_v0 = add(4 * (size_t)n),
                 o_k1 = add(4 * (size_t)n), o_v1 = add(4 * (size_t)n), o_cnt = add(4 * (size_t)(n + 2)),
                 o_ptr = add(4 * (size_t)(n + 2)), o_ctr = add(64);
    void* base;
    GR_TRY_CUDA(c, c->ws.get(WS_GS, need, &base), "colouring scratch");
    char* B = (char*)base;
    int32_t* colour = colour_out ? colour_out : (int32_t*)(B + o_col);
    uint32_t* k0 = (uint32_t*)(B + o_k0);
    uint32_t* v0 = (uint32_t*)(B + o_v0);
    uint32_t* k1 = (uint32_t*)(B + o_k1);
    uint32_t* v1 = (uint32_t*)(B + o_v1);
    int32_t* cnt = (int32_t*)(B + o_cnt);
    int32_t* cptr = (int32_t*)(B + o_ptr);
    int32_t* ctr = (int32_t*)(B + o_ctr);  // [0] left after the round, [1] largest colour
    int64_t* hs = host_scratch();
    if (!hs) return set_error(c, GR_ENOMEM, "colouring: pinned scratch unavailable");
    GR_TRY_CUDA(c, cudaMemsetAsync(colour, 0xff, 4 * (size_t)n, s), "memset");
    GR_TRY_CUDA(c, cudaMemsetAsync(ctr, 0, 64, s), "memset");
    const unsigned gn = (unsigned)ceil_div(n > 0 ? n : 1, 256);
    // every round colours at least the highest-priority uncoloured node
    int64_t left = n;
    for (int64_t round = 0; left > 0; ++round) {
        if (round > n) return set_error(c, GR_ECUDA, "colouring: no progress");
        GR_TRY_CUDA(c, cudaMemsetAsync(ctr, 0, 4, s), "memset");
        k_jp_round<<<gn, 256, 0, s>>>(n, c->rowptr, c->col, colour_seed, colour, ctr, ctr + 1);
        count_launch();
        GR_TRY_CUDA(c, cudaMemcpyAsync(hs, ctr, 8, cudaMemcpyDeviceToHost, s), "readback");
        GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
        const int64_t now = ((int32_t*)hs)[0];
        if (now >= left) return set_error(c, GR_ECUDA, "colouring: a round made no progress");
        left = now;
    }
    const int32_t ncol = n > 0 ? ((int32_t*)hs)[1] + 1 : 0;
    // the nodes in ascending (colour, id): a stable sort of the ids by colour
    GR_TRY_CUDA(c, cudaMemsetAsync(cnt, 0, 4 * (size_t)(ncol + 1), s), "memset");
    if (n > 0) {
        k_colour_keys<<<gn, 256, 0, s>>>(n, colour, k0, v0, cnt);
        count_launch();
    }
    int alt = 0;
    GR_TRY_CUDA(c, radix_sort_u32(k0, v0, k1, v1, n, bits_for((uint64_t)(ncol > 1 ? ncol - 1 : 1)), c->ws, s, &alt),
                "sort by colour");
    GR_TRY_CUDA(c, scan_exclusive_i32(cnt, cptr, ncol + 1, c->ws, s), "scan");
    if (!c->gs_order) GR_TRY_CUDA(c, cudaMallocAsync(&c->gs_order, 4 * (size_t)(n > 0 ? n : 1), s), "alloc");
    GR_TRY_CUDA(c, cudaMemcpyAsync(c->gs_order, alt ? v1 : v0, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s), "copy");
    std::vector<int32_t> hp((size_t)ncol + 1);
    GR_TRY_CUDA(c, cudaMemcpyAsync(hp.data(), cptr, 4 * (size_t)(ncol + 1), cudaMemcpyDeviceToHost, s), "readback");
    GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
    c->gs_ptr.assign(hp.begin(), hp.end());
    c->gs_seed = colour_seed;
    c->gs_ready = true;
    return GR_OK;
}

gr_status colour_impl(gr_ctx* c, uint64_t colour_seed, int32_t* colour_out, int32_t* ncolours_out) {
    gr_status st = gs_prepare(c, colour_seed, colour_out);
    if (st != GR_OK) return st;
    *ncolours_out = (int32_t)c->gs_ptr.size() - 1;
    return GR_OK;
}

// Update the listed rows (one colour) in place: G lanes per row, one chunk
// each; the neighbours have other colours and are not written by this launch.
template <typename T, int K>
__global__ void __launch_bounds__(SM_THREADS) k_gs_class(int64_t cnt, const int32_t* __restrict__ rows,
                                                         const int64_t* __restrict__ rowptr,
                                                         const typename SlotOf<T>::type* __restrict__ slots,
                                                         T* __restrict__ X, double omega_d) {
    using Slot = typename SlotOf<T>::type;
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G, RPW = 32 / G;
    const int lane = threadIdx.x & 31, seg = lane / G, q = lane % G;
    if (seg >= RPW) return;
    const int64_t r = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW + seg;
    if (r >= cnt) return;
    const int64_t i = rows[r];
    const int64_t b = rowptr[i], e = rowptr[i + 1];
    const Acc omega = (Acc)omega_d, one_m = (Acc)(1.0 - omega_d);
    Acc xi[E];
    load_chunk<T, E>(X + i * K + q * E, xi);
    if (b == e) return;  // isolated: keeps its value
    Acc acc[E];
#pragma unroll
    for (int t = 0; t < E; ++t) acc[t] = Acc(0);
    for (int64_t j = b; j < e; j += 2) {
        const bool two = j + 1 < e;
        const Slot v0 = __ldg(slots + j);
        const Slot v1 = __ldg(slots + (two ? j + 1 : j));
        Acc x0[E], x1[E];
        load_chunk<T, E>(X + (int64_t)slot_col(v0) * K + q * E, x0);
        load_chunk<T, E>(X + (int64_t)slot_col(v1) * K + q * E, x1);
        const Acc w0 = slot_w(v0, Acc(0)), w1 = slot_w(v1, Acc(0));
#pragma unroll
        for (int t = 0; t < E; ++t) {
            acc[t] = fma(w0, x0[t], acc[t]);
            if (two) acc[t] = fma(w1, x1[t], acc[t]);
        }
    }
    Acc y[E];
#pragma unroll
    for (int t = 0; t < E; ++t) y[t] = one_m * xi[t] + omega * acc[t];
    store_chunk<T, E>(X + i * K + q * E, y);
}

// column sums and sums of squares of X (FP64 per-block partials, last-block finish)
template <typename T, int K>
__global__ void __launch_bounds__(SM_THREADS) k_col_stats(int64_t n, const T* __restrict__ A, double* __restrict__ part,
                                                          unsigned* __restrict__ counter,
                                                          double* __restrict__ stats_out) {
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G, GP = L::GP;
    constexpr int RPW = 32 / GP;
    const int lane = threadIdx.x & 31;
    const int q = lane % GP, seg = lane / GP;
    Acc s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) s1[e] = s2[e] = Acc(0);
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp_global * RPW; r0 < n; r0 += nwarps * RPW) {
        const int64_t row = r0 + seg;
        if (row < n && q < G) {
            Acc x[E];
            load_chunk<T, E>(A + row * K + q * E, x);
            add_sums<Acc, E>(s1, s2, x);
        }
    }
    block_stats<Acc, K, E, G, GP>(s1, s2, part, counter, n, stats_out);
}

// X = (X - mu) * inv_s in place, chunk-parallel (one pointer, plain loads)
template <typename T, int K>
__global__ void k_scale_inplace(int64_t n, T* X, const double* __restrict__ stats) {
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G;
    __shared__ Acc st[2 * K];
    for (int i = threadIdx.x; i < 2 * K; i += blockDim.x) st[i] = (Acc)stats[i];
    __syncthreads();
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * G) return;
    const int64_t row = idx / G;
    const int q = (int)(idx % G);
    T* p = X + row * K + q * E;
    Acc x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = (Acc)p[e];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = q * E + e;
        x[e] = (x[e] - st[k]) * st[K + k];
    }
    store_chunk<T, E>(p, x);
}

template <typename T, int K>
static gr_status run_smooth_gs(gr_ctx* c, int sweeps, double omega, uint64_t seed, int level, uint64_t colour_seed,
                               T* X) {
    if (!c->gs_ready || c->gs_seed != colour_seed) {
        gr_status st = gs_prepare(c, colour_seed, nullptr);
        if (st != GR_OK) return st;
    }
    cudaStream_t s = c->stream;
    const int64_t n = c->n;
    constexpr int G = RowLayout<T, K>::G;
    void *p_st, *p_part;
    GR_TRY_CUDA(c, c->ws.get(WS_SMOOTH_STATS, stats_bytes<K>(), &p_st), "scratch");
    double* st = (double*)p_st;
    unsigned* counter = (unsigned*)(st + 4 * K);
    const int igrid = init_grid<T, K>(c, n);
    GR_TRY_CUDA(c, c->ws.get(WS_SMOOTH_PART, sizeof(double) * 2 * K * (size_t)igrid, &p_part), "scratch");
    double* part = (double*)p_part;
    GR_TRY_CUDA(c, cudaMemsetAsync(counter, 0, STATS_COUNTER_BYTES, s), "memset");
    const typename SlotOf<T>::type* slots;
    if constexpr (sizeof(T) == 8) {
        if (!c->cw64) {
            GR_TRY_CUDA(c, cudaMallocAsync(&c->cw64, sizeof(int4) * (size_t)(2 * c->m > 0 ? 2 * c->m : 1), s),
                        "alloc");
            if (c->m > 0) {
                k_pack64<<<(unsigned)ceil_div(2 * c->m, 256), 256, 0, s>>>(2 * c->m, c->col, c->wn64, c->cw64);
                count_launch();
            }
        }
        slots = c->cw64;
    } else {
        slots = c->cw32;
    }
    const unsigned ga = (unsigned)ceil_div(n * G > 0 ? n * G : 1, 256);
    // X0, centred and normalised
    k_init<T, K><<<igrid, SM_THREADS, 0, s>>>(n, seed, (uint64_t)level, X, part, counter, st);
    count_launch();
    if (n > 0) {
        k_scale_inplace<T, K><<<ga, 256, 0, s>>>(n, X, st);
        count_launch();
    }
    constexpr int RPB = SM_WARPS * (32 / G);  // rows per block in k_gs_class
    for (int it = 0; it < sweeps; ++it) {
        for (size_t col = 0; col + 1 < c->gs_ptr.size(); ++col) {
            const int64_t b = c->gs_ptr[col], cnt = c->gs_ptr[col + 1] - b;
            if (cnt <= 0) continue;
            k_gs_class<T, K><<<(unsigned)ceil_div(cnt, RPB), SM_THREADS, 0, s>>>(cnt, c->gs_order + b, c->rowptr,
                                                                                slots, X, omega);
            count_launch();
        }
        k_col_stats<T, K><<<igrid, SM_THREADS, 0, s>>>(n, X, part, counter, st);
        count_launch();
        if (n > 0) {
            k_scale_inplace<T, K><<<ga, 256, 0, s>>>(n, X, st);
            count_launch();
        }
    }
    GR_TRY_CUDA(c, cudaGetLastError(), "gauss-seidel kernels");
    return GR_OK;
}

template <typename T>
static gr_status smooth_gs_typed(gr_ctx* c, int K, int sweeps, double omega, uint64_t seed, int level,
                                 uint64_t colour_seed, void* X) {
    switch (K) {
        case 4: return run_smooth_gs<T, 4>(c, sweeps, omega, seed, level, colour_seed, (T*)X);
        case 8: return run_smooth_gs<T, 8>(c, sweeps, omega, seed, level, colour_seed, (T*)X);
        case 16: return run_smooth_gs<T, 16>(c, sweeps, omega, seed, level, colour_seed, (T*)X);
        case 24: return run_smooth_gs<T, 24>(c, sweeps, omega, seed, level, colour_seed, (T*)X);
        case 32: return run_smooth_gs<T, 32>(c, sweeps, omega, seed, level, colour_seed, (T*)X);
    }
    return set_error(c, GR_EINVAL, "smooth_gs: unsupported K");
}

gr_status smooth_gs_impl(gr_ctx* c, int K, int sweeps, double omega, uint64_t seed, int level,
                         uint64_t colour_seed, gr_prec prec, void* X) {
    switch (prec) {
        case GR_F64: return smooth_gs_typed<double>(c, K, sweeps, omega, seed, level, colour_seed, X);
        case GR_F32: return smooth_gs_typed<float>(c, K, sweeps, omega, seed, level, colour_seed, X);
        case GR_BF16: return smooth_gs_typed<__nv_bfloat16>(c, K, sweeps, omega, seed, level, colour_seed, X);
        default: return set_error(c, GR_EINVAL, "smooth_gs: unknown precision");
    }
}

}  // namespace gr

// ---------------------------------------------------------------------------
// Allocation-free smoothing (graph_reduce_smooth_noalloc)
//
// Some callers may not allocate device memory once set up: code that runs
// while a stream is being captured into a CUDA graph, or under an allocator
// policy that forbids growth after initialisation.  This variant launches the
// same kernels as graph_reduce_smooth but takes its scratch (the second
// vector block, the column statistics and the per-block partial sums) from
// one file-scope device array instead of the context's workspace.  Every GPU
// that loads the library holds this array until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace gr {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device (the host
// symbol is only a stand-in and must never reach a kernel).
static void* g_noalloc_addr[64];
static std::mutex g_noalloc_mu;

static cudaError_t noalloc_scratch_addr(int device, void** out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        int prev = -1;
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[device] = p;
    }
    *out = g_noalloc_addr[device];
    return cudaSuccess;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename T, int K>
static gr_status run_smooth_noalloc(gr_ctx* c, int sweeps, double omega, uint64_t seed, int level,
                                    T* X) {
    const int64_t n = c->n;
    const int cap = part_capacity(c);
    // layout of the fixed array: [second vector block | statistics | partials |
    // launcher scratch (packed FP64 slots, row partition) the context lacks]
    const size_t b_buf = align256(sizeof(T) * (size_t)n * K);
    const size_t b_st = align256(stats_bytes<K>());
    const size_t b_part = align256(sizeof(double) * 2 * K * (size_t)cap);
    if (b_buf + b_st + b_part > NOALLOC_SCRATCH_BYTES)
        return set_error(c, GR_EINVAL,
                         "smooth_noalloc: n*K*sizeof(element) plus statistics exceeds the 32 MiB "
                         "allocation-free scratch");
    void* base = nullptr;
    cudaError_t e = noalloc_scratch_addr(c->device, &base);
    if (e != cudaSuccess) return cuda_error(c, e, "smooth_noalloc: scratch address");
    char* B = (char*)base;
    SweepScratch sc;
    sc.base = B + b_buf + b_st + b_part;
    sc.bytes = NOALLOC_SCRATCH_BYTES - (b_buf + b_st + b_part);
    e = run_sweeps<T, K>(c, sc, sweeps, omega, seed, level, X, (T*)B, (double*)(B + b_buf),
                         (double*)(B + b_buf + b_st), cap, nullptr, nullptr);
    if (e == cudaErrorMemoryAllocation)
        return set_error(c, GR_EINVAL,
                         "smooth_noalloc: the packed FP64 slots or the row partition of this graph do not "
                         "fit the rest of the 32 MiB allocation-free scratch");
    if (e != cudaSuccess) return cuda_error(c, e, "smooth_noalloc");
    return GR_OK;
}

template <typename T>
static gr_status smooth_noalloc_typed(gr_ctx* c, int K, int sweeps, double omega, uint64_t seed,
                                      int level, void* X) {
    switch (K) {
        case 4: return run_smooth_noalloc<T, 4>(c, sweeps, omega, seed, level, (T*)X);
        case 8: return run_smooth_noalloc<T, 8>(c, sweeps, omega, seed, level, (T*)X);
        case 16: return run_smooth_noalloc<T, 16>(c, sweeps, omega, seed, level, (T*)X);
        case 24: return run_smooth_noalloc<T, 24>(c, sweeps, omega, seed, level, (T*)X);
        case 32: return run_smooth_noalloc<T, 32>(c, sweeps, omega, seed, level, (T*)X);
    }
    return set_error(c, GR_EINVAL, "smooth_noalloc: K must be 4, 8, 16, 24 or 32");
}

}  // namespace gr

extern "C" gr_status graph_reduce_smooth_noalloc(gr_ctx* ctx, int K, int sweeps, double omega,
                                                 uint64_t seed, int level, gr_prec prec, void* X) {
    using namespace gr;
    if (!ctx) return set_error(nullptr, GR_EINVAL, "smooth_noalloc: ctx is NULL");
    if (sweeps < 0 || !(omega > 0.0 && omega <= 1.0))
        return set_error(ctx, GR_EINVAL, "smooth_noalloc: need sweeps >= 0 and 0 < omega <= 1");
    if (level < 0 || level >= (1 << 20)) return set_error(ctx, GR_EINVAL, "smooth_noalloc: level out of range");
    if (!X || ((uintptr_t)X & 15u)) return set_error(ctx, GR_EINVAL, "smooth_noalloc: X must be a 16-byte aligned device pointer");
    switch (prec) {
        case GR_F64: return smooth_noalloc_typed<double>(ctx, K, sweeps, omega, seed, level, X);
        case GR_F32: return smooth_noalloc_typed<float>(ctx, K, sweeps, omega, seed, level, X);
        case GR_BF16: return smooth_noalloc_typed<__nv_bfloat16>(ctx, K, sweeps, omega, seed, level, X);
    }
    return set_error(ctx, GR_EINVAL, "smooth_noalloc: bad precision");
}
