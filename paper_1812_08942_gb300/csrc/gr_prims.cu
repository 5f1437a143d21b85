// Device primitives: stream-ordered workspace, exclusive scan, stable LSD
// radix sort of (key, value) pairs.  Used by CSR construction, aggregation
// and Galerkin coarsening.
#include <atomic>

#include "gr_internal.cuh"

namespace gr {

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
cudaError_t Workspace::get(int slot, size_t bytes, void** out) {
    if ((int)slots.size() <= slot) slots.resize(slot + 1);
    Slot& s = slots[slot];
    if (bytes == 0) bytes = 16;
    if (s.bytes < bytes) {
        if (s.ptr) {
            cudaError_t e = cudaFreeAsync(s.ptr, stream);
            s.ptr = nullptr;
            s.bytes = 0;
            if (e != cudaSuccess) return e;
        }
        size_t want = bytes + bytes / 4;
        want = (want + 255) & ~size_t(255);
        cudaError_t e = cudaMallocAsync(&s.ptr, want, stream);
        if (e != cudaSuccess) {
            s.ptr = nullptr;
            return e;
        }
        s.bytes = want;
    }
    *out = s.ptr;
    return cudaSuccess;
}

void Workspace::release() {
    for (Slot& s : slots)
        if (s.ptr) cudaFreeAsync(s.ptr, stream);
    slots.clear();
}

int64_t* host_scratch() {
    static thread_local int64_t* buf = nullptr;
    if (!buf && cudaMallocHost(&buf, 64) != cudaSuccess) buf = nullptr;
    return buf;
}

void tune_mempool(int device) {
    static bool done[64] = {false};
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[device] = true;
}

int bits_for(uint64_t v) {
    int b = 1;
    while (b < 64 && (v >> b) != 0) ++b;
    return b;
}

// ---------------------------------------------------------------------------
// Exclusive scan: reduce tiles -> scan tile sums -> scan tiles with offsets
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T x, T* warp_tot, T* block_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        T t = lane < nw ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == 31) *block_total = ti;
    }
    __syncthreads();
    T r = warp_tot[warp] + inc - x;
    return r;
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t count, T* __restrict__ bsum) {
    __shared__ T red[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < count) s += in[idx];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += red[w];
        bsum[blockIdx.x] = t;
    }
}

// one block: exclusive scan of nb tile sums in place, chunk by chunk
template <typename T>
__global__ void k_scan_bsums(T* __restrict__ bsum, int64_t nb) {
    __shared__ T warp_tot[SCAN_THREADS / 32];
    __shared__ T total;
    T carry = 0;
    for (int64_t base = 0; base < nb; base += SCAN_THREADS) {
        int64_t idx = base + threadIdx.x;
        T x = idx < nb ? bsum[idx] : T(0);
        T ex = block_exclusive_scan<T>(x, warp_tot, &total);
        if (idx < nb) bsum[idx] = ex + carry;
        carry += total;
        __syncthreads();
    }
}

template <typename T>
__global__ void k_scan_apply(const T* __restrict__ in, T* __restrict__ out, int64_t count,
                             const T* __restrict__ bsum) {
    __shared__ T tile[SCAN_TILE];
    __shared__ T warp_tot[SCAN_THREADS / 32];
    __shared__ T total;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        tile[i * SCAN_THREADS + threadIdx.x] = idx < count ? in[idx] : T(0);
    }
    __syncthreads();
    T loc[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        loc[i] = s;
        s += tile[threadIdx.x * SCAN_ITEMS + i];
    }
    T ex = block_exclusive_scan<T>(s, warp_tot, &total) + bsum[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) tile[threadIdx.x * SCAN_ITEMS + i] = ex + loc[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + (int64_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < count) out[idx] = tile[i * SCAN_THREADS + threadIdx.x];
    }
}

template <typename T>
static cudaError_t scan_exclusive(const T* in, T* out, int64_t count, Workspace& ws,
                                  cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    int64_t nb = ceil_div(count, SCAN_TILE);
    void* p = nullptr;
    GR_CUDA(ws.get(WS_SCAN, sizeof(T) * (size_t)nb, &p));
    T* bsum = (T*)p;
    k_scan_reduce<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, count, bsum); count_launch();
    k_scan_bsums<T><<<1, SCAN_THREADS, 0, s>>>(bsum, nb); count_launch();
    k_scan_apply<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, count, bsum); count_launch();
    return cudaGetLastError();
}

cudaError_t scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t count, Workspace& ws,
                               cudaStream_t s) {
    return scan_exclusive<int64_t>(in, out, count, ws, s);
}
cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t count, Workspace& ws,
                               cudaStream_t s) {
    return scan_exclusive<int32_t>(in, out, count, ws, s);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.  Per pass: per-tile digit histogram,
// one exclusive scan over the digit-major histogram, then a stable scatter in
// which every warp ranks its keys chunk by chunk with __match_any_sync.
// ---------------------------------------------------------------------------
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_CHUNKS = 8;  // chunks of 32 keys per warp
constexpr int SORT_TILE = SORT_THREADS * SORT_CHUNKS;
static_assert(SORT_THREADS == RADIX, "the scatter handles one digit per thread");

template <typename KT>
__global__ void __launch_bounds__(SORT_THREADS) k_radix_hist(const KT* __restrict__ keys,
                                                             int64_t count, int shift,
                                                             int32_t* __restrict__ hist, int nb) {
    __shared__ int32_t cnt[RADIX];
    for (int d = threadIdx.x; d < RADIX; d += SORT_THREADS) cnt[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
#pragma unroll
    for (int i = 0; i < SORT_CHUNKS; ++i) {
        int64_t idx = base + (int64_t)i * SORT_THREADS + threadIdx.x;
        if (idx < count) atomicAdd(&cnt[(int)((keys[idx] >> shift) & (RADIX - 1))], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += SORT_THREADS) hist[(int64_t)d * nb + blockIdx.x] = cnt[d];
}

// Stable scatter of one tile.  Every warp ranks its 8 chunks of 32 keys per
// digit with __match_any_sync (warp order = input order); the block then
// places its keys in shared memory in (digit, input) order and writes them
// out sequentially, so consecutive threads store consecutive addresses of a
// digit's output run instead of scattering one key per lane.
template <typename KT>
__global__ void __launch_bounds__(SORT_THREADS) k_radix_scatter(
    const KT* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t count, int shift,
    const int32_t* __restrict__ offs, int nb, KT* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out) {
    __shared__ int32_t whist[SORT_WARPS][RADIX];  // counts, then smem bases per (warp, digit)
    __shared__ int32_t tstart[RADIX];            // tile-local start of each digit
    __shared__ int32_t gbase[RADIX];             // global start of this tile's run of each digit
    __shared__ int32_t wsum[SORT_WARPS];
    __shared__ KT skey[SORT_TILE];
    __shared__ uint32_t sval[SORT_TILE];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t tbase = (int64_t)blockIdx.x * SORT_TILE;
    const int64_t wbase = tbase + (int64_t)warp * 32 * SORT_CHUNKS;
    KT k[SORT_CHUNKS];
    uint32_t v[SORT_CHUNKS];
    int dig[SORT_CHUNKS], rnk[SORT_CHUNKS];
#pragma unroll
    for (int c = 0; c < SORT_CHUNKS; ++c) {
        const int64_t idx = wbase + c * 32 + lane;
        if (idx < count) {
            k[c] = keys[idx];
            v[c] = vals[idx];
            dig[c] = (int)((k[c] >> shift) & (RADIX - 1));
        } else {
            k[c] = 0;
            v[c] = 0;
            dig[c] = RADIX;  // sentinel: never touches shared memory
        }
    }
    for (int d = lane; d < RADIX; d += 32) whist[warp][d] = 0;
    __syncwarp();
    // rank of every key among the warp's keys of its digit
#pragma unroll
    for (int c = 0; c < SORT_CHUNKS; ++c) {
        const unsigned peers = __match_any_sync(0xffffffffu, dig[c]);
        const int leader = __ffs(peers) - 1;
        const int before = dig[c] < RADIX ? whist[warp][dig[c]] : 0;
        rnk[c] = before + __popc(peers & lt_mask);
        __syncwarp();
        if (lane == leader && dig[c] < RADIX) whist[warp][dig[c]] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit (one thread each): the tile's count, the warps' bases within
    // the digit, and the digit's global start
    const int d = threadIdx.x;  // SORT_THREADS == RADIX
    int32_t tot = 0;
    for (int w = 0; w < SORT_WARPS; ++w) {
        const int32_t c = whist[w][d];
        whist[w][d] = tot;
        tot += c;
    }
    gbase[d] = offs[(int64_t)d * nb + blockIdx.x];
    // exclusive scan of the digit totals over the block
    int32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    const int32_t start = wpre + incl - tot;
    tstart[d] = start;
    for (int w = 0; w < SORT_WARPS; ++w) whist[w][d] += start;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < SORT_CHUNKS; ++c) {
        if (dig[c] < RADIX) {
            const int32_t pos = whist[warp][dig[c]] + rnk[c];
            skey[pos] = k[c];
            sval[pos] = v[c];
        }
    }
    __syncthreads();
    int32_t total = 0;
    for (int w = 0; w < SORT_WARPS; ++w) total += wsum[w];
    for (int j = threadIdx.x; j < total; j += SORT_THREADS) {
        const KT key = skey[j];
        const int dj = (int)((key >> shift) & (RADIX - 1));
        const int32_t g = gbase[dj] + (j - tstart[dj]);
        keys_out[g] = key;
        vals_out[g] = sval[j];
    }
}

template <typename KT>
static cudaError_t radix_sort(KT* keys, uint32_t* vals, KT* keys_alt, uint32_t* vals_alt,
                              int64_t count, int bits, Workspace& ws, cudaStream_t s,
                              int* result_in_alt) {
    *result_in_alt = 0;
    if (count <= 1 || bits <= 0) return cudaSuccess;
    const int nb = (int)ceil_div(count, SORT_TILE);
    void* p = nullptr;
    GR_CUDA(ws.get(WS_SORT_HIST, sizeof(int32_t) * (size_t)RADIX * nb, &p));
    int32_t* hist = (int32_t*)p;
    KT* ki = keys;
    uint32_t* vi = vals;
    KT* ko = keys_alt;
    uint32_t* vo = vals_alt;
    int flips = 0;
    for (int shift = 0; shift < bits; shift += RADIX_BITS) {
        k_radix_hist<KT><<<nb, SORT_THREADS, 0, s>>>(ki, count, shift, hist, nb); count_launch();
        GR_CUDA(scan_exclusive_i32(hist, hist, (int64_t)RADIX * nb, ws, s));
        k_radix_scatter<KT><<<nb, SORT_THREADS, 0, s>>>(ki, vi, count, shift, hist, nb, ko, vo); count_launch();
        GR_CUDA(cudaGetLastError());
        KT* tk = ki; ki = ko; ko = tk;
        uint32_t* tv = vi; vi = vo; vo = tv;
        flips ^= 1;
    }
    *result_in_alt = flips;
    return cudaSuccess;
}

cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                           uint32_t* vals_alt, int64_t count, int bits, Workspace& ws,
                           cudaStream_t s, int* result_in_alt) {
    return radix_sort<uint32_t>(keys, vals, keys_alt, vals_alt, count, bits, ws, s, result_in_alt);
}
cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                           uint32_t* vals_alt, int64_t count, int bits, Workspace& ws,
                           cudaStream_t s, int* result_in_alt) {
    return radix_sort<uint64_t>(keys, vals, keys_alt, vals_alt, count, bits, ws, s, result_in_alt);
}

}  // namespace gr
