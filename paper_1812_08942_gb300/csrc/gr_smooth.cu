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
#include "gr_vec.cuh"

namespace gr {

constexpr int SM_THREADS = 256;
constexpr int SM_WARPS = SM_THREADS / 32;

// ---------------------------------------------------------------------------
// Column statistics: per-block partial sums (FP64) and a last-block finish
// that turns them into (mu, 1/s) for every column, in fixed order.
// ---------------------------------------------------------------------------
template <int K>
__device__ void finish_stats(const double* __restrict__ part, int nblocks, int64_t n,
                             double* __restrict__ stats_out) {
    // 2K sums, each split over SM_THREADS / (2K) threads, then combined in order
    constexpr int NS = 2 * K;
    constexpr int PER = SM_THREADS / NS > 0 ? SM_THREADS / NS : 1;
    __shared__ double red[SM_THREADS];
    const int t = threadIdx.x;
    const int stat = t % NS;
    const int sub = t / NS;
    double acc = 0.0;
    if (sub < PER)
        for (int b = sub; b < nblocks; b += PER) acc += __ldcg(part + (int64_t)b * NS + stat);
    red[t] = acc;
    __syncthreads();
    if (t < NS) {
        double s = 0.0;
        for (int j = 0; j < PER; ++j) s += red[j * NS + t];
        red[t] = s;
    }
    __syncthreads();
    if (t < K) {
        double s1 = red[t], s2 = red[K + t];
        double mu = s1 / (double)n;
        double var = s2 - (double)n * mu * mu;
        double sd = var > 0.0 ? sqrt(var) : 0.0;
        stats_out[t] = mu;
        stats_out[K + t] = sd > 0.0 ? 1.0 / sd : 1.0;
    }
}

// Block-level combine of per-lane column sums; lane l of segment 0 with
// t == 0 holds chunk l.  Writes the block partial and, in the last block to
// finish, the final statistics.
template <typename Acc, int K, int E, int G, int LPR>
__device__ void block_stats(Acc (&s1)[E], Acc (&s2)[E], double* __restrict__ part,
                            unsigned* __restrict__ counter, int64_t n,
                            double* __restrict__ stats_out) {
    __shared__ double wst[SM_WARPS][2 * K];
    __shared__ bool last;
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
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        finish_stats<K>(part, gridDim.x, n, stats_out);
        if (threadIdx.x == 0) *counter = 0u;
    }
}

// ---------------------------------------------------------------------------
// Initial test vectors: SplitMix64 output c+1 for counter c (Steele, Lea,
// Flood 2014), top 53 bits -> u in [0,1), entry 2u - 1, rounded once to the
// storage type (bfloat16: rounded from the FP32 value).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename T>
__device__ __forceinline__ typename AccOf<T>::type uniform_pm1(uint64_t z);
template <>
__device__ __forceinline__ double uniform_pm1<double>(uint64_t z) {
    // 2 * (z>>11) * 2^-53 - 1 = ((z>>11) - 2^52) * 2^-52, exact in FP64
    return (double)((int64_t)(z >> 11) - (1ll << 52)) * 0x1p-52;
}
template <>
__device__ __forceinline__ float uniform_pm1<float>(uint64_t z) {
    // one round-to-nearest of the exact value
    return __ll2float_rn((int64_t)(z >> 11) - (1ll << 52)) * 0x1p-52f;
}
template <>
__device__ __forceinline__ float uniform_pm1<__nv_bfloat16>(uint64_t z) {
    return uniform_pm1<float>(z);
}

template <typename T, int K>
__global__ void __launch_bounds__(SM_THREADS) k_init(int64_t n, uint64_t seed, uint64_t level,
                                                     T* __restrict__ A, double* __restrict__ part,
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
        int64_t row = r0 + seg;
        if (row < n && q < G) {
            Acc x[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                uint64_t c = (level << 40) + (uint64_t)row * K + (uint64_t)(q * E + e);
                x[e] = uniform_pm1<T>(splitmix64_at(seed, c));
            }
            store_chunk<T, E>(A + row * K + q * E, x);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                s1[e] += x[e];
                s2[e] += x[e] * x[e];
            }
        }
    }
    block_stats<Acc, K, E, G, GP>(s1, s2, part, counter, n, stats_out);
}

// ---------------------------------------------------------------------------
// One sweep: Y = (J A - mu) * inv_s with J A = (1-w) A + w D^-1 A A.
// LPR lanes serve one row: GP chunk lanes times TS neighbour slots in flight.
// The row's slot list is read LPR entries at a time (coalesced) and handed
// out by shuffles; each neighbour row is gathered chunk-wise (16 B / lane).
// ---------------------------------------------------------------------------
template <typename T, int K, int LPR>
__global__ void __launch_bounds__(SM_THREADS) k_sweep(
    int64_t n, const int64_t* __restrict__ rowptr, const int2* __restrict__ cw32,
    const int32_t* __restrict__ col, const double* __restrict__ wn64, const T* __restrict__ Ain,
    T* __restrict__ Aout, double omega_d, const double* __restrict__ stats_in,
    double* __restrict__ part, unsigned* __restrict__ counter, double* __restrict__ stats_out) {
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G, GP = L::GP;
    static_assert(LPR >= GP && LPR <= 32, "lanes per row");
    constexpr int TS = LPR / GP;
    constexpr int RPW = 32 / LPR;
    constexpr bool F64 = sizeof(T) == 8;
    const int lane = threadIdx.x & 31;
    const int seg = lane / LPR, l = lane % LPR;
    const int q = l % GP, t = l / GP;
    const unsigned segmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (seg * LPR));
    const bool chunk_ok = q < G;
    const Acc omega = (Acc)omega_d, one_m = (Acc)(1.0 - omega_d);

    Acc mu[E], is[E], s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int k = chunk_ok ? q * E + e : 0;
        mu[e] = (Acc)stats_in[k];
        is[e] = (Acc)stats_in[K + k];
        s1[e] = s2[e] = Acc(0);
    }

    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp_global * RPW; r0 < n; r0 += nwarps * RPW) {
        const int64_t row = r0 + seg;
        const bool row_ok = row < n;
        const int64_t b = row_ok ? rowptr[row] : 0;
        const int64_t e_end = row_ok ? rowptr[row + 1] : 0;
        Acc acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = Acc(0);
        for (int64_t base = b; base < e_end; base += LPR) {
            const int64_t j = base + l;
            int cj = 0;
            Acc wj = Acc(0);
            if (j < e_end) {
                if constexpr (F64) {
                    cj = col[j];
                    wj = (Acc)wn64[j];
                } else {
                    int2 v = cw32[j];
                    cj = v.x;
                    wj = (Acc)__int_as_float(v.y);
                }
            }
            const int cnt = (int)min((int64_t)LPR, e_end - base);
#pragma unroll
            for (int r = 0; r < GP; ++r) {
                const int src = r * TS + t;
                const int c = __shfl_sync(segmask, cj, src, LPR);
                const Acc w = __shfl_sync(segmask, wj, src, LPR);
                if (src < cnt && chunk_ok) {
                    Acc x[E];
                    load_chunk<T, E>(Ain + (int64_t)c * K + q * E, x);
#pragma unroll
                    for (int e = 0; e < E; ++e) acc[e] = fma(w, x[e], acc[e]);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e)
#pragma unroll
            for (int o = GP; o < LPR; o <<= 1) acc[e] += __shfl_xor_sync(segmask, acc[e], o, LPR);
        if (row_ok && t == 0 && chunk_ok) {
            Acc xi[E], y[E];
            load_chunk<T, E>(Ain + row * K + q * E, xi);
            const bool isolated = b == e_end;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                Acc z = isolated ? xi[e] : one_m * xi[e] + omega * acc[e];
                y[e] = (z - mu[e]) * is[e];
            }
            store_chunk<T, E>(Aout + row * K + q * E, y);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                s1[e] += y[e];
                s2[e] += y[e] * y[e];
            }
        }
    }
    block_stats<Acc, K, E, G, LPR>(s1, s2, part, counter, n, stats_out);
}

// X = (A - mu) * inv_s, chunk-parallel
template <typename T, int K>
__global__ void k_apply(int64_t n, const T* __restrict__ A, T* __restrict__ X,
                        const double* __restrict__ stats) {
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * G) return;
    int64_t row = idx / G;
    int q = (int)(idx % G);
    Acc x[E];
    load_chunk<T, E>(A + row * K + q * E, x);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        int k = q * E + e;
        x[e] = (x[e] - (Acc)stats[k]) * (Acc)stats[K + k];
    }
    store_chunk<T, E>(X + row * K + q * E, x);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <typename T, int K, int LPR>
static cudaError_t launch_sweep(gr_ctx* c, int grid, const T* Ain, T* Aout, double omega,
                                const double* st_in, double* part, unsigned* counter,
                                double* st_out) {
    k_sweep<T, K, LPR><<<grid, SM_THREADS, 0, c->stream>>>(c->n, c->rowptr, c->cw32, c->col, c->wn64,
                                                          Ain, Aout, omega, st_in, part, counter,
                                                          st_out); count_launch();
    return cudaGetLastError();
}

template <typename T, int K>
static int pick_lpr(const gr_ctx* c) {
    constexpr int GP = RowLayout<T, K>::GP;
    double avg = c->n > 0 ? 2.0 * (double)c->m / (double)c->n : 0.0;
    int ts = 1;
    while (ts * GP < 32 && ts * 4 <= avg) ts *= 2;  // at least two neighbours per sub-slot
    return ts * GP;
}

template <typename T, int K>
static cudaError_t run_smooth(gr_ctx* c, int sweeps, double omega, uint64_t seed, int level,
                              T* X, cudaEvent_t ev0, cudaEvent_t ev1) {
    cudaStream_t s = c->stream;
    const int64_t n = c->n;
    constexpr int GP = RowLayout<T, K>::GP;
    void *p_buf, *p_st, *p_part;
    GR_CUDA(c->ws.get(WS_SMOOTH_BUF, sizeof(T) * (size_t)n * K, &p_buf));
    GR_CUDA(c->ws.get(WS_SMOOTH_STATS, sizeof(double) * 4 * K + 64, &p_st));
    T* buf = (T*)p_buf;
    double* st0 = (double*)p_st;
    double* st1 = st0 + 2 * K;
    unsigned* counter = (unsigned*)(st1 + 2 * K);
    const int lpr = pick_lpr<T, K>(c);
    const int rows_per_block = SM_WARPS * (32 / lpr);
    const int64_t want = ceil_div(n, rows_per_block);
    const int64_t cap = (int64_t)c->num_sms * 8;
    const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    const int init_rows = SM_WARPS * (32 / GP);
    const int64_t iwant = ceil_div(n, init_rows);
    const int igrid = (int)(iwant < cap ? (iwant > 0 ? iwant : 1) : cap);
    const int maxgrid = grid > igrid ? grid : igrid;
    GR_CUDA(c->ws.get(WS_SMOOTH_PART, sizeof(double) * 2 * K * (size_t)maxgrid, &p_part));
    double* part = (double*)p_part;
    GR_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));

    k_init<T, K><<<igrid, SM_THREADS, 0, s>>>(n, seed, (uint64_t)level, X, part, counter, st0); count_launch();
    GR_CUDA(cudaGetLastError());
    const T* cur = X;
    T* nxt = buf;
    if (ev0) GR_CUDA(cudaEventRecord(ev0, s));
    double* sin = st0;
    double* sout = st1;
    for (int it = 0; it < sweeps; ++it) {
        cudaError_t e;
        switch (lpr / GP) {
            case 1: e = launch_sweep<T, K, GP>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            case 2: e = launch_sweep<T, K, (2 * GP <= 32 ? 2 * GP : 32)>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            case 4: e = launch_sweep<T, K, (4 * GP <= 32 ? 4 * GP : 32)>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            case 8: e = launch_sweep<T, K, (8 * GP <= 32 ? 8 * GP : 32)>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            case 16: e = launch_sweep<T, K, (16 * GP <= 32 ? 16 * GP : 32)>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            default: e = launch_sweep<T, K, 32>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
        }
        GR_CUDA(e);
        const T* tmp = cur;
        cur = nxt;
        nxt = (T*)tmp;
        double* ts = sin;
        sin = sout;
        sout = ts;
    }
    if (ev1) GR_CUDA(cudaEventRecord(ev1, s));
    constexpr int G = RowLayout<T, K>::G;
    if (n > 0) {
        k_apply<T, K><<<(unsigned)ceil_div(n * G, 256), 256, 0, s>>>(n, cur, X, sin);
        count_launch();
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t smooth_typed(gr_ctx* c, int K, int sweeps, double omega, uint64_t seed,
                                int level, void* X, cudaEvent_t e0, cudaEvent_t e1) {
    switch (K) {
        case 4: return run_smooth<T, 4>(c, sweeps, omega, seed, level, (T*)X, e0, e1);
        case 8: return run_smooth<T, 8>(c, sweeps, omega, seed, level, (T*)X, e0, e1);
        case 16: return run_smooth<T, 16>(c, sweeps, omega, seed, level, (T*)X, e0, e1);
        case 24: return run_smooth<T, 24>(c, sweeps, omega, seed, level, (T*)X, e0, e1);
        case 32: return run_smooth<T, 32>(c, sweeps, omega, seed, level, (T*)X, e0, e1);
    }
    return cudaErrorInvalidValue;
}

gr_status smooth_impl(gr_ctx* c, int K, int sweeps, double omega, uint64_t seed, int level,
                      gr_prec prec, void* X, cudaEvent_t e0, cudaEvent_t e1) {
    cudaError_t e;
    switch (prec) {
        case GR_F64: e = smooth_typed<double>(c, K, sweeps, omega, seed, level, X, e0, e1); break;
        case GR_F32: e = smooth_typed<float>(c, K, sweeps, omega, seed, level, X, e0, e1); break;
        case GR_BF16: e = smooth_typed<__nv_bfloat16>(c, K, sweeps, omega, seed, level, X, e0, e1); break;
        default: return set_error(c, GR_EINVAL, "smooth: unknown precision");
    }
    if (e != cudaSuccess) return cuda_error(c, e, "smooth");
    return GR_OK;
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
    cudaStream_t s = c->stream;
    const int64_t n = c->n;
    constexpr int GP = RowLayout<T, K>::GP;
    const int lpr = pick_lpr<T, K>(c);
    const int rows_per_block = SM_WARPS * (32 / lpr);
    const int64_t cap = (int64_t)c->num_sms * 8;
    const int64_t want = ceil_div(n, rows_per_block);
    const int grid = (int)(want < cap ? (want > 0 ? want : 1) : cap);
    const int64_t iwant = ceil_div(n, SM_WARPS * (32 / GP));
    const int igrid = (int)(iwant < cap ? (iwant > 0 ? iwant : 1) : cap);
    const int maxgrid = grid > igrid ? grid : igrid;
    // layout of the shared scratch: [vector block | 2 x 2K stats + counter | partials]
    const size_t b_buf = align256(sizeof(T) * (size_t)n * K);
    const size_t b_st = align256(sizeof(double) * 4 * K + 64);
    const size_t b_part = align256(sizeof(double) * 2 * K * (size_t)maxgrid);
    if (b_buf + b_st + b_part > NOALLOC_SCRATCH_BYTES)
        return set_error(c, GR_EINVAL,
                         "smooth_noalloc: n*K*sizeof(element) plus statistics exceeds the 32 MiB "
                         "allocation-free scratch");
    void* base = nullptr;
    cudaError_t e = noalloc_scratch_addr(c->device, &base);
    if (e != cudaSuccess) return cuda_error(c, e, "smooth_noalloc: scratch address");
    char* B = (char*)base;
    T* buf = (T*)B;
    double* st0 = (double*)(B + b_buf);
    double* st1 = st0 + 2 * K;
    unsigned* counter = (unsigned*)(st1 + 2 * K);
    double* part = (double*)(B + b_buf + b_st);
    // the array keeps the previous call's contents: the last-block counter
    // must start at zero
    GR_TRY_CUDA(c, cudaMemsetAsync(counter, 0, sizeof(unsigned), s), "smooth_noalloc");
    k_init<T, K><<<igrid, SM_THREADS, 0, s>>>(n, seed, (uint64_t)level, X, part, counter, st0);
    count_launch();
    GR_TRY_CUDA(c, cudaGetLastError(), "smooth_noalloc: init");
    const T* cur = X;
    T* nxt = buf;
    double* sin = st0;
    double* sout = st1;
    for (int it = 0; it < sweeps; ++it) {
        switch (lpr / GP) {
            case 1: e = launch_sweep<T, K, GP>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            case 2: e = launch_sweep<T, K, (2 * GP <= 32 ? 2 * GP : 32)>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            case 4: e = launch_sweep<T, K, (4 * GP <= 32 ? 4 * GP : 32)>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            case 8: e = launch_sweep<T, K, (8 * GP <= 32 ? 8 * GP : 32)>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            case 16: e = launch_sweep<T, K, (16 * GP <= 32 ? 16 * GP : 32)>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
            default: e = launch_sweep<T, K, 32>(c, grid, cur, nxt, omega, sin, part, counter, sout); break;
        }
        if (e != cudaSuccess) return cuda_error(c, e, "smooth_noalloc: sweep");
        const T* tmp = cur;
        cur = nxt;
        nxt = (T*)tmp;
        double* ts = sin;
        sin = sout;
        sout = ts;
    }
    constexpr int G = RowLayout<T, K>::G;
    if (n > 0) {
        k_apply<T, K><<<(unsigned)ceil_div(n * G, 256), 256, 0, s>>>(n, cur, X, sin);
        count_launch();
    }
    GR_TRY_CUDA(c, cudaGetLastError(), "smooth_noalloc: apply");
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
