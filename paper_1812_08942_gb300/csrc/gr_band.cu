// Band sweep: one weighted-Jacobi sweep Y = (J A - mu) / s of the test-vector
// block (Alg. 3, Sec. 3.2.1) for graphs whose neighbours mostly lie within H
// rows of the row itself, apart from a few far ranges (banded orderings:
// meshes and grids, whose far neighbours are the next and previous planes).
//
// The rows are cut into bands of R consecutive rows, the bands into chunks of
// BAND_CB consecutive bands; each block runs its chunks' bands in order,
// chunks grid-strided (all blocks work on one front of rows, so the far
// planes stay in L2).  A producer warp moves, per band, with bulk copies on
// the copy engine (completion counted in bytes on an mbarrier):
//   - the band's R + 1 row pointers and its slots into a stage,
//   - the window rows [r0 - H, r0 + R + H) not yet held into a ring buffer of
//     vector rows: a chunk's first band loads its whole window, every later
//     band only the R rows that enter it, so each vector row is read once,
//   - the two far runs of the band -- the column range of its neighbours
//     below the window and the range above it -- into the stage's part of a
//     far area, when each is at most FC rows long.
// Three stages are in flight.  Where each slot's neighbour will sit in shared
// memory depends only on the plan and the grid, so a per-plan pass stores it
// in the slot in place of the column (-(column + 1) when it is read from
// global memory); the consumer warps (band_cw: 15 or 16) then gather every
// neighbour with one shared-memory load and turn the band into output rows.
//
// Products are added in slot order exactly as in the row-group kernel, so the
// sweep result equals that kernel's given the same statistics.  Every wait is
// bounded (about a second of clock cycles); a wait that runs out sets the
// error word, the block drains its own copies and returns, and its NaN
// partials make every later output NaN.
#include <cuda_bf16.h>

#include <limits.h>

#include "gr_internal.cuh"
#include "gr_sweep.cuh"
#include "gr_vec.cuh"

namespace gr {

// Consumer warps per block: 15 (with the producer, four warps per SM
// sub-partition and 128 registers a thread), or 16 for FP32 blocks of 24
// columns, where a 17th warp still fits the 96 registers the kernel needs and
// the larger band fits 224 KB (measured: 117 against 122 us per sweep on the
// 128^3 mesh; the other shapes ran slower with 16)
template <typename T, int K>
__host__ __device__ constexpr int band_cw() { return sizeof(T) == 4 && K == 24 ? 16 : 15; }
template <typename T, int K>
__host__ __device__ constexpr int band_threads() { return (band_cw<T, K>() + 1) * 32; }
template <typename T, int K>
__host__ __device__ constexpr int band_smem_max() { return (band_cw<T, K>() == 16 ? 224 : 216) * 1024; }
constexpr int BAND_NS = 3;                         // stages in flight
constexpr int BAND_CB = 8;                         // consecutive bands per chunk
constexpr long long BAND_WAIT_CYCLES = 2000000000ll;  // ~1 s at 2 GHz

// ---------------------------------------------------------------------------
// Asynchronous copies and mbarriers (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(sm_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(sm_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bulk copy global -> shared on the copy engine; 16-byte aligned addresses,
// size a multiple of 16; completion counted in bytes on mbarrier b
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(sm_addr(b))
                 : "memory");
}
// bounded wait for the phase of parity `par`; gives up when another thread
// has given up (*abort) or after BAND_WAIT_CYCLES (then sets *abort)
__device__ bool mbar_wait(uint64_t* b, uint32_t par, volatile int* abort) {
    if (mbar_test(b, par)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_test(b, par)) return true;
        if (abort && *abort) return false;
        if (clock64() - t0 > BAND_WAIT_CYCLES) {
            if (abort) *abort = 1;
            return false;
        }
    }
}

// 16-byte chunk of a vector row from shared memory, in the accumulator type
template <typename T, int E>
__device__ __forceinline__ void lds_chunk(uint32_t a, typename AccOf<T>::type (&x)[E]) {
    if constexpr (sizeof(T) == 8) {
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(x[0]), "=d"(x[1]) : "r"(a));
    } else if constexpr (sizeof(T) == 4) {
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3])
                     : "r"(a));
    } else {
        uint32_t v[4];
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                     : "r"(a));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&v[i]));
            x[2 * i] = f.x;
            x[2 * i + 1] = f.y;
        }
    }
}

// ---------------------------------------------------------------------------
// Band geometry, shared by the sweep kernel's producer and the per-plan
// passes that precompute where each slot's neighbour sits.
// ---------------------------------------------------------------------------
// rows [r0, r0 + nrows) of band b and its window [w0, w1)
__device__ __forceinline__ void band_rows(int b, int n, int R, int H, int& r0, int& nrows, int& w0, int& w1) {
    r0 = b * R;
    nrows = min(R, n - r0);
    w0 = max(0, r0 - H);
    w1 = min(n, r0 + nrows + H);
}
// number of bands block `blk` of `grid` runs, and its k-th band
__device__ __forceinline__ int band_count(int blk, int grid, int nbands) {
    int nb = 0;
    for (int ch = blk; ch * BAND_CB < nbands; ch += grid) nb += min(BAND_CB, nbands - ch * BAND_CB);
    return nb;
}
__device__ __forceinline__ int band_at(int blk, int grid, int k) { return (blk + (k / BAND_CB) * grid) * BAND_CB + k % BAND_CB; }

// Ring placement.  A block's ring holds WR vector rows; a chunk's first band
// loads its whole window from the ring's next free position, every later band
// of the chunk the rows past the previous window.  For a band with window
// [w0, w1): pw0 = ring position of row w0, la = first row loaded, p = its
// ring position (positions wrap modulo WR).
struct RingState {
    int vpos = 0, w0 = 0, w1 = 0, pw0 = 0;
};
__device__ __forceinline__ void ring_place(RingState& s, bool first, int w0, int w1, int WR, int& pw0, int& la,
                                           int& p) {
    if (first) {
        la = w0;
        pw0 = s.vpos;
        p = s.vpos;
    } else {
        la = s.w1;
        pw0 = (s.pw0 + (w0 - s.w0)) % WR;
        p = (pw0 + (la - w0)) % WR;
    }
    s.vpos = (p + (w1 - la)) % WR;
    s.w0 = w0;
    s.w1 = w1;
    s.pw0 = pw0;
}
// rows of a far run held in shared memory: the run, if it fits FC rows
__device__ __forceinline__ int far_held(int len, int FC) { return len <= FC ? len : 0; }

// ---------------------------------------------------------------------------
// Per-plan passes
// ---------------------------------------------------------------------------
// Far runs per band b: the column range of its neighbours below its window
// and the range above it, {lo, lo_len, hi, hi_len}.  Warp per band.
__global__ void k_band_runs(int n, int nbands, int R, int H, const int64_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, int4* __restrict__ runs) {
    const int lane = threadIdx.x & 31;
    const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (b >= nbands) return;
    int r0, nrows, w0, w1;
    band_rows(b, n, R, H, r0, nrows, w0, w1);
    int lo_min = INT_MAX, lo_max = -1, hi_min = INT_MAX, hi_max = -1;
    for (int64_t j = rowptr[r0] + lane; j < rowptr[r0 + nrows]; j += 32) {
        const int c = col[j];
        if (c < w0) {
            lo_min = min(lo_min, c);
            lo_max = max(lo_max, c);
        } else if (c >= w1) {
            hi_min = min(hi_min, c);
            hi_max = max(hi_max, c);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo_min = min(lo_min, __shfl_xor_sync(0xffffffffu, lo_min, o));
        lo_max = max(lo_max, __shfl_xor_sync(0xffffffffu, lo_max, o));
        hi_min = min(hi_min, __shfl_xor_sync(0xffffffffu, hi_min, o));
        hi_max = max(hi_max, __shfl_xor_sync(0xffffffffu, hi_max, o));
    }
    if (lane == 0)
        runs[b] = make_int4(lo_max >= 0 ? lo_min : 0, lo_max >= 0 ? lo_max - lo_min + 1 : 0,
                            hi_max >= 0 ? hi_min : 0, hi_max >= 0 ? hi_max - hi_min + 1 : 0);
}

// Ring position of each band's window and its stage: thread per block of the
// sweep grid, walking that block's bands in the sweep's order.
__global__ void k_band_layout(int n, int nbands, int grid, int R, int H, int WR, int2* __restrict__ lay) {
    const int blk = blockIdx.x * blockDim.x + threadIdx.x;
    if (blk >= grid) return;
    const int nb = band_count(blk, grid, nbands);
    RingState rs;
    for (int k = 0; k < nb; ++k) {
        const int b = band_at(blk, grid, k);
        int r0, nrows, w0, w1, pw0, la, p;
        band_rows(b, n, R, H, r0, nrows, w0, w1);
        ring_place(rs, (k % BAND_CB) == 0, w0, w1, WR, pw0, la, p);
        lay[b] = make_int2(pw0, k % BAND_NS);
    }
}

// Shared-memory row of every slot's neighbour for one plan: the ring
// position inside the band's window, else the row of the band's stage in the
// far area (lo run, then hi run), else -(column + 1): read from global
// memory.  FP32 / BF16 blocks get (row, weight bits) pairs, FP64 blocks the
// rows alone (the weights stay in wn64).  *nglobal counts the slots read
// from global memory.  Warp per band.
template <bool F64>
__global__ void k_band_slots(int n, int nbands, int R, int H, int WR, int FC, const int64_t* __restrict__ rowptr,
                             const int32_t* __restrict__ col, const int2* __restrict__ cw32,
                             const int4* __restrict__ runs, const int2* __restrict__ lay, void* __restrict__ out,
                             unsigned long long* __restrict__ nglobal) {
    const int lane = threadIdx.x & 31;
    const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (b >= nbands) return;
    int r0, nrows, w0, w1;
    band_rows(b, n, R, H, r0, nrows, w0, w1);
    const int4 run = runs[b];
    const int2 ly = lay[b];
    const int nlo = far_held(run.y, FC), nhi = far_held(run.w, FC);
    const int far0 = WR + ly.y * 2 * FC;
    unsigned ng = 0;
    for (int64_t j = rowptr[r0] + lane; j < rowptr[r0 + nrows]; j += 32) {
        const int c = col[j];
        int u;
        if (c >= w0 && c < w1) {
            u = ly.x + (c - w0);
            if (u >= WR) u -= WR;
        } else if (c >= run.x && c < run.x + nlo) {
            u = far0 + (c - run.x);
        } else if (c >= run.z && c < run.z + nhi) {
            u = far0 + FC + (c - run.z);
        } else {
            u = -(c + 1);
            ++ng;
        }
        if constexpr (F64) reinterpret_cast<int32_t*>(out)[j] = u;
        else reinterpret_cast<int2*>(out)[j] = make_int2(u, cw32[j].y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ng += __shfl_xor_sync(0xffffffffu, ng, o);
    if (lane == 0 && ng) atomicAdd(nglobal, (unsigned long long)ng);
}

// ---------------------------------------------------------------------------
// Locality profile: histogram of |c - r| over all slots in log2 buckets
// ---------------------------------------------------------------------------
// A warp takes 32 consecutive rows: their slots are one contiguous range,
// which the lanes run over a slot each (the row of each slot from a
// shared-memory map); ranges longer than HIST_CAP slots are run row by row.
constexpr int HIST_CAP = 1024;

__global__ void __launch_bounds__(256) k_offset_hist(int64_t n, const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ col,
                                                     unsigned long long* __restrict__ hist) {
    __shared__ unsigned int sh[33];
    __shared__ uint8_t s_row[8][HIST_CAP];
    constexpr unsigned FULL = 0xffffffffu;
    for (int i = threadIdx.x; i < 33; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    auto bucket = [](int64_t d) {
        const int bk = d <= 1 ? 0 : 64 - __clzll((long long)(d - 1));
        return bk < 32 ? bk : 32;
    };
    for (int64_t pw = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)); pw < n;
         pw += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = pw + lane;
        const bool in = r < n;
        const int64_t b = in ? rowptr[r] : 0, e = in ? rowptr[r + 1] : 0;
        const int lv = (int)((n - pw < 32 ? n - pw : 32) - 1);
        const int64_t R0 = __shfl_sync(FULL, b, 0), R1 = __shfl_sync(FULL, e, lv);
        if (R1 - R0 <= HIST_CAP) {
            uint8_t* S = s_row[wp];
            for (int64_t j = b; j < e; ++j) S[j - R0] = (uint8_t)lane;
            __syncwarp();
            const int ns = (int)(R1 - R0);
            for (int j0 = 0; j0 < ns; j0 += 32) {
                const int j = j0 + lane;
                const int bk = j < ns ? bucket(llabs((int64_t)col[R0 + j] - (pw + S[j]))) : -1;
                // one shared atomic per bucket among the warp's lanes
                const unsigned peers = __match_any_sync(FULL, bk);
                if (bk >= 0 && lane == __ffs(peers) - 1) atomicAdd(&sh[bk], (unsigned)__popc(peers));
            }
            __syncwarp();
        } else {
            for (int64_t j = b; j < e; ++j) atomicAdd(&sh[bucket(llabs((int64_t)col[j] - r))], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 33; i += blockDim.x)
        if (sh[i]) atomicAdd(hist + i, (unsigned long long)sh[i]);
}

cudaError_t ensure_locality(gr_ctx* c, void* scratch264) {
    if (c->loc_ready) return cudaSuccess;
    unsigned long long* hist = (unsigned long long*)scratch264;
    GR_CUDA(cudaMemsetAsync(hist, 0, 33 * sizeof(unsigned long long), c->stream));
    if (c->n > 0 && c->m > 0) {
        const int64_t want = ceil_div(c->n, 256), cap = (int64_t)c->num_sms * 8;
        k_offset_hist<<<(unsigned)(want < cap ? want : cap), 256, 0, c->stream>>>(c->n, c->rowptr, c->col, hist);
        count_launch();
        GR_CUDA(cudaGetLastError());
    }
    unsigned long long h[33];
    GR_CUDA(cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    GR_CUDA(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 33; ++i) c->loc_hist[i] = h[i];
    c->loc_ready = true;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Sweep kernel
// ---------------------------------------------------------------------------
struct BandMeta {
    int64_t s0a;  // first slot copied (the band's first slot rounded down to 4)
    int r0, nrows;
    int w0, pw0;  // window start and its ring position
    int nsc;      // local slots [0, nsc) are held in the stage
};

template <typename T>
struct BandArgs {
    const int64_t* rowptr;
    const int2* bs32;     // FP32 / BF16 blocks: (shared row or -(column + 1), FP32 weight bits)
    const int32_t* bs64;  // FP64 blocks: shared row or -(column + 1) ...
    const double* wn64;   // ... and the FP64 weight
    const int4* runs;     // far runs per band
    const T* Ain;
    T* Aout;
    const double* stats_in;
    double* part;
    unsigned* counter;
    double* stats_out;
    int* err;
    double omega;
    int64_t n64;
    int n, nbands, R, H, SC, FC, WR;
    int off_stage, stage_bytes, off_sw;
};

// Neighbour chunk of slot value v: shared row v, or column -(v + 1) of the
// input block in global memory.
template <typename T, int K>
__device__ __forceinline__ void band_gather(int v, uint32_t rows_q, const T* Aq,
                                            typename AccOf<T>::type (&x)[RowLayout<T, K>::E]) {
    constexpr int E = RowLayout<T, K>::E, RB = RowLayout<T, K>::RB;
    if (v >= 0) lds_chunk<T, E>(rows_q + (uint32_t)v * RB, x);
    else load_chunk<T, E>(Aq + (size_t)(-(v + 1)) * K, x);
}

// U consecutive slots j ... j + U - 1 of a stage (slot values in sl, FP64
// weights in sw; FP32 weights beside the values), added to acc in slot
// order; one branch for the group when all its neighbours are in shared memory.
template <typename T, int K, int U>
__device__ __forceinline__ void band_group(const unsigned char* sl, const unsigned char* sw, int j, uint32_t rows_q,
                                           const T* Aq, typename AccOf<T>::type (&acc)[RowLayout<T, K>::E]) {
    using Acc = typename AccOf<T>::type;
    constexpr int E = RowLayout<T, K>::E, RB = RowLayout<T, K>::RB;
    int v[U];
    Acc w[U];
    Acc x[U][E];
    int any = 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if constexpr (sizeof(T) == 8) {
            v[u] = reinterpret_cast<const int32_t*>(sl)[j + u];
            w[u] = reinterpret_cast<const double*>(sw)[j + u];
        } else {
            const int2 t = reinterpret_cast<const int2*>(sl)[j + u];
            v[u] = t.x;
            w[u] = (Acc)__int_as_float(t.y);
        }
        any |= v[u];
    }
    if (any >= 0) {
#pragma unroll
        for (int u = 0; u < U; ++u) lds_chunk<T, E>(rows_q + (uint32_t)v[u] * RB, x[u]);
    } else {
#pragma unroll
        for (int u = 0; u < U; ++u) band_gather<T, K>(v[u], rows_q, Aq, x[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = fma(w[u], x[u][e], acc[e]);
}

template <typename T, int K>
__global__ void __launch_bounds__(band_threads<T, K>(), 1) k_sweep_band(const __grid_constant__ BandArgs<T> a) {
    constexpr int BAND_CW = band_cw<T, K>(), BAND_CT = BAND_CW * 32;
    using L = RowLayout<T, K>;
    using Acc = typename AccOf<T>::type;
    constexpr int E = L::E, G = L::G, RB = L::RB;
    constexpr int RPW = 32 / G;
    constexpr bool F64 = sizeof(T) == 8;
    static_assert(L::CB == 16, "band rows are whole 16-byte chunks");
    extern __shared__ __align__(128) unsigned char bsm[];
    __shared__ __align__(8) uint64_t ld_bar[BAND_NS];
    __shared__ __align__(8) uint64_t empty_bar[BAND_NS];
    __shared__ BandMeta meta[BAND_NS];
    __shared__ int abort_flag;
    __shared__ Acc st_sh[2 * K];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < BAND_NS; ++s) {
            mbar_init(&ld_bar[s], 1);
            mbar_init(&empty_bar[s], BAND_CT);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    for (int i = tid; i < 2 * K; i += blockDim.x) st_sh[i] = (Acc)a.stats_in[i];
    __syncthreads();
    volatile int* abortp = &abort_flag;
    const int nb = band_count(blockIdx.x, gridDim.x, a.nbands);
    const int slots_off = 8 * (a.R + 2);
    const uint32_t sbase = sm_addr(bsm);

    Acc s1[E], s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) s1[e] = s2[e] = Acc(0);

    if (warp == BAND_CW) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int issued = 0;
            RingState rs;
            int64_t nx0 = 0, nx1 = 0;  // row pointers of the next band, loaded one band ahead
            int4 nrun = make_int4(0, 0, 0, 0);
            auto fetch = [&](int k) {
                int r0, nrows, w0, w1;
                const int b = band_at(blockIdx.x, gridDim.x, k);
                band_rows(b, a.n, a.R, a.H, r0, nrows, w0, w1);
                nx0 = __ldg(a.rowptr + r0);
                nx1 = __ldg(a.rowptr + r0 + nrows);
                nrun = __ldg(a.runs + b);
            };
            if (nb > 0) fetch(0);
            for (int k = 0; k < nb; ++k) {
                const int st = k % BAND_NS;
                const int64_t s0 = nx0, s1x = nx1;
                const int4 run = nrun;
                if (k + 1 < nb) fetch(k + 1);
                // the consumers are done with the band that last used this stage
                // (and with the ring rows the loads below overwrite)
                if (k >= BAND_NS && !mbar_wait(&empty_bar[st], ((k / BAND_NS) - 1) & 1, abortp)) break;
                const int b = band_at(blockIdx.x, gridDim.x, k);
                int r0, nrows, w0, w1, pw0, la, p;
                band_rows(b, a.n, a.R, a.H, r0, nrows, w0, w1);
                ring_place(rs, (k % BAND_CB) == 0, w0, w1, a.WR, pw0, la, p);
                const int lcount = w1 - la;
                const int64_t s0a = s0 & ~(int64_t)3;
                const int64_t span = ((s1x - s0a) + 3) & ~(int64_t)3;
                const int ncp = (int)(span < (int64_t)a.SC ? span : (int64_t)a.SC);
                const int nlo = far_held(run.y, a.FC), nhi = far_held(run.w, a.FC);
                BandMeta& M = meta[st];
                M.s0a = s0a;
                M.r0 = r0;
                M.nrows = nrows;
                M.w0 = w0;
                M.pw0 = pw0;
                M.nsc = (int)((s1x - s0a) < (int64_t)ncp ? (s1x - s0a) : (int64_t)ncp);
                const uint32_t S = sbase + (uint32_t)(a.off_stage + st * a.stage_bytes);
                const uint32_t F = sbase + (uint32_t)(a.WR + st * 2 * a.FC) * RB;
                const uint32_t rp_bytes = (uint32_t)(((nrows + 2) & ~1) * 8);
                const uint32_t sl_bytes = (uint32_t)ncp * (F64 ? 4u : 8u);
                const uint32_t sw_bytes = F64 ? (uint32_t)ncp * 8u : 0u;
                const uint32_t x_bytes = (uint32_t)(lcount + nlo + nhi) * (uint32_t)RB;
                mbar_expect_tx(&ld_bar[st], rp_bytes + sl_bytes + sw_bytes + x_bytes);
                bulk_load(S, a.rowptr + r0, rp_bytes, &ld_bar[st]);
                if (ncp > 0) {
                    if constexpr (F64) {
                        bulk_load(S + slots_off, a.bs64 + s0a, sl_bytes, &ld_bar[st]);
                        bulk_load(S + a.off_sw, a.wn64 + s0a, sw_bytes, &ld_bar[st]);
                    } else {
                        bulk_load(S + slots_off, a.bs32 + s0a, sl_bytes, &ld_bar[st]);
                    }
                }
                // window rows [la, w1) at ring positions [p, p + lcount) mod WR
                if (lcount > 0) {
                    const int c1 = lcount < a.WR - p ? lcount : a.WR - p;
                    bulk_load(sbase + (uint32_t)p * RB, a.Ain + (size_t)la * K, (uint32_t)c1 * RB, &ld_bar[st]);
                    if (lcount > c1)
                        bulk_load(sbase, a.Ain + (size_t)(la + c1) * K, (uint32_t)(lcount - c1) * RB, &ld_bar[st]);
                }
                if (nlo > 0) bulk_load(F, a.Ain + (size_t)run.x * K, (uint32_t)nlo * RB, &ld_bar[st]);
                if (nhi > 0)
                    bulk_load(F + (uint32_t)a.FC * RB, a.Ain + (size_t)run.z * K, (uint32_t)nhi * RB, &ld_bar[st]);
                issued = k + 1;
            }
            if (*abortp) {
                // let the copies already issued land before the block exits
                for (int k = issued > BAND_NS ? issued - BAND_NS : 0; k < issued; ++k)
                    mbar_wait(&ld_bar[k % BAND_NS], (k / BAND_NS) & 1, nullptr);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ consumers
        const int seg = lane / G, q = lane % G;
        const bool lane_ok = seg < RPW;
        const Acc omega = (Acc)a.omega, one_m = (Acc)(1.0 - a.omega);
        const T* Aq = a.Ain + q * E;
        const uint32_t rows_q = sbase + q * 16;
        // this lane's columns of the input statistics, held for the whole sweep
        Acc mu[E], is[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            mu[e] = st_sh[q * E + e];
            is[e] = st_sh[K + q * E + e];
        }
        bool ok = true;
        for (int k = 0; ok && k < nb; ++k) {
            const int st = k % BAND_NS;
            // each warp goes at its own pace; a wait that gave up ends the
            // whole warp's work (and, through the abort word, every warp's)
            const bool fail = !mbar_wait(&ld_bar[st], (k / BAND_NS) & 1, abortp);
            if (__any_sync(0xffffffffu, fail)) {
                *abortp = 1;
                ok = false;
                break;
            }
            const BandMeta M = meta[st];
            const unsigned char* S = bsm + a.off_stage + st * a.stage_bytes;
            // the low words of the row pointers give the local slot range
            const int* rp32 = reinterpret_cast<const int*>(S);
            const int s0lo = (int)M.s0a;
            for (int lr0 = warp * RPW; lr0 < M.nrows; lr0 += BAND_CW * RPW) {
                const int lr = lr0 + seg;
                if (!lane_ok || lr >= M.nrows) continue;
                const int r = M.r0 + lr;
                const int jb = rp32[2 * lr] - s0lo, je = rp32[2 * lr + 2] - s0lo;
                const int jm = je < M.nsc ? je : M.nsc;  // slots from jm on are read from global memory
                Acc acc[E];
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] = Acc(0);
                int j = jb;
                const unsigned char* sl = S + slots_off;
                const unsigned char* sw = S + a.off_sw;
                for (; j + 4 <= jm; j += 4) band_group<T, K, 4>(sl, sw, j, rows_q, Aq, acc);
                if (j + 2 <= jm) {
                    band_group<T, K, 2>(sl, sw, j, rows_q, Aq, acc);
                    j += 2;
                }
                if (j < jm) band_group<T, K, 1>(sl, sw, j, rows_q, Aq, acc);
                for (int j = jm > jb ? jm : jb; j < je; ++j) {  // past the stage's slot capacity
                    int v;
                    Acc w;
                    if constexpr (F64) {
                        v = __ldg(a.bs64 + M.s0a + j);
                        w = __ldg(a.wn64 + M.s0a + j);
                    } else {
                        const int2 t = __ldg(a.bs32 + M.s0a + j);
                        v = t.x;
                        w = (Acc)__int_as_float(t.y);
                    }
                    Acc x[E];
                    band_gather<T, K>(v, rows_q, Aq, x);
#pragma unroll
                    for (int e = 0; e < E; ++e) acc[e] = fma(w, x[e], acc[e]);
                }
                int pos = M.pw0 + (r - M.w0);
                if (pos >= a.WR) pos -= a.WR;
                Acc xi[E];
                lds_chunk<T, E>(rows_q + (uint32_t)pos * RB, xi);
                const bool isolated = jb == je;
                Acc y[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    Acc z = isolated ? xi[e] : one_m * xi[e] + omega * acc[e];
                    y[e] = (z - mu[e]) * is[e];
                }
                store_chunk<T, E>(a.Aout + (size_t)r * K + q * E, y);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    s1[e] += y[e];
                    s2[e] += y[e] * y[e];
                }
            }
            mbar_arrive(&empty_bar[st]);
        }
    }

    // ---------------------------------------------------------------- statistics
    // lanes q < G collect the FP32 sums of lanes q + r G (same chunk, other
    // rows); warps combined in FP64 in fixed order.  The pipeline's shared
    // memory is idle now and holds the per-warp sums.
    __syncthreads();
    double* wst = reinterpret_cast<double*>(bsm);  // [BAND_CW][2K]
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
        for (int r = 1; r < RPW; ++r) {
            const Acc t1 = __shfl_sync(0xffffffffu, s1[e], (lane + r * G) & 31);
            const Acc t2 = __shfl_sync(0xffffffffu, s2[e], (lane + r * G) & 31);
            if (lane < G) {
                s1[e] += t1;
                s2[e] += t2;
            }
        }
    if (warp < BAND_CW && lane < G) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            wst[warp * 2 * K + lane * E + e] = (double)s1[e];
            wst[warp * 2 * K + K + lane * E + e] = (double)s2[e];
        }
    }
    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(a.err, 1);
    if (tid < 2 * K) {
        double t = 0.0;
        for (int w = 0; w < BAND_CW; ++w) t += wst[w * 2 * K + tid];
        // a block that gave up leaves its rows unwritten: NaN partials make the
        // statistics, and so every later output, NaN
        a.part[(int64_t)blockIdx.x * 2 * K + tid] = abort_flag ? __longlong_as_double(0x7ff8000000000000ll) : t;
    }
    __threadfence();
    __syncthreads();
    finish_stats<K, 256>(a.part, gridDim.x, a.counter, a.n64, a.stats_out);
}

// ---------------------------------------------------------------------------
// Plan: halo, band size, capacities, shared-memory layout
//   [ring: WR rows | far area: BAND_NS stages x 2 runs x FC rows | stages:
//    row pointers, slots (FP64: + weights)]
// ---------------------------------------------------------------------------
static int align128(int x) { return (x + 127) & ~127; }

template <typename T, int K>
static bool band_plan(const gr_ctx* c, bool forced, BandPlan* bp) {
    using L = RowLayout<T, K>;
    constexpr int RB = L::RB, G = L::G, RPW = 32 / G;
    constexpr bool F64 = sizeof(T) == 8;
    if (L::CB != 16 || !c->loc_ready || c->n < 2 || c->m < 1) return false;
    const double slots = 2.0 * (double)c->m;
    double cum[33];
    double run = 0.0;
    for (int b = 0; b < 33; ++b) {
        run += (double)c->loc_hist[b];
        cum[b] = run / slots;  // share of slots with |c - r| <= 2^b
    }
    // the smallest halo 2^h (1 ... 1024 rows) within 2 % of the share 1,024
    // rows catch (the rest is for the far runs)
    int h = 0;
    while (h < 10 && cum[h] < cum[10] - 0.02) ++h;
    if (!forced && cum[h] < 0.5) return false;
    const double avg = slots / (double)c->n;
    // the largest band that fits; when forced, smaller halos until one does
    for (int hh = h; hh >= (forced ? 0 : h); --hh)
        for (int P = 16; P >= 1; --P) {
            const int H = 1 << hh;
            constexpr int BAND_CW = band_cw<T, K>(), BAND_SMEM_MAX = band_smem_max<T, K>();
            const int R = P * BAND_CW * RPW;  // whole passes of the consumer warps
            if (R & 1) continue;              // row pointers copied in 16-byte units
            const int Rn = (int64_t)R < c->n ? R : (int)c->n;
            const int SC = ((int)(Rn * avg * 1.15) + 16 + 3) & ~3;
            if (SC > (1 << 20)) continue;
            const int FC = R + 8;  // far-run capacity, rows per run
            const int WR = BAND_NS * R + 4 * H;
            const int off_sl = 8 * (R + 2);  // 16-byte multiple (R even)
            const int off_sw = F64 ? align128(off_sl + 4 * SC) : 0;
            const int stage_bytes = align128(F64 ? off_sw + 8 * SC : off_sl + 8 * SC);
            const int64_t rows = (int64_t)WR + (int64_t)BAND_NS * 2 * FC;
            if (rows * RB > BAND_SMEM_MAX) continue;
            const int off_stage = align128((int)(rows * RB));
            size_t total = (size_t)off_stage + (size_t)BAND_NS * stage_bytes;
            if (total > (size_t)BAND_SMEM_MAX) continue;
            // the statistics' per-warp sums reuse the pipeline's shared memory
            if (total < (size_t)BAND_CW * 2 * K * sizeof(double)) total = (size_t)BAND_CW * 2 * K * sizeof(double);
            bp->R = R;
            bp->H = H;
            bp->SC = SC;
            bp->FC = FC;
            bp->WR = WR;
            bp->off_stage = off_stage;
            bp->stage_bytes = stage_bytes;
            bp->off_sw = off_sw;
            bp->nbands = (int)ceil_div(c->n, R);
            const int nchunks = (int)ceil_div(bp->nbands, BAND_CB);
            bp->grid = nchunks < c->num_sms ? nchunks : c->num_sms;
            bp->smem = total;
            return true;
        }
    return false;
}

#define GR_BAND_DISPATCH(FN, ...)                                   \
    do {                                                            \
        if (prec == GR_F64) {                                       \
            switch (K) {                                            \
                case 4: return FN<double, 4>(__VA_ARGS__);          \
                case 8: return FN<double, 8>(__VA_ARGS__);          \
                case 16: return FN<double, 16>(__VA_ARGS__);        \
                case 24: return FN<double, 24>(__VA_ARGS__);        \
                case 32: return FN<double, 32>(__VA_ARGS__);        \
            }                                                       \
        } else if (prec == GR_F32) {                                \
            switch (K) {                                            \
                case 4: return FN<float, 4>(__VA_ARGS__);           \
                case 8: return FN<float, 8>(__VA_ARGS__);           \
                case 16: return FN<float, 16>(__VA_ARGS__);         \
                case 24: return FN<float, 24>(__VA_ARGS__);         \
                case 32: return FN<float, 32>(__VA_ARGS__);         \
            }                                                       \
        } else {                                                    \
            switch (K) {                                            \
                case 8: return FN<__nv_bfloat16, 8>(__VA_ARGS__);   \
                case 16: return FN<__nv_bfloat16, 16>(__VA_ARGS__); \
                case 24: return FN<__nv_bfloat16, 24>(__VA_ARGS__); \
                case 32: return FN<__nv_bfloat16, 32>(__VA_ARGS__); \
            }                                                       \
        }                                                           \
    } while (0)

void band_release(gr_ctx* c) {
    if (c->band_runs) cudaFreeAsync(c->band_runs, c->stream);
    if (c->band_slots) cudaFreeAsync(c->band_slots, c->stream);
    c->band_runs = nullptr;
    c->band_slots = nullptr;
    c->band_key_R = c->band_key_H = c->band_key_grid = c->band_key_f64 = 0;
    c->band_nglobal = -1;
}

bool band_usable(const gr_ctx* c, int prec, int K, bool forced, BandPlan* bp) {
    GR_BAND_DISPATCH(band_plan, c, forced, bp);
    return false;
}

// The plan's far runs and slot rows: in the context (built once per plan), or,
// when `fixed` and the context holds none for this plan, rebuilt in `scratch`
// on every call.  With nglobal, also the number of slots read from global
// memory (a readback and a stream synchronisation unless already known).
cudaError_t band_prepare(gr_ctx* c, const BandPlan& bp, bool f64, bool fixed, void* scratch, size_t scratch_bytes,
                         const int4** runs_out, const void** slots_out, int64_t* nglobal) {
    const size_t nb = (size_t)bp.nbands;
    const size_t b_runs = (sizeof(int4) * nb + 255) & ~size_t(255);
    const size_t b_lay = (sizeof(int2) * nb + 255) & ~size_t(255);
    const size_t b_cnt = 256;
    if (c->band_runs && c->band_key_R == bp.R && c->band_key_H == bp.H && c->band_key_grid == bp.grid &&
        c->band_key_f64 == (int)f64) {
        *runs_out = c->band_runs;
        *slots_out = c->band_slots;
        if (nglobal) {
            if (c->band_nglobal < 0) {
                int64_t* hs = host_scratch();
                if (!hs) return cudaErrorMemoryAllocation;
                GR_CUDA(cudaMemcpyAsync(hs, (char*)c->band_runs + b_runs + b_lay, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, c->stream));
                GR_CUDA(cudaStreamSynchronize(c->stream));
                c->band_nglobal = hs[0];
            }
            *nglobal = c->band_nglobal;
        }
        return cudaSuccess;
    }
    const size_t b_slots = (f64 ? sizeof(int32_t) : sizeof(int2)) * ((size_t)(2 * c->m) + CSR_PAD_SLOTS);
    char* base = nullptr;
    void* slots = nullptr;
    if (fixed) {
        if (!scratch || b_runs + b_lay + b_cnt + b_slots > scratch_bytes) return cudaErrorMemoryAllocation;
        base = (char*)scratch;
        slots = base + b_runs + b_lay + b_cnt;
    } else {
        band_release(c);
        GR_CUDA(cudaMallocAsync((void**)&c->band_runs, b_runs + b_lay + b_cnt, c->stream));
        GR_CUDA(cudaMallocAsync(&c->band_slots, b_slots, c->stream));
        c->band_key_R = bp.R;
        c->band_key_H = bp.H;
        c->band_key_grid = bp.grid;
        c->band_key_f64 = (int)f64;
        base = (char*)c->band_runs;
        slots = c->band_slots;
    }
    int4* runs = (int4*)base;
    int2* lay = (int2*)(base + b_runs);
    unsigned long long* cnt = (unsigned long long*)(base + b_runs + b_lay);
    GR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), c->stream));
    const int n = (int)c->n;
    const unsigned wblocks = (unsigned)ceil_div((int64_t)bp.nbands * 32, 256);
    k_band_runs<<<wblocks, 256, 0, c->stream>>>(n, bp.nbands, bp.R, bp.H, c->rowptr, c->col, runs);
    count_launch();
    k_band_layout<<<(unsigned)ceil_div(bp.grid, 128), 128, 0, c->stream>>>(n, bp.nbands, bp.grid, bp.R, bp.H,
                                                                          bp.WR, lay);
    count_launch();
    if (f64)
        k_band_slots<true><<<wblocks, 256, 0, c->stream>>>(n, bp.nbands, bp.R, bp.H, bp.WR, bp.FC, c->rowptr,
                                                           c->col, c->cw32, runs, lay, slots, cnt);
    else
        k_band_slots<false><<<wblocks, 256, 0, c->stream>>>(n, bp.nbands, bp.R, bp.H, bp.WR, bp.FC, c->rowptr,
                                                            c->col, c->cw32, runs, lay, slots, cnt);
    count_launch();
    GR_CUDA(cudaGetLastError());
    *runs_out = runs;
    *slots_out = slots;
    if (nglobal) {
        int64_t* hs = host_scratch();
        if (!hs) return cudaErrorMemoryAllocation;
        GR_CUDA(cudaMemcpyAsync(hs, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        GR_CUDA(cudaStreamSynchronize(c->stream));
        *nglobal = hs[0];
        if (!fixed) c->band_nglobal = hs[0];
    }
    return cudaSuccess;
}

template <typename T, int K>
static cudaError_t band_launch(gr_ctx* c, const BandPlan& bp, const int4* runs, const void* slots, const void* Ain,
                               void* Aout, double omega, const double* st_in, double* part, int part_cap,
                               unsigned* counter, double* st_out, int* err) {
    BandArgs<T> a{};
    a.rowptr = c->rowptr;
    if constexpr (sizeof(T) == 8) a.bs64 = (const int32_t*)slots;
    else a.bs32 = (const int2*)slots;
    a.wn64 = c->wn64;
    a.runs = runs;
    a.Ain = (const T*)Ain;
    a.Aout = (T*)Aout;
    a.stats_in = st_in;
    a.part = part;
    a.counter = counter;
    a.stats_out = st_out;
    a.err = err;
    a.omega = omega;
    a.n64 = c->n;
    a.n = (int)c->n;
    a.nbands = bp.nbands;
    a.R = bp.R;
    a.H = bp.H;
    a.SC = bp.SC;
    a.FC = bp.FC;
    a.WR = bp.WR;
    a.off_stage = bp.off_stage;
    a.stage_bytes = bp.stage_bytes;
    a.off_sw = bp.off_sw;
    if (bp.grid > part_cap) return cudaErrorInvalidValue;
    auto kern = k_sweep_band<T, K>;
    GR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bp.smem));
    kern<<<bp.grid, band_threads<T, K>(), bp.smem, c->stream>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t sweep_band(gr_ctx* c, int prec, int K, const BandPlan& bp, const int4* runs, const void* slots,
                       const void* Ain, void* Aout, double omega, const double* st_in, double* part, int part_cap,
                       unsigned* counter, double* st_out, int* err) {
    GR_BAND_DISPATCH(band_launch, c, bp, runs, slots, Ain, Aout, omega, st_in, part, part_cap, counter, st_out, err);
    return cudaErrorInvalidValue;
}

#undef GR_BAND_DISPATCH

}  // namespace gr
