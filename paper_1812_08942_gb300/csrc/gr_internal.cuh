// Internal declarations shared by the translation units of libgraphreduce.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "graph_reduce.h"

namespace gr {

// ---------------------------------------------------------------------------
// Error plumbing: every internal routine returns cudaError_t or gr_status;
// the API layer turns CUDA errors into GR_ECUDA with a message.
// ---------------------------------------------------------------------------
#define GR_CUDA(expr)                                   \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return _e;               \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Allocated entries past the end of the CSR arrays (rowptr, and col / eid /
// cw32 / wn64): the band sweep copies row pointers and slots in 16-byte units
// and may read up to one row pointer and three slots past the last one in use.
constexpr int64_t CSR_PAD_ROWS = 1;
constexpr size_t CSR_PAD_SLOTS = 4;

// Shape of the band sweep on one graph (gr_band.cu)
struct BandPlan {
    int R = 0, H = 0;       // rows per band, halo rows on each side of a band
    int SC = 0, FC = 0;     // slot capacity of a stage, rows per far run held
    int WR = 0;             // rows of the window ring
    int nbands = 0, grid = 0;
    int off_stage = 0, stage_bytes = 0, off_sw = 0;
    size_t smem = 0;        // dynamic shared memory per block
};

// Grow-only device scratch, stream-ordered (cudaMallocAsync / cudaFreeAsync).
struct Workspace {
    struct Slot {
        void* ptr = nullptr;
        size_t bytes = 0;
    };
    std::vector<Slot> slots;
    cudaStream_t stream = nullptr;
    cudaError_t get(int slot, size_t bytes, void** out);
    void release();
};

// Named workspace slots (each owner uses disjoint slots).
enum WsSlot {
    WS_SORT_A = 0, WS_SORT_B, WS_SORT_C, WS_SORT_D, WS_SORT_HIST, WS_SCAN,
    WS_SMOOTH_BUF, WS_SMOOTH_STATS, WS_SMOOTH_PART,
    WS_AGG_STATE, WS_AGG_LIST, WS_AGG_KEYS, WS_AGG_SMALL,
    WS_COARSE_KEYS, WS_COARSE_VALS, WS_COARSE_TMP,
    WS_GAL_KEYS, WS_GAL_UCOL, WS_GAL_UW, WS_GAL_ROWS,
    WS_EIG, WS_EIG_WORK, WS_DATASET, WS_GS, WS_SCALE,
    WS_LOSS_A, WS_LOSS_B, WS_LOSS_C,
    WS_ML_X, WS_ML_D, WS_ML_AGG,
    WS_PINNED_UNUSED,
    WS_COUNT
};

}  // namespace gr

struct gr_ctx {
    int64_t n = 0, m = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    // canonical edge list (owned)
    int32_t* eu = nullptr;
    int32_t* ev = nullptr;
    double* ew = nullptr;
    int64_t* eptr = nullptr;    // n+1: edges with u == p are [eptr[p], eptr[p+1])
    // symmetric CSR; row order = ascending neighbour = ascending edge id
    int64_t* rowptr = nullptr;  // n+1
    int32_t* col = nullptr;     // 2m
    int32_t* eid = nullptr;     // 2m
    int2* cw32 = nullptr;       // 2m: (col, float bits of w / deg_row)
    double* wn64 = nullptr;     // 2m: w / deg_row
    double* deg = nullptr;      // n
    // slot-balanced row partition for the streaming sweep (W+1 row starts)
    int32_t* wpart = nullptr;
    int64_t wpart_W = 0;
    int4* cw64 = nullptr;       // 2m: (col, 0, w / deg_row as FP64), built on first FP64 sweep
    // sweep kernel selection (gr_sweep_kernel)
    int sweep_kind = GR_SWEEP_AUTO;
    // locality profile for the band sweep: slots with |col - row| in
    // (2^(b-1), 2^b] per bucket b (bucket 0: <= 1, 32: beyond), built on first use
    unsigned long long loc_hist[33] = {};
    bool loc_ready = false;
    // band sweep tables for one plan (band size, halo, grid, FP64 or not):
    // far runs and window ring positions per band, and the slots' shared rows
    int4* band_runs = nullptr;
    void* band_slots = nullptr;
    int band_key_R = 0, band_key_H = 0, band_key_grid = 0, band_key_f64 = 0;
    int64_t band_nglobal = -1;  // slots of those tables read from global memory (-1: not read back)
    // the automatic kernel choice's verdict on the band kernel for one plan
    // (-1: not decided)
    int band_auto_R = 0, band_auto_H = 0, band_auto_grid = 0, band_auto_f64 = 0, band_auto_ok = -1;
    // multicolour Gauss-Seidel ordering for one colouring seed, built on first use:
    // nodes in ascending (colour, id) and each colour's range in that list
    int32_t* gs_order = nullptr;
    std::vector<int64_t> gs_ptr;
    uint64_t gs_seed = 0;
    bool gs_ready = false;
    // mapping from the parent level (coarse contexts only)
    int32_t* parent_map = nullptr;
    int64_t parent_n = 0;
    gr::Workspace ws;
    std::string last_error;
};

namespace gr {

// band sweep (gr_band.cu).  ensure_locality fills the context's locality
// profile (one kernel and a readback into host memory; 264 bytes of device
// scratch).  band_usable: a band plan for (prec, K) fits shared memory; unless
// forced, also that the halo catches at least half of the slots.
// band_prepare: the plan's per-band far runs and per-slot shared rows (16 + 8
// bytes per band, 8 bytes per slot, 4 for FP64 blocks), kept in the context,
// or, when `fixed`, built in `scratch` (scratch_bytes) if the context holds
// none for this plan (cudaErrorMemoryAllocation if they do not fit); with
// nglobal, the count of slots read from global memory (synchronises the
// stream unless known).  band_release frees the context's tables.
// sweep_band launches one sweep (err: device word set to 1 if a wait ran out).
cudaError_t ensure_locality(gr_ctx* c, void* scratch264);
bool band_usable(const gr_ctx* c, int prec, int K, bool forced, BandPlan* bp);
cudaError_t band_prepare(gr_ctx* c, const BandPlan& bp, bool f64, bool fixed, void* scratch, size_t scratch_bytes,
                         const int4** runs_out, const void** slots_out, int64_t* nglobal);
void band_release(gr_ctx* c);
cudaError_t sweep_band(gr_ctx* c, int prec, int K, const BandPlan& bp, const int4* runs, const void* slots,
                       const void* Ain, void* Aout, double omega, const double* st_in, double* part, int part_cap,
                       unsigned* counter, double* st_out, int* err);

// The k smallest eigenpairs of L u = lambda B u on graph c (b: the diagonal
// of B, NULL for B = I; entries that are not positive count as 1), by a
// Chebyshev-filtered subspace iteration (gr_chfsi.cu): lam_dev (device) and
// lam_host (host), k eigenvalues ascending; U (device, n x k row-major) the
// eigenvectors; scratch from ws slot WS_EIG_WORK; *iters (may be NULL) the
// filter iterations run.  GR_ECUDA if it does not converge.
gr_status coarsest_eigenpairs(gr_ctx* c, const double* b, int k, Workspace& ws, cudaStream_t s, double* lam_dev,
                              double* lam_host, double* U, int* iters);
// The same for graphs of at most DENSE_EIG_MAX nodes by the dense route
// (gr_dense_eig.cu: Householder tridiagonalisation, bisection, inverse
// iteration); coarsest_eigenpairs hands such graphs to it when the filtered
// iteration would converge slowly.
constexpr int DENSE_EIG_MAX = 4096;
gr_status dense_eigenpairs(gr_ctx* c, const double* b, int k, Workspace& ws, cudaStream_t s, double* lam_dev,
                           double* lam_host, double* U);

// primitives (gr_prims.cu)
cudaError_t scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t count, Workspace& ws,
                               cudaStream_t s);
cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t count, Workspace& ws,
                               cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
// Buffers a/b ping-pong; on return *result points at the buffers holding the
// sorted data (either the inputs or the alternates).
cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                           uint32_t* vals_alt, int64_t count, int bits, Workspace& ws,
                           cudaStream_t s, int* result_in_alt);
cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                           uint32_t* vals_alt, int64_t count, int bits, Workspace& ws,
                           cudaStream_t s, int* result_in_alt);
int bits_for(uint64_t max_value_inclusive);
// 64 bytes of pinned host memory owned by the calling thread, for small
// readbacks inside one API call (never held across calls).
int64_t* host_scratch();
// keep freed stream-ordered allocations cached in the device's default pool
void tune_mempool(int device);
// process-wide count of kernel launches made by this library
void count_launch();
uint64_t launch_count();

// graph construction (gr_graph.cu).  build_csr checks that the edge list is
// canonical when `check` is set (*invalid reports a failed check, GR_EINVAL).
gr_status build_csr(gr_ctx* c, bool check, bool* invalid);
gr_status build_csr_sorted(gr_ctx* c, const int32_t* lcnt, int64_t* rowcnt);
// deg = row sums of the raw slot weights in wn64, then wn64 / cw32 scaled by 1 / deg
cudaError_t degree_scale(gr_ctx* c);
// Galerkin product assembled row by row (gr_galerkin.cu).  Fills the coarse
// context cc (n = nc set by the caller) or, when the coarse rows are too long
// for per-row sorting, sets *too_long and leaves cc untouched.
gr_status galerkin_rows(gr_ctx* c, const int32_t* agg, int64_t nc, gr_ctx* cc, bool* too_long);

// Slot of the calling thread in a list that grows by one entry per thread
// with `keep` set: one atomic per block, entries in thread order within the
// block; -1 if !keep.  Every thread of the block must call it (it holds
// barriers); BT is the block size.
template <int BT>
__device__ __forceinline__ int32_t block_slot(bool keep, int32_t* count) {
    __shared__ int32_t wbase[BT / 32];
    __shared__ int32_t bbase;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    __syncthreads();  // the previous call's readers are done
    if (lane == 0) wbase[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t tot = 0;
        for (int w = 0; w < BT / 32; ++w) {
            const int32_t c = wbase[w];
            wbase[w] = tot;
            tot += c;
        }
        bbase = tot > 0 ? atomicAdd(count, tot) : 0;
    }
    __syncthreads();
    return keep ? bbase + wbase[warp] + __popc(bal & ((1u << lane) - 1u)) : -1;
}

// Slot of the calling lane in a list that grows by one entry per lane with
// `keep` set: one atomic per warp, entries in lane order; -1 if !keep.
__device__ __forceinline__ int32_t warp_slot(bool keep, int32_t* count) {
    const unsigned active = __activemask();
    const unsigned ball = __ballot_sync(active, keep);
    if (!ball) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ball) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(ball));
    base = __shfl_sync(active, base, leader);
    return keep ? base + __popc(ball & ((1u << lane) - 1u)) : -1;
}

// kernels entry points used by the API layer
// ev_begin / ev_end (optional) are recorded around the sweep kernels only.
// raw (optional): the last normalisation X = (A - mu) / s is left to the
// caller, who gets the block A (X itself or a workspace buffer of c) and its
// statistics (mu[K] then 1/s[K], FP64, workspace of c) -- valid until c's
// next smoothing call.
struct SmoothRaw {
    const void* A;
    const double* stats;
};
gr_status test_vectors_impl(gr_ctx* c, int K, uint64_t seed, int level, gr_prec prec, void* X);
gr_status smooth_impl(gr_ctx* c, int K, int sweeps, double omega, uint64_t seed, int level,
                      gr_prec prec, void* X, cudaEvent_t ev_begin = nullptr,
                      cudaEvent_t ev_end = nullptr, SmoothRaw* raw = nullptr);
gr_status smooth_gs_impl(gr_ctx* c, int K, int sweeps, double omega, uint64_t seed, int level,
                         uint64_t colour_seed, gr_prec prec, void* X);
gr_status colour_impl(gr_ctx* c, uint64_t colour_seed, int32_t* colour_out, int32_t* ncolours_out);
// stats (optional): X is a block still to be normalised by these column
// statistics (the layout of SmoothRaw), rounded as the stored block would be
gr_status affinity_impl(gr_ctx* c, const void* X, int K, gr_prec prec, void* d, void* a,
                        const double* stats = nullptr);
gr_status aggregate_impl(gr_ctx* c, const void* d, int d_is_f64, int64_t target_nc, int passes,
                         int64_t max_proposals, int32_t* agg, int64_t* nc_out, int64_t* proposals_out);
gr_status coarsen_impl(gr_ctx* c, const int32_t* agg, int64_t nc, gr_ctx** out);
gr_status compose_impl(gr_ctx* const* levels, int nlevels, int32_t* out);
gr_status reduce_data_impl(gr_ctx* const* levels, int nlevels, const void* F, int d, int f64, int mean,
                           void* F_out);
gr_status eigensolve_impl(gr_ctx* const* levels, int nlevels, int k, int normalized, int galerkin_mass,
                          double omega, int iters, double* U_out, double* lambda_out, double* rayleigh_out);
gr_status scale_edges_impl(gr_ctx* fine, gr_ctx* coarse, const int32_t* agg, const float* X, int K, int sweeps,
                           double omega, double alpha, double eta_max, double delta_bar, double eps, int kmax,
                           float* w, int32_t* iters_out, double* loss_hist, double* lam1_hist);
gr_status loss_fwd_impl(gr_ctx* fine, gr_ctx* coarse, const int32_t* agg, const float* X, int K,
                        const float* w_c, int sweeps, double omega, float* loss, float* saved);
gr_status loss_bwd_impl(gr_ctx* coarse, const float* saved, int K, const float* w_c, int sweeps,
                        double omega, const float* grad_loss, float* grad_w);

gr_status sweep_plan_impl(gr_ctx* c, int K, gr_prec prec, int32_t* kind_out);

gr_status set_error(gr_ctx* c, gr_status st, const std::string& msg);
gr_status cuda_error(gr_ctx* c, cudaError_t e, const char* where);

}  // namespace gr

#define GR_TRY_CUDA(ctx, expr, where)                                   \
    do {                                                                \
        cudaError_t _e = (expr);                                        \
        if (_e != cudaSuccess) return gr::cuda_error((ctx), _e, where); \
    } while (0)
