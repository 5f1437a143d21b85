/*
 * graph_reduce.h -- C ABI of the GB300 (sm_103a) spectral node-aggregation
 * library: the Phase (A) hot path of "Nearly-Linear Time Spectral Graph
 * Reduction for Scalable Graph Partitioning and Data Visualization"
 * (Zhao, Wang, Feng; arXiv 1812.08942).
 *
 * The problem statement (Sec. 3.1, Table "symbol", Alg. 4): given the graph
 * Laplacian L_G of a weighted undirected graph, produce a much smaller graph
 * R with Laplacian L_R = H_G^R L_G H_R^G and the node mapping H between them.
 * One level of Phase (A) is
 *     smooth    K random test vectors by weighted-Jacobi sweeps (Alg. 3),
 *     affinity  per-edge spectral affinity / algebraic distance (Eq. eqn:agg),
 *     aggregate nodes joined by small algebraic distance (Sec. 3.2.2),
 *     coarsen   Galerkin product L_R = P^T L_G P (Sec. 3.2.2),
 * repeated level by level.
 *
 * Conventions for every call
 *   Graph input  canonical undirected edge list: u[e] < v[e] < n, sorted by
 *                (u, v), no duplicates, w[e] finite and > 0.  The edge id of an
 *                edge is its position e in that list; every per-edge array
 *                (d, a, w_c, gradients) is indexed by it.
 *   Pointers     device pointers on the context's stream unless the argument
 *                name or a flag says host.  Vector blocks are row-major n x K
 *                (entry (i, k) at X[i*K + k]).
 *   Ownership    the caller owns every buffer it passes; a context owns the
 *                device copy of its graph and its scratch, all released by
 *                graph_reduce_destroy.  Contexts returned by coarsen /
 *                multilevel are owned by the caller and destroyed separately.
 *   Ordering     work is enqueued on the context's CUDA stream; calls that
 *                return a host value (counts, sizes) synchronise that stream.
 *                One context is used by one host thread at a time.
 *   Errors       no exception crosses the ABI.  On a non-zero status the
 *                outputs are unspecified and graph_reduce_last_error(ctx)
 *                describes the failure; the context stays usable except after
 *                GR_ECUDA caused by a sticky CUDA error.
 */
#ifndef GRAPH_REDUCE_H
#define GRAPH_REDUCE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gr_ctx gr_ctx;

typedef enum {
    GR_OK = 0,
    GR_EINVAL = 1,    /* invalid argument or non-canonical graph            */
    GR_ENOMEM = 2,    /* device allocation failed                           */
    GR_ECUDA = 3,     /* CUDA runtime error                                 */
    GR_ETIMEOUT = 4,  /* aggregation exceeded its proposal budget           */
    GR_ESTATE = 5     /* call not valid for this context                    */
} gr_status;

/* Arithmetic of the test-vector block.  GR_F64: FP64 storage and arithmetic.
 * GR_F32: FP32 storage and accumulation, FP64 column statistics.  GR_BF16:
 * BF16 storage of X, FP32 accumulation, FP64 column statistics. */
typedef enum { GR_F64 = 0, GR_F32 = 1, GR_BF16 = 2 } gr_prec;

/* Build a context: the symmetric CSR of the adjacency A_G, the weighted
 * degrees D_G(i,i) = sum_j w_ij (ascending edge id) and the row-scaled weights
 * w_ij / D_G(i,i) used by D_G^-1 A_G (Sec. 2.1, Laplacian definition; Alg. 3).
 *   n, m             node and edge count (n >= 1, 0 <= m < 2^31)
 *   u, v, w          canonical edge list, host arrays if inputs_on_host else
 *                    device arrays; copied, not retained
 *   cuda_stream      cudaStream_t for all work of this context (NULL: legacy
 *                    default stream)
 * GR_EINVAL if the list is not canonical (checked on every create). */
gr_status graph_reduce_create(gr_ctx** out, int64_t n, int64_t m, const int32_t* u,
                              const int32_t* v, const double* w, int inputs_on_host,
                              void* cuda_stream);

/* Node and edge count of a context (host outputs, either may be NULL). */
gr_status graph_reduce_get_info(const gr_ctx* ctx, int64_t* n_out, int64_t* m_out);

/* Test-vector smoothing (Sec. 3.2.1 with the weighted-Jacobi relaxation of
 * Alg. 3).  Draws X0 (n x K, entry (i,k) = 2u - 1 with u the top 53 bits of
 * output number c+1 of SplitMix64 seeded with `seed`, c = level*2^40 + i*K +
 * k), centres every column (1^T x = 0) and scales it to unit 2-norm, then runs
 * `sweeps` sweeps x <- (1-omega) x + omega D^-1 A x, each followed by the same
 * centring and normalisation (column statistics in FP64).  An isolated node
 * keeps its value in a sweep.
 *   K        number of test vectors: 4, 8, 16, 24 or 32
 *   prec     GR_F64 / GR_F32 / GR_BF16: X is double / float / bfloat16
 *   X        device output, n x K row-major */
gr_status graph_reduce_smooth(gr_ctx* ctx, int K, int sweeps, double omega, uint64_t seed,
                              int level, gr_prec prec, void* X);

/* The random test-vector block X0 of graph_reduce_smooth before any centring
 * (Sec. 3.2.1: random vectors to be smoothed): entry (i,k) = 2u - 1 as
 * defined there, rounded once to the storage type (GR_F64: exact; GR_F32:
 * to nearest, ties to even; GR_BF16: the FP32 value rounded to nearest even).
 * Arguments as for graph_reduce_smooth; X (device, n x K row-major) is
 * overwritten. */
gr_status graph_reduce_test_vectors(gr_ctx* ctx, int K, uint64_t seed, int level, gr_prec prec, void* X);

/* Allocation-free variant of graph_reduce_smooth, for callers that must not
 * allocate device memory once they are running: for example code working
 * inside a fixed, pre-reserved memory budget, or under another framework's
 * allocator, where a cudaMalloc / cudaMallocAsync from a library would break
 * the budget or the allocator's bookkeeping.  The paper has no counterpart.
 * It runs graph_reduce_smooth's own launch sequence (same kernels, grids and
 * order of additions), so X is bit for bit the same as graph_reduce_smooth's.
 * The caller passes the graph (ctx, created beforehand) and the output X, as
 * for graph_reduce_smooth.  The scratch -- the second n x K block, the column
 * statistics and per-block partial sums, and, when the context does not hold
 * them yet, the packed FP64 slots (16 bytes per CSR slot, FP64 blocks), the
 * streaming kernel's row partition and the band kernel's tables (24 bytes per
 * band plus 8 bytes per slot, 4 for FP64 blocks) -- lives in one 32 MiB
 * device array inside the library, held by every GPU that loads it until the
 * process exits; what a call needs must fit, else GR_EINVAL (n*K*sizeof
 * (element) plus about 1 MiB of statistics, and the rest as said).  Nothing
 * is cached from the array into the context; only the band kernel's locality
 * profile (33 counts) and the automatic choice's verdict on it, host values
 * measured with stream synchronisations on first use, are kept there.  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and should come before any stream capture.  All
 * calls share the array and it keeps the last call's contents: calls that
 * overlap on the GPU (other streams, other contexts) race and corrupt each
 * other; serialise them.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
gr_status graph_reduce_smooth_noalloc(gr_ctx* ctx, int K, int sweeps, double omega,
                                      uint64_t seed, int level, gr_prec prec, void* X);

/* Sweep kernel behind graph_reduce_smooth and graph_reduce_smooth_noalloc on
 * this context.  The paper has no counterpart: these are implementations of
 * the same weighted-Jacobi sweep (Alg. 3), each adding a row's products in
 * slot order, so they agree within the rounding of the column statistics.
 *   GR_SWEEP_AUTO    (default) the streaming kernel when rows are long (a
 *                    warp's group of 32 / lanes-per-row rows would hold over
 *                    128 slots); else the band kernel when the graph has at
 *                    least 640 rows per SM (enough for a chunk of bands on
 *                    every SM) and is in a banded order: at least half of
 *                    its slots within a halo of at most 1,024 rows that fits
 *                    shared memory, and at least 95 % of the neighbours held
 *                    in shared memory by the band tables (measured once per
 *                    context and plan: two stream synchronisations; tables
 *                    of a graph that fails are freed); else the row-group
 *                    kernel
 *   GR_SWEEP_ROW     row-group kernel: one lane per 16-byte chunk of a vector
 *                    row, several rows per warp, rows grid-strided
 *   GR_SWEEP_STREAM  warp per row over a slot-balanced row partition, the
 *                    slots staged through shared memory
 *   GR_SWEEP_BAND    bands of consecutive rows staged with bulk copies: the
 *                    rows within a halo of the band through a ring buffer in
 *                    shared memory, the band's far neighbours as two
 *                    contiguous runs; for graphs in a banded order (meshes,
 *                    grids).  The first use measures the graph's locality
 *                    (one kernel and a stream synchronisation) and keeps the
 *                    band tables in the context (24 bytes per band, and per
 *                    slot 8 bytes, 4 for FP64 blocks).  Falls back to the
 *                    row-group kernel where no band fits shared memory.
 * GR_EINVAL for any other value. */
typedef enum { GR_SWEEP_AUTO = 0, GR_SWEEP_ROW = 1, GR_SWEEP_STREAM = 2, GR_SWEEP_BAND = 3 } gr_sweep_kernel;

gr_status graph_reduce_set_sweep_kernel(gr_ctx* ctx, gr_sweep_kernel kind);

/* The sweep kernel graph_reduce_smooth runs on this context for K and prec
 * (no counterpart in the paper; for tuning and tests).
 *   kernel_out   host: GR_SWEEP_ROW, GR_SWEEP_STREAM or GR_SWEEP_BAND */
gr_status graph_reduce_sweep_plan(gr_ctx* ctx, int K, gr_prec prec, int32_t* kernel_out);

/* Test-vector smoothing with the Gauss-Seidel relaxation Sec. 3.2.1 names,
 * made parallel by a multicolour ordering.  The paper gives no ordering; this
 * one is the greedy colouring in descending priority (priority of node i =
 * output number c+1 of SplitMix64 seeded with colour_seed, c = 2^62 + i, the
 * larger id winning a tie), each node taking the smallest colour unused by its
 * higher-priority neighbours; a sweep visits the nodes in ascending (colour,
 * id), each update x_i <- (1-omega) x_i + omega (D^-1 A x)_i seeing the latest
 * values (nodes of one colour are never adjacent, so a colour is updated at
 * once).  X0, the centring and normalisation after every sweep, and K, prec
 * and X are as for graph_reduce_smooth.  The ordering is computed on first use
 * for a colour_seed and kept in the context. */
gr_status graph_reduce_smooth_gs(gr_ctx* ctx, int K, int sweeps, double omega, uint64_t seed, int level,
                                 uint64_t colour_seed, gr_prec prec, void* X);

/* The colouring behind graph_reduce_smooth_gs.
 *   colour_out     device, n colours in [0, ncolours)
 *   ncolours_out   host */
gr_status graph_reduce_colour(gr_ctx* ctx, uint64_t colour_seed, int32_t* colour_out, int32_t* ncolours_out);

/* Per-edge affinity a = (X_p,X_q)^2 / ((X_p,X_p)(X_q,X_q)) (Eq. eqn:agg) and
 * algebraic distance d = 1 - a (Sec. 3.2.2), for every edge (p, q) of the
 * canonical list.  d is evaluated without cancellation as
 * |h_p - h_q|^2 |h_p + h_q|^2 / 4 with h = X_row / |X_row|; a zero row gives
 * a = 0, d = 1.
 *   X        device, n x K in the storage type of prec
 *   d_out    device, m entries: double for GR_F64, float otherwise
 *   a_out    device, m entries of the same type, or NULL */
gr_status graph_reduce_affinity(gr_ctx* ctx, const void* X, int K, gr_prec prec, void* d_out,
                                void* a_out);

/* Node aggregation by algebraic distance (Sec. 3.2.2).  The paper names no
 * scheme; this one is greedy matching in ascending (d, edge id) order, run in
 * `passes` passes on the cluster graph (the key of a cluster pair is its
 * smallest fine (d, id)), each pass making at most n_cur - target_nc merges and
 * passes stopping once n_cur <= target_nc.  Computed per pass by the suitor
 * algorithm (Manne & Halappanavar 2014: lock-free proposals, each cluster
 * keeping the best key proposed to it), which yields exactly the greedy
 * matching.  Coarse label = rank of the aggregate's smallest fine node.
 *   d              device, m distances (double if d_is_f64 else float), >= 0
 *   target_nc      >= 1
 *   max_proposals  budget of proposals (successful or not) per pass; <= 0:
 *                  no budget.  A pass makes at least one per matched cluster.
 *   agg_out        device, n labels in [0, nc)
 *   nc_out         host, number of aggregates
 *   proposals_out  host, total proposals over all passes, or NULL
 * GR_ETIMEOUT if a pass made more than max_proposals proposals (its work is
 * done; the outputs are unspecified). */
gr_status graph_reduce_aggregate(gr_ctx* ctx, const void* d, int d_is_f64, int64_t target_nc,
                                 int passes, int64_t max_proposals, int32_t* agg_out, int64_t* nc_out,
                                 int64_t* proposals_out);

/* Galerkin reduced graph L_R = H_G^R L_G H_R^G (Sec. 3.2.2) with H_R^G = P,
 * P[i, agg[i]] = 1, H_G^R = P^T: one reduced edge (A < B) per pair of
 * aggregates joined by fine edges, its weight the FP64 sum of those fine
 * weights in ascending fine edge id; edges inside an aggregate vanish.
 * Returns a new context on the same stream that also keeps `agg` as its
 * mapping from the parent level.
 *   agg      device, n labels in [0, nc); every label must be used */
gr_status graph_reduce_coarsen(gr_ctx* ctx, const int32_t* agg, int64_t nc, gr_ctx** coarse_out);

/* Copy the canonical edge list out.  Pass NULL for u, v and w to query the
 * count only.  outputs_on_host selects host or device destinations. */
gr_status graph_reduce_get_edges(const gr_ctx* ctx, int64_t* m_out, int32_t* u, int32_t* v,
                                 double* w, int outputs_on_host);

/* Copy the mapping a coarse context was built with (parent node -> this
 * context's node), n_parent entries, to device memory `agg_out`.
 * GR_ESTATE for a context not made by coarsen. */
gr_status graph_reduce_get_map(const gr_ctx* ctx, int32_t* agg_out, int64_t* n_parent_out);

/* Reduced data set F_R = H_G^R F (Alg. 6, step 4) with H_G^R = P^T composed
 * over the levels: row A of F_R is the sum of the rows of the fine nodes that
 * end in coarsest aggregate A, added in ascending fine id in FP64 (mean = 1
 * divides by the member count instead -- the paper names no normalisation;
 * the plain P^T sum is its operator).
 *   levels   nlevels >= 1 coarse contexts as from graph_reduce_multilevel
 *            (levels[0] coarsened from the fine graph, each the next one's parent)
 *   F        device, n_fine x d row-major, double if f64 else float
 *   F_out    device, n_coarsest x d, same type
 * GR_ESTATE if a level does not come from coarsen; GR_EINVAL for bad sizes. */
gr_status graph_reduce_reduce_data(gr_ctx* const* levels, int nlevels, const void* F, int d, int f64, int mean,
                                   void* F_out);

/* Multilevel Laplacian eigensolver (Alg. 5, Sec. 4.1; Eqs. equ:lgl and
 * equ:lgs).  The first k eigenpairs of L u = lambda B u on the coarsest level
 * come from a Chebyshev-filtered subspace iteration in FP64 on the coarsest
 * graph (a block of k + max(8, k/2) columns, at most the coarsest size;
 * Rayleigh-Ritz residuals at most 1e-13 times a Gershgorin bound of
 * B^-1/2 L B^-1/2; a seeded start, so results are reproducible); B is, on
 * every level, either that level's own I (ratio cut) or D (normalised cut), as Alg. 5 states, or
 * -- galerkin_mass = 1 -- the Galerkin-consistent mass B_l = P^T B_(l-1) P
 * carried from the finest level's I or D (diagonal: each coarse entry the sum
 * of its members', added in ascending member id), which makes the coarsest
 * problem the projection of the finest one onto the piecewise-constant
 * vectors (the paper does not say which; see Table "symbol" for P).  Then,
 * level by level toward the finest, the block is
 * mapped with H = P (U_fine[i] = U_coarse[map[i]]) and every column k is
 * smoothed by `iters` weighted-Jacobi iterations on (L - lambda_k B) y = 0,
 *   y <- (1 - omega) y + omega (D - lambda_k B)^-1 A y,
 * lambda_k being the coarsest eigenvalue (a row whose shifted diagonal is not
 * positive keeps its value: the paper is silent there); the finest block is
 * orthonormalised by modified Gram-Schmidt in column order.
 *   levels        nlevels >= 1 contexts: levels[0] the finest graph, levels[l]
 *                 (l >= 1) coarsened from levels[l-1] (its parent map is H)
 *   k             1..32, at most the coarsest size (which must be <= 16384)
 *   normalized    0: B = I, 1: B = D (a degree-0 node takes B = 1 on the
 *                 coarsest level, and in the finest mass of galerkin_mass)
 *   galerkin_mass 0: each level's own B; 1: B_l = P^T B_(l-1) P
 *   omega, iters  Jacobi weight (0, 1] and iterations per finer level
 *   U_out         device, n_0 x k row-major FP64, on levels[0]'s stream
 *   lambda_out    host, k FP64: the coarsest eigenvalues, ascending
 *   rayleigh_out  host, k FP64: x'Lx / x'Bx of the returned columns, or NULL
 * GR_EINVAL for a bad hierarchy or sizes; GR_ECUDA if the coarsest iteration
 * does not converge (400 filter iterations). */
gr_status graph_reduce_eigensolve(gr_ctx* const* levels, int nlevels, int k, int normalized, int galerkin_mass,
                                  double omega, int iters, double* U_out, double* lambda_out, double* rayleigh_out);

/* Parameters of the level loop. */
typedef struct gr_params {
    int K;                 /* test vectors per level                          */
    int sweeps;            /* Jacobi sweeps per level                         */
    double omega;          /* Jacobi weight (theta of Alg. 3)                 */
    uint64_t seed;         /* test-vector seed; level l uses counter block l  */
    int prec;              /* gr_prec of X                                    */
    int passes;            /* aggregation passes per level                    */
    int level_ratio;       /* level target = max(ceil(n/level_ratio), final)  */
    int64_t final_target;  /* stop once n <= final_target                     */
    int max_levels;        /* capacity of levels_out                          */
    int64_t max_proposals; /* aggregation proposal budget per pass (<= 0: none) */
} gr_params;

/* Per-level record filled by graph_reduce_multilevel (host).  Times are CUDA
 * event intervals on the context stream, in milliseconds; t_sweeps covers
 * only the `sweeps` Jacobi sweep kernels inside t_smooth. */
typedef struct gr_level_stats {
    int64_t n, m, nc, mc;
    int64_t proposals;     /* aggregation proposals over all passes */
    int32_t sweeps;
    float t_smooth, t_affinity, t_aggregate, t_coarsen;
    float t_sweeps;
} gr_level_stats;

/* The level loop of Phase (A): on level l (fine context = level 0) run
 * smooth(seed, level l) -> affinity -> aggregate(target max(ceil(n_l /
 * level_ratio), final_target)) -> coarsen, until n_l <= final_target, a level
 * makes no merge, or max_levels levels exist.
 *   levels_out   host array of max_levels; receives the coarse contexts
 *                (owned by the caller) in order
 *   nlevels_out  host, number of coarse contexts produced
 *   stats_out    host array of max_levels records, or NULL */
gr_status graph_reduce_multilevel(gr_ctx* fine, const gr_params* params, gr_ctx** levels_out,
                                  int* nlevels_out, gr_level_stats* stats_out);

/* Compose the maps of a chain of coarse contexts (levels[0] made from the
 * fine graph, levels[i] from levels[i-1]) into one fine -> coarsest map.
 *   agg_out  device, n_fine entries */
gr_status graph_reduce_compose_maps(gr_ctx* const* levels, int nlevels, int32_t* agg_out);

/* Spectral-mismatch loss on a reduced graph with free edge weights w_c (not
 * in the paper; it makes the edge-weight sensitivity of Sec. 3.3.3 an exact
 * gradient).  With x_k the columns of X on the fine graph, P the map `agg`
 * (fine -> coarse context nodes) and M_A = |{i : agg[i] = A}|:
 *   R_f[k] = x_k^T L_G x_k / x_k^T x_k
 *   y_0    = M^-1 P^T X                      (aggregate means)
 *   y_{s+1} = (1-omega) y_s + omega D_c^-1 A_c y_s,  s < sweeps_c,
 *            where A_c, D_c use the weights w_c on the coarse edge list
 *   R_c[k] = y^T L_c y / sum_A M_A (y_A - mu_k)^2,  mu_k = sum M_A y_A / sum M
 *   loss   = (1/K) sum_k (R_c[k] / R_f[k] - 1)^2
 *   X        device float, fine n x K;  w_c  device float, coarse m entries
 *   loss_out device float scalar
 *   saved    device float, coarse_n*(K+1) + K entries: receives y_0, R_f and M
 *            for graph_reduce_loss_bwd (nothing else is kept)
 * K: 4, 8, 16, 24 or 32. */
gr_status graph_reduce_loss_fwd(gr_ctx* fine, gr_ctx* coarse, const int32_t* agg, const float* X,
                                int K, const float* w_c, int sweeps_c, double omega,
                                float* loss_out, float* saved);

/* Adjoint of graph_reduce_loss_fwd with respect to w_c: recomputes the
 * sweeps from the saved y_0, then runs the reverse sweeps.
 *   grad_loss   device float scalar (upstream gradient)
 *   grad_w_out  device float, coarse m entries (overwritten) */
gr_status graph_reduce_loss_bwd(gr_ctx* coarse, const float* saved, int K, const float* w_c,
                                int sweeps_c, double omega, const float* grad_loss,
                                float* grad_w_out);

/* Edge-weight scaling of the reduced graph by constrained SGD with momentum
 * (Alg. 1; Eqs. formula_weight_sensitivity2, courant-fischer-3),
 * driven by the exact gradient of the spectral-mismatch loss
 * (graph_reduce_loss_fwd / _bwd).  Alg. 1 scales a sparsifier P of G; here
 * L_P is `coarse` with the weights being scaled and L_G the same graph with
 * the initial weights, so the lambda_1 estimate min_p d_G(p)/d_P(p) starts at
 * 1.  The loss stands in for lambda_n (which needs a Laplacian solver): its
 * gradient is the sensitivity, eta_k = (loss_k / loss_1) eta_max, and the loop
 * stops when (loss_{k-1} - loss_k) / loss_k < eps or after kmax iterations.
 * Per iteration every edge, from the degrees at the iteration's start (the
 * paper gives no edge order), takes dw <- max(alpha dw - eta grad, 0); if
 * min(d_G(p)/(d_P(p)+dw), d_G(q)/(d_P(q)+dw)) <= lambda_1 Delta, with
 * Delta = delta_bar^(1/kmax), dw is capped to keep that ratio at the bound
 * (never below 0); w += dw; then d_P and lambda_1 are recomputed.
 *   agg, X, K, sweeps_c, omega   as for graph_reduce_loss_fwd
 *   w_inout        device, coarse m FP32: the initial weights in, scaled out
 *   iters_out      host, iterations that updated the weights
 *   loss_hist      host, kmax entries or NULL: the loss before each update
 *   lambda1_hist   host, kmax entries or NULL: lambda_1 after each update */
gr_status graph_reduce_scale_edges(gr_ctx* fine, gr_ctx* coarse, const int32_t* agg, const float* X, int K,
                                   int sweeps_c, double omega, double alpha, double eta_max, double delta_bar,
                                   double eps, int kmax, float* w_inout, int32_t* iters_out, double* loss_hist,
                                   double* lambda1_hist);

/* Number of kernels this library has launched in the process so far (a
 * diagnostic counter, not tied to any paper passage). */
uint64_t graph_reduce_launch_count(void);

/* Text of the last error on ctx (or of the last failed create when ctx is
 * NULL).  Valid until the next call on the same context. */
const char* graph_reduce_last_error(const gr_ctx* ctx);

/* Release a context and everything it owns.  NULL-safe. */
void graph_reduce_destroy(gr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GRAPH_REDUCE_H */
