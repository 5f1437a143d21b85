// The C ABI (include/graph_reduce.h): argument checks, context lifetime, the
// level loop.  No exception crosses this boundary.
#include <math.h>
#include <string.h>

#include <new>
#include <string>

#include <vector>

#include "gr_internal.cuh"

namespace gr {

static thread_local std::string g_create_error;

gr_status set_error(gr_ctx* c, gr_status st, const std::string& msg) {
    if (c) c->last_error = msg;
    else g_create_error = msg;
    return st;
}

gr_status cuda_error(gr_ctx* c, cudaError_t e, const char* where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    gr_status st = (e == cudaErrorMemoryAllocation) ? GR_ENOMEM : GR_ECUDA;
    return set_error(c, st, msg);
}

gr_status compose_impl(gr_ctx* const* levels, int nlevels, int32_t* out);

static bool valid_K(int K) { return K == 4 || K == 8 || K == 16 || K == 24 || K == 32; }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// canonical-list check on the host
static bool host_canonical(int64_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w,
                           std::string* why) {
    for (int64_t e = 0; e < m; ++e) {
        if (u[e] < 0 || v[e] >= n || !(u[e] < v[e])) {
            *why = "edge " + std::to_string(e) + " is not 0 <= u < v < n";
            return false;
        }
        if (e > 0 && (u[e] < u[e - 1] || (u[e] == u[e - 1] && v[e] <= v[e - 1]))) {
            *why = "edge " + std::to_string(e) + " breaks the sorted, duplicate-free order";
            return false;
        }
        if (!(w[e] > 0.0) || !isfinite(w[e])) {
            *why = "edge " + std::to_string(e) + " has a weight that is not finite and > 0";
            return false;
        }
    }
    return true;
}


}  // namespace gr

using namespace gr;

extern "C" {

gr_status graph_reduce_create(gr_ctx** out, int64_t n, int64_t m, const int32_t* u, const int32_t* v,
                              const double* w, int inputs_on_host, void* cuda_stream) {
    if (!out) return set_error(nullptr, GR_EINVAL, "create: out is NULL");
    *out = nullptr;
    if (n < 1 || n >= (1ll << 31)) return set_error(nullptr, GR_EINVAL, "create: n must be in [1, 2^31)");
    if (m < 0 || m >= (1ll << 31)) return set_error(nullptr, GR_EINVAL, "create: m must be in [0, 2^31)");
    if (m > 0 && (!u || !v || !w)) return set_error(nullptr, GR_EINVAL, "create: edge arrays are NULL");
    gr_ctx* c = new (std::nothrow) gr_ctx();
    if (!c) return set_error(nullptr, GR_ENOMEM, "create: host allocation failed");
    c->n = n;
    c->m = m;
    c->stream = (cudaStream_t)cuda_stream;
    c->ws.stream = c->stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) tune_mempool(c->device);
    int64_t* hs = host_scratch();
    if (e == cudaSuccess && !hs) e = cudaErrorMemoryAllocation;
    size_t me = (size_t)(m > 0 ? m : 1);
    if (e == cudaSuccess) e = cudaMallocAsync(&c->eu, sizeof(int32_t) * me, c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&c->ev, sizeof(int32_t) * me, c->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&c->ew, sizeof(double) * me, c->stream);
    cudaMemcpyKind kind = inputs_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(c->eu, u, sizeof(int32_t) * m, kind, c->stream);
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(c->ev, v, sizeof(int32_t) * m, kind, c->stream);
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(c->ew, w, sizeof(double) * m, kind, c->stream);
    if (e != cudaSuccess) {
        cuda_error(nullptr, e, "create");
        graph_reduce_destroy(c);
        return e == cudaErrorMemoryAllocation ? GR_ENOMEM : GR_ECUDA;
    }
    // host or device inputs: checked on the device after the copy, in the
    // first pass of the CSR build
    bool invalid = false;
    gr_status st = build_csr(c, true, &invalid);
    if (st != GR_OK) {
        if (invalid) {
            std::string why = "the edge list is not canonical (u < v < n, sorted, unique, w > 0 finite)";
            if (inputs_on_host) host_canonical(n, m, u, v, w, &why);  // name the first bad edge
            set_error(nullptr, GR_EINVAL, "create: " + why);
        } else {
            set_error(nullptr, st, c->last_error);
        }
        graph_reduce_destroy(c);
        return st;
    }
    *out = c;
    return GR_OK;
}

gr_status graph_reduce_get_info(const gr_ctx* ctx, int64_t* n_out, int64_t* m_out) {
    if (!ctx) return GR_EINVAL;
    if (n_out) *n_out = ctx->n;
    if (m_out) *m_out = ctx->m;
    return GR_OK;
}

gr_status graph_reduce_set_sweep_kernel(gr_ctx* ctx, gr_sweep_kernel kind) {
    if (!ctx) return set_error(nullptr, GR_EINVAL, "set_sweep_kernel: ctx is NULL");
    if ((int)kind < (int)GR_SWEEP_AUTO || (int)kind > (int)GR_SWEEP_BAND)
        return set_error(ctx, GR_EINVAL, "set_sweep_kernel: unknown kernel");
    ctx->sweep_kind = (int)kind;
    return GR_OK;
}

gr_status graph_reduce_sweep_plan(gr_ctx* ctx, int K, gr_prec prec, int32_t* kernel_out) {
    if (!ctx) return set_error(nullptr, GR_EINVAL, "sweep_plan: ctx is NULL");
    if (!valid_K(K)) return set_error(ctx, GR_EINVAL, "sweep_plan: K must be 4, 8, 16, 24 or 32");
    if (!kernel_out) return set_error(ctx, GR_EINVAL, "sweep_plan: kernel_out is NULL");
    return sweep_plan_impl(ctx, K, prec, kernel_out);
}

gr_status graph_reduce_smooth(gr_ctx* ctx, int K, int sweeps, double omega, uint64_t seed, int level,
                              gr_prec prec, void* X) {
    if (!ctx) return set_error(nullptr, GR_EINVAL, "smooth: ctx is NULL");
    if (!valid_K(K)) return set_error(ctx, GR_EINVAL, "smooth: K must be 4, 8, 16, 24 or 32");
    if (sweeps < 0 || !(omega > 0.0 && omega <= 1.0))
        return set_error(ctx, GR_EINVAL, "smooth: need sweeps >= 0 and 0 < omega <= 1");
    if (level < 0 || level >= (1 << 20)) return set_error(ctx, GR_EINVAL, "smooth: level out of range");
    if (!X || !aligned16(X)) return set_error(ctx, GR_EINVAL, "smooth: X must be a 16-byte aligned device pointer");
    if (prec != GR_F64 && prec != GR_F32 && prec != GR_BF16) return set_error(ctx, GR_EINVAL, "smooth: bad precision");
    return smooth_impl(ctx, K, sweeps, omega, seed, level, prec, X);
}

gr_status graph_reduce_test_vectors(gr_ctx* ctx, int K, uint64_t seed, int level, gr_prec prec, void* X) {
    if (!ctx) return set_error(nullptr, GR_EINVAL, "test_vectors: ctx is NULL");
    if (!valid_K(K)) return set_error(ctx, GR_EINVAL, "test_vectors: K must be 4, 8, 16, 24 or 32");
    if (level < 0 || level >= (1 << 20)) return set_error(ctx, GR_EINVAL, "test_vectors: level out of range");
    if (!X || !aligned16(X))
        return set_error(ctx, GR_EINVAL, "test_vectors: X must be a 16-byte aligned device pointer");
    if (prec != GR_F64 && prec != GR_F32 && prec != GR_BF16)
        return set_error(ctx, GR_EINVAL, "test_vectors: bad precision");
    return test_vectors_impl(ctx, K, seed, level, prec, X);
}

gr_status graph_reduce_smooth_gs(gr_ctx* ctx, int K, int sweeps, double omega, uint64_t seed, int level,
                                 uint64_t colour_seed, gr_prec prec, void* X) {
    if (!ctx) return set_error(nullptr, GR_EINVAL, "smooth_gs: ctx is NULL");
    if (!valid_K(K)) return set_error(ctx, GR_EINVAL, "smooth_gs: K must be 4, 8, 16, 24 or 32");
    if (sweeps < 0 || !(omega > 0.0 && omega <= 1.0))
        return set_error(ctx, GR_EINVAL, "smooth_gs: need sweeps >= 0 and 0 < omega <= 1");
    if (level < 0 || level >= (1 << 20)) return set_error(ctx, GR_EINVAL, "smooth_gs: level out of range");
    if (!X || !aligned16(X)) return set_error(ctx, GR_EINVAL, "smooth_gs: X must be a 16-byte aligned device pointer");
    if (prec != GR_F64 && prec != GR_F32 && prec != GR_BF16)
        return set_error(ctx, GR_EINVAL, "smooth_gs: bad precision");
    return smooth_gs_impl(ctx, K, sweeps, omega, seed, level, colour_seed, prec, X);
}

gr_status graph_reduce_colour(gr_ctx* ctx, uint64_t colour_seed, int32_t* colour_out, int32_t* ncolours_out) {
    if (!ctx) return set_error(nullptr, GR_EINVAL, "colour: ctx is NULL");
    if (!colour_out || !ncolours_out) return set_error(ctx, GR_EINVAL, "colour: NULL output");
    return colour_impl(ctx, colour_seed, colour_out, ncolours_out);
}

gr_status graph_reduce_affinity(gr_ctx* ctx, const void* X, int K, gr_prec prec, void* d_out, void* a_out) {
    if (!ctx) return set_error(nullptr, GR_EINVAL, "affinity: ctx is NULL");
    if (!valid_K(K)) return set_error(ctx, GR_EINVAL, "affinity: K must be 4, 8, 16, 24 or 32");
    if (!X || !aligned16(X) || !d_out) return set_error(ctx, GR_EINVAL, "affinity: X (16-byte aligned) and d_out required");
    if (prec != GR_F64 && prec != GR_F32 && prec != GR_BF16) return set_error(ctx, GR_EINVAL, "affinity: bad precision");
    return affinity_impl(ctx, X, K, prec, d_out, a_out);
}

gr_status graph_reduce_aggregate(gr_ctx* ctx, const void* d, int d_is_f64, int64_t target_nc, int passes,
                                 int64_t max_proposals, int32_t* agg_out, int64_t* nc_out,
                                 int64_t* proposals_out) {
    if (!ctx) return set_error(nullptr, GR_EINVAL, "aggregate: ctx is NULL");
    if (!agg_out || !nc_out || (ctx->m > 0 && !d)) return set_error(ctx, GR_EINVAL, "aggregate: NULL argument");
    if (target_nc < 1 || passes < 0 || passes > 30)
        return set_error(ctx, GR_EINVAL, "aggregate: need target_nc >= 1 and 0 <= passes <= 30");
    if (proposals_out) *proposals_out = 0;
    return aggregate_impl(ctx, d, d_is_f64, target_nc, passes, max_proposals, agg_out, nc_out, proposals_out);
}

gr_status graph_reduce_coarsen(gr_ctx* ctx, const int32_t* agg, int64_t nc, gr_ctx** coarse_out) {
    if (!ctx) return set_error(nullptr, GR_EINVAL, "coarsen: ctx is NULL");
    if (!agg || !coarse_out) return set_error(ctx, GR_EINVAL, "coarsen: NULL argument");
    *coarse_out = nullptr;
    return coarsen_impl(ctx, agg, nc, coarse_out);
}

gr_status graph_reduce_get_edges(const gr_ctx* cctx, int64_t* m_out, int32_t* u, int32_t* v, double* w,
                                 int outputs_on_host) {
    gr_ctx* ctx = const_cast<gr_ctx*>(cctx);
    if (!ctx) return set_error(nullptr, GR_EINVAL, "get_edges: ctx is NULL");
    if (m_out) *m_out = ctx->m;
    if (ctx->m == 0) return GR_OK;
    cudaMemcpyKind kind = outputs_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (u) GR_TRY_CUDA(ctx, cudaMemcpyAsync(u, ctx->eu, sizeof(int32_t) * ctx->m, kind, ctx->stream), "get_edges");
    if (v) GR_TRY_CUDA(ctx, cudaMemcpyAsync(v, ctx->ev, sizeof(int32_t) * ctx->m, kind, ctx->stream), "get_edges");
    if (w) GR_TRY_CUDA(ctx, cudaMemcpyAsync(w, ctx->ew, sizeof(double) * ctx->m, kind, ctx->stream), "get_edges");
    if (outputs_on_host) GR_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "get_edges");
    return GR_OK;
}

gr_status graph_reduce_get_map(const gr_ctx* cctx, int32_t* agg_out, int64_t* n_parent_out) {
    gr_ctx* ctx = const_cast<gr_ctx*>(cctx);
    if (!ctx) return set_error(nullptr, GR_EINVAL, "get_map: ctx is NULL");
    if (!ctx->parent_map) return set_error(ctx, GR_ESTATE, "get_map: context was not made by coarsen");
    if (n_parent_out) *n_parent_out = ctx->parent_n;
    if (agg_out)
        GR_TRY_CUDA(ctx, cudaMemcpyAsync(agg_out, ctx->parent_map, sizeof(int32_t) * ctx->parent_n,
                                         cudaMemcpyDeviceToDevice, ctx->stream), "get_map");
    return GR_OK;
}

gr_status graph_reduce_compose_maps(gr_ctx* const* levels, int nlevels, int32_t* agg_out) {
    if (!levels || nlevels < 1 || !levels[0] || !agg_out)
        return set_error(nullptr, GR_EINVAL, "compose_maps: need at least one level and an output");
    return compose_impl(levels, nlevels, agg_out);
}

gr_status graph_reduce_reduce_data(gr_ctx* const* levels, int nlevels, const void* F, int d, int f64, int mean,
                                   void* F_out) {
    if (!levels || nlevels < 1 || !levels[0]) return set_error(nullptr, GR_EINVAL, "reduce_data: no levels");
    gr_ctx* c0 = levels[0];
    if (d < 0 || (f64 != 0 && f64 != 1) || (mean != 0 && mean != 1))
        return set_error(c0, GR_EINVAL, "reduce_data: need d >= 0, f64 and mean in {0, 1}");
    if (d > 0 && (!F || !F_out)) return set_error(c0, GR_EINVAL, "reduce_data: NULL data");
    for (int l = 0; l < nlevels; ++l) {
        if (!levels[l] || !levels[l]->parent_map)
            return set_error(c0, GR_ESTATE, "reduce_data: every level must come from coarsen");
        if (l > 0 && levels[l]->parent_n != levels[l - 1]->n)
            return set_error(c0, GR_EINVAL, "reduce_data: levels do not chain");
    }
    return reduce_data_impl(levels, nlevels, F, d, f64, mean, F_out);
}

gr_status graph_reduce_eigensolve(gr_ctx* const* levels, int nlevels, int k, int normalized, int galerkin_mass,
                                  double omega, int iters, double* U_out, double* lambda_out, double* rayleigh_out) {
    if (!levels || nlevels < 1 || !levels[0]) return set_error(nullptr, GR_EINVAL, "eigensolve: no levels");
    gr_ctx* f = levels[0];
    if (!U_out || !lambda_out) return set_error(f, GR_EINVAL, "eigensolve: NULL output");
    if (k < 1 || k > 32 || iters < 0 || !(omega > 0.0 && omega <= 1.0) || (normalized != 0 && normalized != 1) ||
        (galerkin_mass != 0 && galerkin_mass != 1))
        return set_error(f, GR_EINVAL, "eigensolve: need 1 <= k <= 32, iters >= 0, 0 < omega <= 1, flags 0 or 1");
    for (int l = 1; l < nlevels; ++l) {
        if (!levels[l] || !levels[l]->parent_map || levels[l]->parent_n != levels[l - 1]->n)
            return set_error(f, GR_EINVAL, "eigensolve: each level must be coarsened from the one before");
    }
    const int64_t nc = levels[nlevels - 1]->n;
    if (nc > 16384) return set_error(f, GR_EINVAL, "eigensolve: the coarsest level must have at most 16384 nodes");
    if (k > nc) return set_error(f, GR_EINVAL, "eigensolve: k exceeds the coarsest level's size");
    return eigensolve_impl(levels, nlevels, k, normalized, galerkin_mass, omega, iters, U_out, lambda_out,
                           rayleigh_out);
}

// mean degree up to which the level loop leaves the last normalisation of
// the smoothed block to the affinity (measured on the 128^3 mesh, mean
// degree 6: 44 us less at level 0; on a Chung-Lu graph of mean degree 65:
// 22 us more per level)
constexpr double FUSE_MAX_MEAN_DEGREE = 16.0;

gr_status graph_reduce_multilevel(gr_ctx* fine, const gr_params* p, gr_ctx** levels_out, int* nlevels_out,
                                  gr_level_stats* stats_out) {
    if (!fine) return set_error(nullptr, GR_EINVAL, "multilevel: ctx is NULL");
    if (!p || !levels_out || !nlevels_out) return set_error(fine, GR_EINVAL, "multilevel: NULL argument");
    if (!valid_K(p->K) || p->sweeps < 0 || !(p->omega > 0.0 && p->omega <= 1.0) || p->passes < 1 ||
        p->passes > 30 || p->level_ratio < 2 || p->final_target < 1 || p->max_levels < 1 ||
        (p->prec != GR_F64 && p->prec != GR_F32 && p->prec != GR_BF16))
        return set_error(fine, GR_EINVAL, "multilevel: invalid parameters");
    *nlevels_out = 0;
    const gr_prec prec = (gr_prec)p->prec;
    const size_t xsz = prec == GR_F64 ? 8 : (prec == GR_F32 ? 4 : 2);
    const size_t dsz = prec == GR_F64 ? 8 : 4;
    cudaStream_t s = fine->stream;
    // seven events per level, read once after the loop (no per-level wait)
    const bool timed = stats_out != nullptr;
    std::vector<cudaEvent_t> evs;
    gr_ctx* cur = fine;
    gr_status st = GR_OK;
    int nl = 0;
    for (int lvl = 0; lvl < p->max_levels; ++lvl) {
        if (cur->n <= p->final_target || cur->m == 0) break;
        void *px, *pd, *pa;
        cudaError_t e = fine->ws.get(WS_ML_X, xsz * (size_t)cur->n * p->K, &px);
        if (e == cudaSuccess) e = fine->ws.get(WS_ML_D, dsz * (size_t)cur->m, &pd);
        if (e == cudaSuccess) e = fine->ws.get(WS_ML_AGG, sizeof(int32_t) * (size_t)cur->n, &pa);
        if (e != cudaSuccess) {
            st = cuda_error(fine, e, "multilevel scratch");
            break;
        }
        cudaEvent_t* ev = nullptr;
        if (timed) {
            for (int i = 0; i < 7; ++i) {
                cudaEvent_t e = nullptr;
                if (cudaEventCreate(&e) != cudaSuccess) {
                    st = set_error(fine, GR_ECUDA, "multilevel: event");
                    break;
                }
                evs.push_back(e);
            }
            if (st != GR_OK) break;
            ev = &evs[(size_t)7 * lvl];
        }
        if (timed) cudaEventRecord(ev[0], s);
        // the smoothed block is read only by the affinity, which can apply the
        // last normalisation itself (one pass over the block fewer; it then
        // normalises both rows of every edge, which pays on sparse graphs)
        const bool fuse = 2.0 * (double)cur->m <= FUSE_MAX_MEAN_DEGREE * (double)cur->n;
        SmoothRaw raw{px, nullptr};
        st = smooth_impl(cur, p->K, p->sweeps, p->omega, p->seed, lvl, prec, px, timed ? ev[5] : nullptr,
                         timed ? ev[6] : nullptr, fuse ? &raw : nullptr);
        if (timed) cudaEventRecord(ev[1], s);
        if (st == GR_OK) st = affinity_impl(cur, raw.A, p->K, prec, pd, nullptr, raw.stats);
        if (timed) cudaEventRecord(ev[2], s);
        int64_t target = (cur->n + p->level_ratio - 1) / p->level_ratio;
        if (target < p->final_target) target = p->final_target;
        int64_t nc = 0;
        int64_t proposals = 0;
        if (st == GR_OK)
            st = aggregate_impl(cur, pd, prec == GR_F64, target, p->passes, p->max_proposals, (int32_t*)pa, &nc,
                                &proposals);
        if (timed) cudaEventRecord(ev[3], s);
        if (st != GR_OK) {
            if (cur != fine) fine->last_error = cur->last_error;
            break;
        }
        if (nc == cur->n) break;  // no merge possible
        gr_ctx* next = nullptr;
        st = coarsen_impl(cur, (const int32_t*)pa, nc, &next);
        if (timed) cudaEventRecord(ev[4], s);
        if (st != GR_OK) {
            if (cur != fine) fine->last_error = cur->last_error;
            break;
        }
        if (timed) {
            gr_level_stats& L = stats_out[nl];
            L.n = cur->n;
            L.m = cur->m;
            L.nc = next->n;
            L.mc = next->m;
            L.proposals = proposals;
            L.sweeps = p->sweeps;
        }
        levels_out[nl++] = next;
        cur = next;
    }
    if (timed) {
        if (nl > 0) cudaEventSynchronize(evs[(size_t)7 * (nl - 1) + 4]);
        for (int l = 0; l < nl; ++l) {
            const cudaEvent_t* ev = &evs[(size_t)7 * l];
            gr_level_stats& L = stats_out[l];
            cudaEventElapsedTime(&L.t_smooth, ev[0], ev[1]);
            cudaEventElapsedTime(&L.t_affinity, ev[1], ev[2]);
            cudaEventElapsedTime(&L.t_aggregate, ev[2], ev[3]);
            cudaEventElapsedTime(&L.t_coarsen, ev[3], ev[4]);
            L.t_sweeps = 0.f;
            if (p->sweeps > 0) cudaEventElapsedTime(&L.t_sweeps, ev[5], ev[6]);
        }
        for (auto& e : evs) cudaEventDestroy(e);
    }
    *nlevels_out = nl;
    return st;
}

gr_status graph_reduce_loss_fwd(gr_ctx* fine, gr_ctx* coarse, const int32_t* agg, const float* X, int K,
                                const float* w_c, int sweeps_c, double omega, float* loss_out, float* saved) {
    if (!fine || !coarse) return set_error(fine, GR_EINVAL, "loss_fwd: NULL context");
    if (!agg || !X || !w_c || !loss_out || !saved) return set_error(fine, GR_EINVAL, "loss_fwd: NULL argument");
    if (!valid_K(K) || sweeps_c < 0 || !(omega > 0.0 && omega <= 1.0))
        return set_error(fine, GR_EINVAL, "loss_fwd: need K in {4,8,16,24,32}, sweeps >= 0, 0 < omega <= 1");
    if (coarse->stream != fine->stream) return set_error(fine, GR_EINVAL, "loss_fwd: contexts must share a stream");
    return loss_fwd_impl(fine, coarse, agg, X, K, w_c, sweeps_c, omega, loss_out, saved);
}

gr_status graph_reduce_loss_bwd(gr_ctx* coarse, const float* saved, int K, const float* w_c, int sweeps_c,
                                double omega, const float* grad_loss, float* grad_w_out) {
    if (!coarse) return set_error(nullptr, GR_EINVAL, "loss_bwd: NULL context");
    if (!saved || !w_c || !grad_loss || !grad_w_out) return set_error(coarse, GR_EINVAL, "loss_bwd: NULL argument");
    if (!valid_K(K) || sweeps_c < 0 || !(omega > 0.0 && omega <= 1.0))
        return set_error(coarse, GR_EINVAL, "loss_bwd: need K in {4,8,16,24,32}, sweeps >= 0, 0 < omega <= 1");
    return loss_bwd_impl(coarse, saved, K, w_c, sweeps_c, omega, grad_loss, grad_w_out);
}

gr_status graph_reduce_scale_edges(gr_ctx* fine, gr_ctx* coarse, const int32_t* agg, const float* X, int K,
                                   int sweeps_c, double omega, double alpha, double eta_max, double delta_bar,
                                   double eps, int kmax, float* w_inout, int32_t* iters_out, double* loss_hist,
                                   double* lambda1_hist) {
    if (!fine || !coarse) return set_error(fine, GR_EINVAL, "scale_edges: NULL context");
    if (!agg || !X || !w_inout) return set_error(fine, GR_EINVAL, "scale_edges: NULL argument");
    if (!valid_K(K) || sweeps_c < 0 || !(omega > 0.0 && omega <= 1.0))
        return set_error(fine, GR_EINVAL, "scale_edges: need K in {4,8,16,24,32}, sweeps >= 0, 0 < omega <= 1");
    if (!(alpha >= 0.0 && alpha < 1.0) || !(eta_max >= 0.0) || !(delta_bar > 0.0 && delta_bar <= 1.0) ||
        !(eps == eps) || kmax < 1)
        return set_error(fine, GR_EINVAL, "scale_edges: need 0 <= alpha < 1, eta_max >= 0, 0 < delta_bar <= 1, kmax >= 1");
    if (coarse->stream != fine->stream) return set_error(fine, GR_EINVAL, "scale_edges: contexts must share a stream");
    return scale_edges_impl(fine, coarse, agg, X, K, sweeps_c, omega, alpha, eta_max, delta_bar, eps, kmax, w_inout,
                            iters_out, loss_hist, lambda1_hist);
}

uint64_t graph_reduce_launch_count(void) { return launch_count(); }

const char* graph_reduce_last_error(const gr_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

void graph_reduce_destroy(gr_ctx* c) {
    if (!c) return;
    cudaStream_t s = c->stream;
    void* ptrs[] = {c->eu, c->ev, c->ew, c->eptr, c->rowptr, c->col, c->eid, c->cw32, c->wn64, c->deg,
                    c->parent_map, c->wpart, c->cw64, c->gs_order, c->band_runs, c->band_slots};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, s);
    c->ws.release();
    delete c;
}

}  // extern "C"
