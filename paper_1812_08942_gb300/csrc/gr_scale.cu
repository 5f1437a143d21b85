// Edge-weight scaling of a reduced graph by constrained SGD with momentum
// (Alg. 1), driven by the exact gradient of the spectral-mismatch loss.
//
// L_P is the reduced graph with the weights being scaled, L_G the same graph
// with its initial weights, so the lambda_1 estimate min_p d_G(p) / d_P(p)
// (Eq. courant-fischer-3) starts at 1.  The loss stands in for lambda_n:
// its gradient is the weight sensitivity, its ratio to the first loss scales
// the step size, its relative decrease is the convergence test.
// Every edge of an iteration updates from the degrees at the iteration's start
// (the paper gives no edge order, and this order parallelises); updates never
// go below zero, as the scheme only scales weights up.
#include "gr_internal.cuh"

namespace gr {

namespace {

constexpr int ST = 256;

// for every edge: momentum step, the lambda_1 guard, the update
__global__ void k_sgd_edges(int64_t m, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev,
                            const float* __restrict__ grad, const double* __restrict__ dG,
                            const double* __restrict__ dP, double bound, double alpha, double eta,
                            float* __restrict__ dw, float* __restrict__ w) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t p = eu[e], q = ev[e];
    double d = alpha * (double)dw[e] - eta * (double)grad[e];
    d = d > 0.0 ? d : 0.0;
    const double phi_p = dG[p] / (dP[p] + d), phi_q = dG[q] / (dP[q] + d);
    if ((phi_p < phi_q ? phi_p : phi_q) <= bound) {
        const double cp = dG[p] / bound - dP[p], cq = dG[q] / bound - dP[q];
        const double cap = cp < cq ? cp : cq;
        d = cap > 0.0 ? cap : 0.0;
    }
    dw[e] = (float)d;
    w[e] = (float)((double)w[e] + d);
}

// d_P(p) = sum of the row's current weights in slot order (= ascending edge id)
__global__ void k_row_weight_sums(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ eid,
                                  const float* __restrict__ w, double* __restrict__ d) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double s = 0.0;
    for (int64_t j = rowptr[p]; j < rowptr[p + 1]; ++j) s += (double)w[eid[j]];
    d[p] = s;
}

// lambda_1 estimate: min over nodes with d_P > 0 of d_G / d_P (positive
// doubles order like their bit patterns, so an integer minimum is exact)
__global__ void k_min_ratio(int64_t n, const double* __restrict__ dG, const double* __restrict__ dP,
                            unsigned long long* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = ~0ull;
    if (p < n && dP[p] > 0.0) v = (unsigned long long)__double_as_longlong(dG[p] / dP[p]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, v, o);
        v = x < v ? x : v;
    }
    if ((threadIdx.x & 31) == 0 && v != ~0ull) atomicMin(out, v);
}

__global__ void k_set_f32(float* __restrict__ p, float v) { *p = v; }

}  // namespace

gr_status scale_edges_impl(gr_ctx* fine, gr_ctx* coarse, const int32_t* agg, const float* X, int K, int sweeps,
                           double omega, double alpha, double eta_max, double delta_bar, double eps, int kmax,
                           float* w, int32_t* iters_out, double* loss_hist, double* lam1_hist) {
    cudaStream_t s = fine->stream;
    const int64_t nc = coarse->n, mc = coarse->m;
    size_t need = 0;
    auto add = [&](size_t bytes) {
        size_t off = need;
        need += (bytes + 255) & ~size_t(255);
        return off;
    };
    const size_t o_dG = add(8 * (size_t)nc), o_dP = add(8 * (size_t)nc), o_dw = add(4 * (size_t)mc),
                 o_g = add(4 * (size_t)mc), o_saved = add(4 * ((size_t)nc * (K + 1) + K)), o_sc = add(64);
    void* base;
    GR_TRY_CUDA(fine, fine->ws.get(WS_SCALE, need, &base), "scaling scratch");
    char* B = (char*)base;
    double* dG = (double*)(B + o_dG);
    double* dP = (double*)(B + o_dP);
    float* dw = (float*)(B + o_dw);
    float* grad = (float*)(B + o_g);
    float* saved = (float*)(B + o_saved);
    float* loss = (float*)(B + o_sc);
    float* one = loss + 1;
    unsigned long long* lmin = (unsigned long long*)(B + o_sc + 8);
    int64_t* hs = host_scratch();
    if (!hs) return set_error(fine, GR_ENOMEM, "scale_edges: pinned scratch unavailable");
    const unsigned gn = (unsigned)ceil_div(nc > 0 ? nc : 1, ST), gm = (unsigned)ceil_div(mc > 0 ? mc : 1, ST);

    GR_TRY_CUDA(fine, cudaMemsetAsync(dw, 0, 4 * (size_t)mc, s), "memset");
    k_set_f32<<<1, 1, 0, s>>>(one, 1.0f);
    count_launch();
    k_row_weight_sums<<<gn, ST, 0, s>>>(nc, coarse->rowptr, coarse->eid, w, dG);
    count_launch();
    GR_TRY_CUDA(fine, cudaMemcpyAsync(dP, dG, 8 * (size_t)nc, cudaMemcpyDeviceToDevice, s), "copy");
    const double step_delta = pow(delta_bar, 1.0 / kmax);  // per-iteration share of the bound
    double lam1 = 1.0, eta = eta_max, L0 = 0.0, L_prev = 0.0;
    int it = 0;
    for (int k = 1; k <= kmax; ++k) {
        gr_status st = loss_fwd_impl(fine, coarse, agg, X, K, w, sweeps, omega, loss, saved);
        if (st != GR_OK) return st;
        GR_TRY_CUDA(fine, cudaMemcpyAsync(hs, loss, 4, cudaMemcpyDeviceToHost, s), "readback");
        GR_TRY_CUDA(fine, cudaStreamSynchronize(s), "sync");
        const double L = (double)((const float*)hs)[0];
        if (k == 1) L0 = L;
        if (k > 1 && (L_prev - L) / L < eps) break;  // convergence test
        st = loss_bwd_impl(coarse, saved, K, w, sweeps, omega, one, grad);
        if (st != GR_OK) return st;
        if (mc > 0) {
            k_sgd_edges<<<gm, ST, 0, s>>>(mc, coarse->eu, coarse->ev, grad, dG, dP, lam1 * step_delta, alpha, eta,
                                         dw, w);
            count_launch();
        }
        k_row_weight_sums<<<gn, ST, 0, s>>>(nc, coarse->rowptr, coarse->eid, w, dP);
        count_launch();
        GR_TRY_CUDA(fine, cudaMemsetAsync(lmin, 0xff, 8, s), "memset");
        k_min_ratio<<<gn, ST, 0, s>>>(nc, dG, dP, lmin);
        count_launch();
        GR_TRY_CUDA(fine, cudaMemcpyAsync(hs, lmin, 8, cudaMemcpyDeviceToHost, s), "readback");
        GR_TRY_CUDA(fine, cudaStreamSynchronize(s), "sync");
        const unsigned long long bits = ((const unsigned long long*)hs)[0];
        if (bits != ~0ull) {
            double r;
            memcpy(&r, &bits, 8);
            lam1 = r;  // new lambda_1 estimate
        }
        eta = (L / L0) * eta_max;  // step size from the loss ratio
        if (loss_hist) loss_hist[it] = L;
        if (lam1_hist) lam1_hist[it] = lam1;
        ++it;
        L_prev = L;
    }
    if (iters_out) *iters_out = it;
    GR_TRY_CUDA(fine, cudaGetLastError(), "scale_edges kernels");
    return GR_OK;
}

}  // namespace gr
