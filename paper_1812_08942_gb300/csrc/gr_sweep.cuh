// Column statistics shared by the sweep kernels (Sec. 3.2.1: the test vectors
// are kept orthogonal to the all-ones vector and of unit norm between sweeps).
//
// Every sweep kernel sums, per column k, s1 = sum_i y_ik and s2 = sum_i y_ik^2
// of the block it stores, block by block; the last block to finish turns the
// per-block partial sums (FP64) into mu = s1 / n and 1 / s with
// s^2 = s2 - n mu^2, in a fixed order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gr {

// Finish of the column statistics: 2K sums over `nblocks` partials.  The
// first NT threads of the block do the work; every thread of the block must
// call it (it holds block barriers).
template <int K, int NT>
__device__ void finish_stats(const double* __restrict__ part, int nblocks, int64_t n,
                             double* __restrict__ stats_out) {
    // 2K sums, each split over NT / (2K) threads, then combined in order
    constexpr int NS = 2 * K;
    constexpr int PER = NT / NS > 0 ? NT / NS : 1;
    __shared__ double red[NT];
    const int t = threadIdx.x;
    const int stat = t % NS;
    const int sub = t / NS;
    // eight interleaved accumulators keep eight loads in flight; the order of
    // the additions depends only on nblocks, so results are reproducible
    double acc = 0.0;
    if (t < NT && sub < PER) {
        double a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = 0.0;
        int b = sub;
        for (; b + 7 * PER < nblocks; b += 8 * PER) {
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] += __ldcg(part + (int64_t)(b + u * PER) * NS + stat);
        }
        for (; b < nblocks; b += PER) a[0] += __ldcg(part + (int64_t)b * NS + stat);
        acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
    if (t < NT) red[t] = acc;
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

}  // namespace gr
