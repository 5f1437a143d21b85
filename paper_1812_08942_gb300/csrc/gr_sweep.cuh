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

// Partials are combined in two levels: blocks form groups of STATS_GROUP
// consecutive blocks; the last block of a group to finish (one ticket per
// group) sums its group's partial rows and stores the group sum in the
// group's first row; the last group to finish (the kernel's ticket) sums the
// group rows and writes the statistics.  Each finishing block reads at most
// max(STATS_GROUP, groups) rows, one round of loads in flight, where one
// block summing every partial row would wait on a dozen dependent rounds of
// L2 loads (k_init's 912 partials on 152 SMs).  The order of the additions
// depends only on the number of blocks, so results are reproducible.
//
// Counter words (all zero before the kernel; the finishing blocks reset them):
//   counter[0]                       kernel ticket
//   counter[1]                       the band sweep's error word
//   counter[STATS_GCOUNT_OFF + g]    ticket of group g < STATS_MAX_GROUPS
constexpr int STATS_GROUP = 32;
constexpr int STATS_MAX_GROUPS = 64;
constexpr int STATS_GCOUNT_OFF = 16;
// bytes of counter words that follow the statistics sets
constexpr size_t STATS_COUNTER_BYTES = sizeof(unsigned) * (STATS_GCOUNT_OFF + STATS_MAX_GROUPS);

// red[s] = sum over r < nrows of base[r * rstride + s], s < 2K, in a fixed
// order (each of the first PER * 2K threads sums every PER-th row with eight
// interleaved accumulators, then the PER sums of a column are added in
// order).  Every thread of the block must call it (block barriers).
template <int K, int NT>
__device__ __forceinline__ void sum_partial_rows(const double* base, int nrows, int64_t rstride,
                                                 double* red) {
    constexpr int NS = 2 * K;
    constexpr int PER = NT / NS > 0 ? NT / NS : 1;
    const int t = threadIdx.x;
    const int stat = t % NS;
    const int sub = t / NS;
    double acc = 0.0;
    if (t < NT && sub < PER) {
        double a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = 0.0;
        int r = sub;
        for (; r + 7 * PER < nrows; r += 8 * PER) {
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] += __ldcg(base + (int64_t)(r + u * PER) * rstride + stat);
        }
        for (; r < nrows; r += PER) a[0] += __ldcg(base + (int64_t)r * rstride + stat);
        acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
    if (t < NT) red[t] = acc;
    __syncthreads();
    if (t < NS) {
        double s = 0.0;
        for (int j = 0; j < PER; ++j) s += red[j * NS + t];
        red[t] = s;  // row 0 of red is read only by its own thread above
    }
    __syncthreads();
}

// Called by every thread of a block once its partial row part[blockIdx.x]
// (2K doubles: the K column sums, then the K sums of squares) is written and
// fenced.  The last block overall writes mu = s1 / n and 1 / s with
// s^2 = s2 - n mu^2 into stats_out.  NT >= 2K threads take part in the sums.
template <int K, int NT>
__device__ void finish_stats(double* part, int nblocks, unsigned* counter, int64_t n,
                             double* __restrict__ stats_out) {
    constexpr int NS = 2 * K;
    __shared__ double red[NT];
    __shared__ int s_go;
    const int t = threadIdx.x;
    const int g = blockIdx.x / STATS_GROUP, g0 = g * STATS_GROUP;
    const int gs = min(STATS_GROUP, nblocks - g0);
    const int ngroups = (nblocks + STATS_GROUP - 1) / STATS_GROUP;
    unsigned* gcount = counter + STATS_GCOUNT_OFF;
    if (t == 0) s_go = atomicAdd(gcount + g, 1u) == (unsigned)(gs - 1);
    __syncthreads();
    if (!s_go) return;
    __threadfence();
    sum_partial_rows<K, NT>(part + (int64_t)g0 * NS, gs, NS, red);
    // every row of the group has been read (barrier above): the group sum
    // takes the group's first row
    if (t < NS) part[(int64_t)g0 * NS + t] = red[t];
    if (t == 0) gcount[g] = 0u;
    __threadfence();
    __syncthreads();
    if (t == 0) s_go = atomicAdd(counter, 1u) == (unsigned)(ngroups - 1);
    __syncthreads();
    if (!s_go) return;
    __threadfence();
    sum_partial_rows<K, NT>(part, ngroups, (int64_t)STATS_GROUP * NS, red);
    if (t < K) {
        double s1 = red[t], s2 = red[K + t];
        double mu = s1 / (double)n;
        double var = s2 - (double)n * mu * mu;
        double sd = var > 0.0 ? sqrt(var) : 0.0;
        stats_out[t] = mu;
        stats_out[K + t] = sd > 0.0 ? 1.0 / sd : 1.0;
    }
    if (t == 0) *counter = 0u;
}

}  // namespace gr
