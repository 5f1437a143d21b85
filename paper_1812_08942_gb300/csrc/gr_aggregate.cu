// Node aggregation by algebraic distance (Sec. 3.2.2).
//
// Edges are ordered by the key (d, edge id), a strict total order.  A pass
// computes the greedy matching of the current cluster graph in that order
// with the suitor algorithm (Manne & Halappanavar 2014): lock-free proposals
// resolved by an atomic minimum per cluster, one kernel per pass.  With a
// strict total order the result is the unique locally-dominant matching,
// equal to the sequential greedy one (Preis 1999).  A pass that would exceed
// the allowed merge count keeps its smallest keys, which equals stopping the
// greedy scan early.  Clusters are identified by their smallest fine node; a
// cluster's members form a linked list starting there.
#include "gr_internal.cuh"

namespace gr {

struct Key {
    uint64_t hi;
    uint32_t lo;
};
__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// FP64 distance key: double bits in hi, edge id in lo; a negative or NaN
// distance raises the error flag (and still orders totally).
template <bool D64>
__device__ __forceinline__ Key make_key(const void* __restrict__ d, int32_t e, int32_t* err) {
    static_assert(D64, "FP32 keys are packed per slot by k_slot_keys");
    Key k;
    const double x = __ldg((const double*)d + e);
    if (!(x >= 0.0)) atomicExch(err, 1);
    k.hi = x == 0.0 ? 0ull : (uint64_t)__double_as_longlong(x);
    k.lo = (uint32_t)e;
    return k;
}

struct AggState {
    int32_t* cl;       // n: cluster (smallest member) of each fine node
    int32_t* nxt;      // n: next member in the cluster list, -1 ends
    int32_t* tail;     // n: last member (valid for cluster heads)
    void* ws;          // n: current suitor of each cluster head (key or edge id)
    int32_t* wl;       // cluster heads of the current pass (second pass on)
    int32_t* pc;       // matched pairs: smaller head
    int32_t* pb;       //                larger head
    uint64_t* phi;     //                key
    uint32_t* plo;
    int32_t* keep;     // per pair
    int32_t* flags;    // n: label scan input
    int32_t* lab;      // n
    uint64_t* keys;    // 2m per-slot keys (FP32 distances), else unused
    int32_t* ctr;      // [0] heads, [1] pairs, [2..3] proposals (u64), [4..7] error flags,
                       // [8..11] the same counts of a first pass merged without readback
};

__global__ void k_agg_init(int64_t n, int32_t* __restrict__ cl, int32_t* __restrict__ nxt,
                           int32_t* __restrict__ tail) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cl[i] = (int32_t)i;
    nxt[i] = -1;
    tail[i] = (int32_t)i;
}

// Per-slot keys for FP32 distances: (float bits << 32 | edge id) of the slot's
// edge, so the scans read one coalesced 8-byte key per slot.
__global__ void k_slot_keys(int64_t slots, const int32_t* __restrict__ eid, const float* __restrict__ d,
                            uint64_t* __restrict__ keys, int32_t* __restrict__ err) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= slots) return;
    const int32_t e = eid[j];
    const float x = __ldg(d + e);
    if (!(x >= 0.f)) atomicExch(err, 1);
    const uint64_t b = x == 0.f ? 0ull : (uint64_t)(uint32_t)__float_as_int(x);
    keys[j] = (b << 32) | (uint64_t)(uint32_t)e;
}

__device__ __forceinline__ Key key_inf() {
    Key k;
    k.hi = ~0ull;
    k.lo = ~0u;
    return k;
}
__device__ __forceinline__ bool key_is_inf(const Key& k) { return k.hi == ~0ull; }

// ---------------------------------------------------------------------------
// Suitor matching (Manne & Halappanavar 2014).  Every cluster b holds the
// best key proposed to it so far, ws[b].  A cluster a proposes to the
// neighbouring cluster b with the smallest key(a, b) among those with
// key(a, b) < ws[b]; a successful proposal displaces b's previous suitor,
// which then proposes again (the same lane group carries on with it); a
// proposal that lost a race is retried after a fresh scan.  ws only
// decreases, so every scan that sees a stale ws[b] overestimates b's
// eligibility and at worst costs one failed proposal.  At termination the
// suitor relation is symmetric and equals the greedy matching in key order
// (the locally-dominant matching of a strict total order).
//
// ws holds, per cluster: FP32 distances -> the packed 64-bit key itself
// (atomicMin is the proposal); FP64 distances -> the edge id (-1 none) of the
// key, replaced by compare-and-swap after comparing (d, id).
// ---------------------------------------------------------------------------
__device__ __forceinline__ Key key_of_edge64(const double* __restrict__ d, int32_t e) {
    Key k;
    const double x = __ldg(d + e);
    k.hi = x == 0.0 ? 0ull : (uint64_t)__double_as_longlong(x);
    k.lo = (uint32_t)e;
    return k;
}

// Key handling per distance precision.  FP32: the packed 64-bit key itself,
// compared as an integer, and ws holds it (the proposal is an atomicMin).
// FP64: (double bits, edge id), and ws holds the edge id (compare-and-swap
// after comparing keys).
template <bool D64>
struct SK;

template <>
struct SK<false> {
    using K = unsigned long long;
    static __device__ __forceinline__ K inf() { return ~0ull; }
    static __device__ __forceinline__ bool less(K a, K b) { return a < b; }
    static __device__ __forceinline__ bool is_inf(K a) { return a == ~0ull; }
    static __device__ __forceinline__ int32_t edge(K a) { return (int32_t)(uint32_t)a; }
    static __device__ __forceinline__ uint64_t hi(K a) { return a; }
    static __device__ __forceinline__ uint32_t lo(K) { return 0u; }
    static __device__ __forceinline__ K slot(int64_t j, const int32_t* __restrict__, const uint64_t* __restrict__ keys,
                                             const void* __restrict__, int32_t*) {
        return keys[j];
    }
    // current suitor key of cluster b, read from L2 (other blocks update it)
    static __device__ __forceinline__ K load(const void* ws, const void* __restrict__, int32_t b) {
        return __ldcg((const unsigned long long*)ws + b);
    }
    // true if k is now b's key; old = the key it displaced (inf if none) or,
    // on failure, the smaller key that holds b
    static __device__ __forceinline__ bool propose(void* ws, const void* __restrict__, int32_t b, K k, K& old) {
        old = atomicMin((unsigned long long*)ws + b, k);
        return old > k;
    }
    static __device__ __forceinline__ K shfl_xor(unsigned mask, K a, int o, int w) {
        return __shfl_xor_sync(mask, a, o, w);
    }
};

template <>
struct SK<true> {
    using K = Key;
    static __device__ __forceinline__ K inf() { return key_inf(); }
    static __device__ __forceinline__ bool less(const K& a, const K& b) { return key_less(a, b); }
    static __device__ __forceinline__ bool is_inf(const K& a) { return key_is_inf(a); }
    static __device__ __forceinline__ int32_t edge(const K& a) { return (int32_t)a.lo; }
    static __device__ __forceinline__ uint64_t hi(const K& a) { return a.hi; }
    static __device__ __forceinline__ uint32_t lo(const K& a) { return a.lo; }
    static __device__ __forceinline__ K slot(int64_t j, const int32_t* __restrict__ eid, const uint64_t* __restrict__,
                                             const void* __restrict__ d, int32_t* err) {
        return make_key<true>(d, eid[j], err);
    }
    static __device__ __forceinline__ K load(const void* ws, const void* __restrict__ d, int32_t b) {
        const int32_t e = __ldcg((const int32_t*)ws + b);
        return e < 0 ? key_inf() : key_of_edge64((const double*)d, e);
    }
    static __device__ __forceinline__ bool propose(void* ws, const void* __restrict__ d, int32_t b, const K& k,
                                                   K& old) {
        int32_t* w = (int32_t*)ws + b;
        int32_t cur = __ldcg(w);
        // every failed swap sees a strictly smaller key, so this ends within deg(b) + 1 tries
        while (true) {
            old = cur < 0 ? key_inf() : key_of_edge64((const double*)d, cur);
            if (!key_less(k, old)) return false;
            const int32_t prev = atomicCAS(w, cur, (int32_t)k.lo);
            if (prev == cur) return true;
            cur = prev;
        }
    }
    static __device__ __forceinline__ K shfl_xor(unsigned mask, const K& a, int o, int w) {
        K r;
        r.hi = __shfl_xor_sync(mask, a.hi, o, w);
        r.lo = __shfl_xor_sync(mask, a.lo, o, w);
        return r;
    }
};

// the cluster at the other end of edge e, seen from cluster b
template <bool FIRST_PASS>
__device__ __forceinline__ int32_t other_end(int32_t e, int32_t b, const int32_t* __restrict__ eu,
                                             const int32_t* __restrict__ ev, const int32_t* __restrict__ cl) {
    int32_t p = __ldg(eu + e), q = __ldg(ev + e);
    if (!FIRST_PASS) {
        p = __ldg(cl + p);
        q = __ldg(cl + q);
    }
    return p == b ? q : p;
}

// Best eligible neighbour over the slots [jb, je) of one member, one thread:
// eight slots at a time, their suitor keys fetched together (fewer
// dependent round trips than fetching only for improving slots).
template <bool D64, bool FIRST_PASS>
__device__ __forceinline__ void scan_slots_thread(int64_t jb, int64_t je, int32_t cur, const int32_t* __restrict__ col,
                                                  const int32_t* __restrict__ eid, const uint64_t* __restrict__ keys,
                                                  const void* __restrict__ d, const int32_t* __restrict__ cl,
                                                  const void* ws, int32_t* err, typename SK<D64>::K& bk,
                                                  int32_t& bb) {
    using T = SK<D64>;
    constexpr int U = 4;
    for (int64_t j0 = jb; j0 < je; j0 += U) {
        int32_t b[U];
        typename T::K k[U], w[U];
#pragma unroll
        for (int t = 0; t < U; ++t) {
            b[t] = -1;
            if (j0 + t < je) {
                const int32_t q = col[j0 + t];
                b[t] = FIRST_PASS ? q : __ldg(cl + q);
                if (!FIRST_PASS && b[t] == cur) b[t] = -1;
            }
        }
#pragma unroll
        for (int t = 0; t < U; ++t) {
            if (b[t] >= 0) {
                k[t] = T::slot(j0 + t, eid, keys, d, err);
                w[t] = T::load(ws, d, b[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < U; ++t)
            if (b[t] >= 0 && T::less(k[t], bk) && T::less(k[t], w[t])) {
                bk = k[t];
                bb = b[t];
            }
    }
}

// LPC lanes per cluster (1: a thread per cluster).  The first pass runs over
// all nodes (every node its own cluster, no cluster-id gather); later passes
// over the list of heads.
template <bool D64, int LPC, bool FIRST_PASS>
__global__ void __launch_bounds__(256) k_suitor(
    const int32_t* __restrict__ wl, const int32_t* __restrict__ wl_count, int64_t n,
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ eid,
    const uint64_t* __restrict__ keys, const void* __restrict__ d, const int32_t* __restrict__ cl,
    const int32_t* __restrict__ nxt, const int32_t* __restrict__ eu, const int32_t* __restrict__ ev, void* ws,
    int64_t chain_cap, unsigned long long* __restrict__ proposals, int32_t* __restrict__ err_key,
    int32_t* __restrict__ err_chain) {
    using T = SK<D64>;
    using K = typename T::K;
    const int l = threadIdx.x % LPC;
    const unsigned gmask = LPC == 32 ? 0xffffffffu : (((1u << LPC) - 1u) << ((threadIdx.x & 31) / LPC * LPC));
    const int64_t count = FIRST_PASS ? n : (int64_t)*wl_count;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / LPC;
    unsigned long long mine = 0;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPC; g < count; g += groups) {
        int32_t cur = FIRST_PASS ? (int32_t)g : wl[g];
        int64_t steps = 0;
        while (cur >= 0) {
            K bk = T::inf();
            int32_t bb = -1;
            for (int32_t p = cur; p >= 0; p = FIRST_PASS ? -1 : nxt[p]) {
                const int64_t e_end = rowptr[p + 1];
                if constexpr (LPC == 1) {
                    scan_slots_thread<D64, FIRST_PASS>(rowptr[p], e_end, cur, col, eid, keys, d, cl, ws, err_key, bk,
                                                       bb);
                } else {
                    for (int64_t j = rowptr[p] + l; j < e_end; j += LPC) {
                        const int32_t b = FIRST_PASS ? col[j] : __ldg(cl + col[j]);
                        if (!FIRST_PASS && b == cur) continue;
                        const K k = T::slot(j, eid, keys, d, err_key);
                        if (!T::less(k, bk)) continue;
                        if (T::less(k, T::load(ws, d, b))) {
                            bk = k;
                            bb = b;
                        }
                    }
                }
            }
            if constexpr (LPC > 1) {
                // group minimum; keys of different slots differ, so all lanes agree
#pragma unroll
                for (int o = LPC / 2; o > 0; o >>= 1) {
                    const K ok = T::shfl_xor(gmask, bk, o, LPC);
                    const int32_t ob = __shfl_xor_sync(gmask, bb, o, LPC);
                    if (T::less(ok, bk)) {
                        bk = ok;
                        bb = ob;
                    }
                }
            }
            if (bb < 0) break;  // no eligible neighbour: cur stays unmatched
            if (++steps > chain_cap) {
                if (l == 0) atomicExch(err_chain, 1);
                break;
            }
            int32_t next = -1;
            if (l == 0) {
                K old;
                if (T::propose(ws, d, bb, bk, old))
                    next = T::is_inf(old) ? -1 : other_end<FIRST_PASS>(T::edge(old), bb, eu, ev, cl);
                else
                    next = cur;  // lost a race: rescan
            }
            if constexpr (LPC > 1) cur = __shfl_sync(gmask, next, 0, LPC);
            else cur = next;
        }
        if (l == 0) mine += (unsigned long long)steps;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(proposals, mine);
}

// start of a pass: clear the suitor keys; from the second pass on, list the
// heads (one atomic per block on the list length: about half the nodes are
// heads, and one per warp serialised on the counter)
constexpr int INIT_THREADS = 256;

template <bool D64>
__global__ void __launch_bounds__(INIT_THREADS) k_suitor_init(int64_t n, const int32_t* __restrict__ cl, void* ws,
                                                              int32_t* __restrict__ wl, int32_t* __restrict__ count,
                                                              int list_heads) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < n;
    if (in) {
        if constexpr (D64) ((int32_t*)ws)[i] = -1;
        else ((unsigned long long*)ws)[i] = ~0ull;
    }
    if (!list_heads) return;  // uniform over the grid
    const bool head = in && cl[i] == (int32_t)i;
    const int32_t k = block_slot<INIT_THREADS>(head, count);
    if (k >= 0) wl[k] = (int32_t)i;
}

// Matched pairs: b and its suitor a hold each other's key.  Any one-sided
// suitor left at termination is an internal error (flag).  Every block runs
// the same number of rounds, so the pair list grows by one atomic per block
// and round.
constexpr int PAIR_THREADS = 256;

template <bool D64, bool FIRST_PASS>
__global__ void __launch_bounds__(PAIR_THREADS) k_suitor_pairs(const int32_t* __restrict__ wl, const int32_t* __restrict__ wl_count, int64_t n,
                               const void* ws, const void* __restrict__ d, const int32_t* __restrict__ eu,
                               const int32_t* __restrict__ ev, const int32_t* __restrict__ cl,
                               int32_t* __restrict__ pc, int32_t* __restrict__ pb, uint64_t* __restrict__ phi,
                               uint32_t* __restrict__ plo, int32_t* __restrict__ npairs,
                               int32_t* __restrict__ err_mutual) {
    using T = SK<D64>;
    const int64_t count = FIRST_PASS ? n : (int64_t)*wl_count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x; r < count; r += stride) {
        const int64_t i = r + threadIdx.x;
        int32_t b = -1, a = -1;
        typename T::K k{};
        bool emit = false;
        if (i < count) {
            b = FIRST_PASS ? (int32_t)i : wl[i];
            k = T::load(ws, d, b);
            if (!T::is_inf(k)) {
                a = other_end<FIRST_PASS>(T::edge(k), b, eu, ev, cl);
                const typename T::K ka = T::load(ws, d, a);
                if (T::less(ka, k) || T::less(k, ka)) atomicExch(err_mutual, 1);
                emit = b < a;
            }
        }
        const int32_t s = block_slot<PAIR_THREADS>(emit, npairs);
        if (s >= 0) {
            pc[s] = b;
            pb[s] = a;
            phi[s] = T::hi(k);
            plo[s] = T::lo(k);
        }
    }
}

__global__ void k_pairs_keys(int32_t npairs, const uint64_t* __restrict__ phi,
                             const uint32_t* __restrict__ plo, uint64_t* __restrict__ khi,
                             uint32_t* __restrict__ klo, uint32_t* __restrict__ idx) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    khi[i] = phi[i];
    klo[i] = plo[i];
    idx[i] = (uint32_t)i;
}

// Truncation without a sort: keep[i] = 1 for the `allowed` smallest of the
// npairs unique keys (hi, lo), ordered lexicographically, 0 for the others.
// One block finds the key of rank allowed - 1 by radix selection, 8-bit
// digits from the top (8 passes over hi, then 4 over lo when lo is part of
// the key), then marks every key at or below it.
constexpr int SELECT_THREADS = 1024;
constexpr int32_t SELECT_MAX = 65536;  // larger sets take the radix sort

template <bool D64>
__global__ void __launch_bounds__(SELECT_THREADS) k_select_smallest(int32_t npairs, int32_t allowed,
                                                                     const uint64_t* __restrict__ phi,
                                                                     const uint32_t* __restrict__ plo,
                                                                     int32_t* __restrict__ keep) {
    __shared__ uint32_t hist[256];
    __shared__ uint64_t pre_hi;
    __shared__ uint32_t pre_lo;
    __shared__ int32_t rank;
    constexpr int NPASS = D64 ? 12 : 8;
    if (threadIdx.x == 0) {
        pre_hi = 0ull;
        pre_lo = 0u;
        rank = allowed - 1;
    }
    for (int pass = 0; pass < NPASS; ++pass) {
        for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0u;
        __syncthreads();
        const bool in_hi = pass < 8;
        const int sh = in_hi ? 56 - 8 * pass : 24 - 8 * (pass - 8);
        const uint64_t mhi = in_hi ? (pass == 0 ? 0ull : ~0ull << (64 - 8 * pass)) : ~0ull;
        const uint32_t mlo = in_hi || pass == 8 ? 0u : ~0u << (32 - 8 * (pass - 8));
        const uint64_t ph = pre_hi;
        const uint32_t pl = pre_lo;
        for (int32_t i = threadIdx.x; i < npairs; i += blockDim.x) {
            const uint64_t h = phi[i];
            const uint32_t l = D64 ? plo[i] : 0u;
            if ((h & mhi) == (ph & mhi) && (l & mlo) == (pl & mlo)) {
                const uint32_t dig = in_hi ? (uint32_t)(h >> sh) & 255u : (l >> sh) & 255u;
                atomicAdd(&hist[dig], 1u);
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            uint32_t c[8], sum = 0u;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                c[j] = hist[lane * 8 + j];
                sum += c[j];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += x;
            }
            const uint32_t excl = incl - sum, r = (uint32_t)rank;
            if (excl <= r && r < incl) {  // exactly one lane: rank < number of matching keys
                uint32_t below = excl;
                int b = lane * 8;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (r < below + c[j]) {
                        b = lane * 8 + j;
                        break;
                    }
                    below += c[j];
                }
                if (in_hi) pre_hi = ph | ((uint64_t)b << sh);
                else pre_lo = pl | ((uint32_t)b << sh);
                rank = (int32_t)(r - below);
            }
        }
        __syncthreads();
    }
    const uint64_t kh = pre_hi;
    const uint32_t kl = pre_lo;
    for (int32_t i = threadIdx.x; i < npairs; i += blockDim.x) {
        const uint64_t h = phi[i];
        const bool le = D64 ? (h < kh || (h == kh && plo[i] <= kl)) : h <= kh;
        keep[i] = le ? 1 : 0;
    }
}

__global__ void k_keep_first(int32_t npairs, int64_t allowed, const uint32_t* __restrict__ sorted_idx,
                             int32_t* __restrict__ keep) {
    int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npairs) return;
    keep[sorted_idx[t]] = t < allowed ? 1 : 0;
}

__global__ void k_fill_i32(int32_t* __restrict__ a, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// merge the larger head's list into the smaller head's list
__global__ void k_merge(int32_t npairs, const int32_t* __restrict__ pc, const int32_t* __restrict__ pb,
                        const int32_t* __restrict__ keep, int32_t* __restrict__ cl,
                        int32_t* __restrict__ nxt, int32_t* __restrict__ tail) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs || !keep[i]) return;
    const int32_t c = pc[i], b = pb[i];
    for (int32_t p = b; p >= 0; p = nxt[p]) cl[p] = c;
    nxt[tail[c]] = b;
    tail[c] = tail[b];
}

// every pair merges (the pass cannot exceed its merge budget); pair count on the device
__global__ void k_merge_all(const int32_t* __restrict__ npairs, const int32_t* __restrict__ pc,
                            const int32_t* __restrict__ pb, int32_t* __restrict__ cl, int32_t* __restrict__ nxt,
                            int32_t* __restrict__ tail) {
    const int32_t cnt = *npairs;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int32_t c = pc[i], b = pb[i];
        for (int32_t p = b; p >= 0; p = nxt[p]) cl[p] = c;
        nxt[tail[c]] = b;
        tail[c] = tail[b];
    }
}

__global__ void k_head_flags(int64_t n, const int32_t* __restrict__ cl, int32_t* __restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = cl[i] == (int32_t)i ? 1 : 0;
}

__global__ void k_labels(int64_t n, const int32_t* __restrict__ cl, const int32_t* __restrict__ lab,
                         const int32_t* __restrict__ flags, int32_t* __restrict__ agg,
                         int64_t* __restrict__ nc_out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) agg[i] = lab[cl[i]];
    if (i == n - 1) *nc_out = (int64_t)lab[i] + flags[i];
}

__global__ void k_gather_u64(const uint64_t* __restrict__ src, const uint32_t* __restrict__ idx,
                             int32_t count, uint64_t* __restrict__ out) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = src[idx[i]];
}

template <bool D64, int LPC, bool FIRST_PASS>
static void launch_suitor(gr_ctx* c, AggState& S, int64_t count, const void* d, int64_t chain_cap) {
    const int64_t want = count > 0 ? ceil_div(count * LPC, 256) : 1;
    const int64_t cap = (int64_t)c->num_sms * 64;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    k_suitor<D64, LPC, FIRST_PASS><<<grid, 256, 0, c->stream>>>(
        S.wl, S.ctr + 0, c->n, c->rowptr, c->col, c->eid, S.keys, d, S.cl, S.nxt, c->eu, c->ev, S.ws, chain_cap,
        (unsigned long long*)(S.ctr + 2), S.ctr + 5, S.ctr + 6);
    count_launch();
    const int64_t pwant = count > 0 ? ceil_div(count, 256) : 1, pcap = (int64_t)c->num_sms * 16;
    k_suitor_pairs<D64, FIRST_PASS><<<(unsigned)(pwant < pcap ? pwant : pcap), PAIR_THREADS, 0, c->stream>>>(
        S.wl, S.ctr + 0, c->n, S.ws, d, c->eu, c->ev, S.cl, S.pc, S.pb, S.phi, S.plo, S.ctr + 1, S.ctr + 7);
    count_launch();
}

template <bool D64, int LPC>
static void launch_suitor_pass(gr_ctx* c, AggState& S, int64_t count, const void* d, int64_t chain_cap,
                               bool first_pass) {
    if (first_pass) launch_suitor<D64, LPC, true>(c, S, count, d, chain_cap);
    else launch_suitor<D64, LPC, false>(c, S, count, d, chain_cap);
}

template <bool D64>
static void launch_suitor_lpc(gr_ctx* c, AggState& S, int lpc, int64_t count, const void* d, int64_t chain_cap,
                              bool first_pass) {
    if (lpc == 32) launch_suitor_pass<D64, 32>(c, S, count, d, chain_cap, first_pass);
    else if (lpc == 8) launch_suitor_pass<D64, 8>(c, S, count, d, chain_cap, first_pass);
    else launch_suitor_pass<D64, 1>(c, S, count, d, chain_cap, first_pass);
}

gr_status aggregate_impl(gr_ctx* c, const void* d, int d_is_f64, int64_t target_nc, int passes,
                         int64_t max_proposals, int32_t* agg, int64_t* nc_out, int64_t* proposals_out) {
    const int64_t n = c->n;
    cudaStream_t s = c->stream;
    // scratch
    size_t need = 0;
    auto add = [&](size_t bytes) {
        size_t off = need;
        need += (bytes + 255) & ~size_t(255);
        return off;
    };
    const size_t o_cl = add(4 * n), o_nxt = add(4 * n), o_tail = add(4 * n), o_ws = add(8 * n),
                 o_wl = add(4 * n), o_pc = add(4 * n), o_pb = add(4 * n), o_phi = add(8 * n),
                 o_plo = add(4 * n), o_keep = add(4 * n), o_flags = add(4 * n), o_lab = add(4 * n),
                 o_keys = add(d_is_f64 ? 8 : 8 * 2 * c->m), o_ctr = add(64);
    void* base;
    GR_TRY_CUDA(c, c->ws.get(WS_AGG_STATE, need, &base), "aggregate scratch");
    char* B = (char*)base;
    AggState S;
    S.cl = (int32_t*)(B + o_cl);
    S.nxt = (int32_t*)(B + o_nxt);
    S.tail = (int32_t*)(B + o_tail);
    S.ws = (void*)(B + o_ws);
    S.wl = (int32_t*)(B + o_wl);
    S.pc = (int32_t*)(B + o_pc);
    S.pb = (int32_t*)(B + o_pb);
    S.phi = (uint64_t*)(B + o_phi);
    S.plo = (uint32_t*)(B + o_plo);
    S.keep = (int32_t*)(B + o_keep);
    S.flags = (int32_t*)(B + o_flags);
    S.lab = (int32_t*)(B + o_lab);
    S.keys = (uint64_t*)(B + o_keys);
    S.ctr = (int32_t*)(B + o_ctr);
    int64_t* hs = host_scratch();
    if (!hs) return set_error(c, GR_ENOMEM, "aggregate: pinned scratch unavailable");
    int32_t* hctr = (int32_t*)hs;  // pinned: the 8 counters and flags

    const unsigned gn = (unsigned)ceil_div(n > 0 ? n : 1, 256);
    k_agg_init<<<gn, 256, 0, s>>>(n, S.cl, S.nxt, S.tail); count_launch();
    GR_TRY_CUDA(c, cudaMemsetAsync(S.ctr, 0, 64, s), "memset");
    if (!d_is_f64 && c->m > 0) {
        k_slot_keys<<<(unsigned)ceil_div(2 * c->m, 256), 256, 0, s>>>(2 * c->m, c->eid, (const float*)d, S.keys,
                                                                       S.ctr + 4);
        count_launch();
    }
    const double avg = n > 0 ? 2.0 * (double)c->m / (double)n : 0.0;
    const int lpc = avg >= 24 ? 32 : (avg >= 12 ? 8 : 1);
    // a proposal chain can never be longer than the number of suitor-key
    // decreases (at most 2m) plus the failed races; far beyond that is a fault
    const int64_t chain_cap = 4 * c->m + 2 * n + 64;

    int64_t n_cur = n;
    int64_t total_proposals = 0;
    // When 2 target <= n the first pass cannot exceed its merge budget (a
    // matching has at most n/2 pairs), so it merges on the device without a
    // readback; its counts are checked at the next pass's readback.
    bool deferred = false;
    for (int pass = 0; pass < passes; ++pass) {
        if (!deferred && n_cur <= target_nc) break;
        const bool first = pass == 0;
        GR_TRY_CUDA(c, cudaMemsetAsync(S.ctr, 0, 16, s), "memset");
        const unsigned gi = (unsigned)ceil_div(n > 0 ? n : 1, INIT_THREADS);
        if (d_is_f64) k_suitor_init<true><<<gi, INIT_THREADS, 0, s>>>(n, S.cl, S.ws, S.wl, S.ctr + 0, first ? 0 : 1);
        else k_suitor_init<false><<<gi, INIT_THREADS, 0, s>>>(n, S.cl, S.ws, S.wl, S.ctr + 0, first ? 0 : 1);
        count_launch();
        if (d_is_f64) launch_suitor_lpc<true>(c, S, lpc, n_cur, d, chain_cap, first);
        else launch_suitor_lpc<false>(c, S, lpc, n_cur, d, chain_cap, first);
        GR_TRY_CUDA(c, cudaGetLastError(), "aggregate matching");
        if (first && passes > 1 && 2 * target_nc <= n_cur) {
            k_merge_all<<<(unsigned)ceil_div(n / 2 > 0 ? n / 2 : 1, 256), 256, 0, s>>>(S.ctr + 1, S.pc, S.pb, S.cl,
                                                                                     S.nxt, S.tail);
            count_launch();
            // keep this pass's heads, pairs and proposals for the next readback
            GR_TRY_CUDA(c, cudaMemcpyAsync(S.ctr + 8, S.ctr, 16, cudaMemcpyDeviceToDevice, s), "copy");
            deferred = true;
            continue;
        }
        GR_TRY_CUDA(c, cudaMemcpyAsync(hctr, S.ctr, 48, cudaMemcpyDeviceToHost, s), "readback");
        GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
        if (hctr[4] || hctr[5]) return set_error(c, GR_EINVAL, "aggregate: distances must be >= 0 and not NaN");
        if (hctr[6]) return set_error(c, GR_ECUDA, "aggregate: a proposal chain exceeded its bound");
        if (hctr[7]) return set_error(c, GR_ECUDA, "aggregate: one-sided suitor at termination");
        if (deferred) {  // the first pass, merged on the device
            const int64_t p0 = (int64_t)(((const unsigned long long*)hctr)[5]);
            total_proposals += p0;
            if (max_proposals > 0 && p0 > max_proposals)
                return set_error(c, GR_ETIMEOUT, "aggregate: proposal budget exceeded");
            n_cur -= hctr[9];
            deferred = false;
        }
        const int64_t pass_proposals = (int64_t)(((const unsigned long long*)hctr)[1]);
        total_proposals += pass_proposals;
        if (proposals_out) *proposals_out = total_proposals;
        if (!first && hctr[0] != n_cur) return set_error(c, GR_ECUDA, "aggregate: internal cluster count mismatch");
        if (max_proposals > 0 && pass_proposals > max_proposals)
            return set_error(c, GR_ETIMEOUT, "aggregate: proposal budget exceeded");
        const int64_t allowed = n_cur - target_nc;
        const int32_t npairs = hctr[1];
        if (npairs == 0 || allowed <= 0) break;
        const unsigned gp = (unsigned)ceil_div(npairs, 256);
        if ((int64_t)npairs > allowed && npairs <= SELECT_MAX) {
            // keep the `allowed` smallest keys: one block selects them
            if (d_is_f64) {
                k_select_smallest<true><<<1, SELECT_THREADS, 0, s>>>(npairs, (int32_t)allowed, S.phi, S.plo, S.keep);
            } else {
                k_select_smallest<false><<<1, SELECT_THREADS, 0, s>>>(npairs, (int32_t)allowed, S.phi, S.plo, S.keep);
            }
            count_launch();
            n_cur -= allowed;
        } else if ((int64_t)npairs > allowed) {
            // keep the `allowed` smallest keys: stable sort by lo, then by hi
            void* pk;
            GR_TRY_CUDA(c, c->ws.get(WS_AGG_KEYS, (size_t)npairs * 32 + 1024, &pk), "scratch");
            uint64_t* khi = (uint64_t*)pk;
            uint64_t* khi2 = khi + npairs;
            uint32_t* idx = (uint32_t*)(khi2 + npairs);
            uint32_t* idx2 = idx + npairs;
            uint32_t* klo = (uint32_t*)S.flags;  // n >= npairs entries of scratch
            uint32_t* klo2 = (uint32_t*)S.lab;
            k_pairs_keys<<<gp, 256, 0, s>>>(npairs, S.phi, S.plo, khi, klo, idx); count_launch();
            int alt = 0;
            uint32_t* ci = idx;
            if (d_is_f64) {
                GR_TRY_CUDA(c, radix_sort_u32(klo, idx, klo2, idx2, npairs, 32, c->ws, s, &alt), "sort");
                ci = alt ? idx2 : idx;
                uint32_t* ci_alt = alt ? idx : idx2;
                // hi keys in the order of the first sort
                k_gather_u64<<<gp, 256, 0, s>>>(S.phi, ci, npairs, khi); count_launch();
                GR_TRY_CUDA(c, radix_sort_u64(khi, ci, khi2, ci_alt, npairs, 64, c->ws, s, &alt), "sort");
                ci = alt ? ci_alt : ci;
            } else {
                GR_TRY_CUDA(c, radix_sort_u64(khi, idx, khi2, idx2, npairs, 64, c->ws, s, &alt), "sort");
                ci = alt ? idx2 : idx;
            }
            k_keep_first<<<gp, 256, 0, s>>>(npairs, allowed, ci, S.keep); count_launch();
            n_cur -= allowed;
        } else {
            k_fill_i32<<<gp, 256, 0, s>>>(S.keep, npairs, 1); count_launch();
            n_cur -= npairs;
        }
        k_merge<<<gp, 256, 0, s>>>(npairs, S.pc, S.pb, S.keep, S.cl, S.nxt, S.tail); count_launch();
        GR_TRY_CUDA(c, cudaGetLastError(), "aggregate merge");
    }
    if (deferred) return set_error(c, GR_ECUDA, "aggregate: internal pass bookkeeping");
    // labels: rank of each cluster head (= its smallest member)
    k_head_flags<<<gn, 256, 0, s>>>(n, S.cl, S.flags); count_launch();
    GR_TRY_CUDA(c, scan_exclusive_i32(S.flags, S.lab, n, c->ws, s), "scan labels");
    k_labels<<<gn, 256, 0, s>>>(n, S.cl, S.lab, S.flags, agg, hs + 2); count_launch();
    GR_TRY_CUDA(c, cudaGetLastError(), "labels");
    GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
    *nc_out = hs[2];
    if (*nc_out != n_cur) return set_error(c, GR_ECUDA, "aggregate: internal count mismatch");
    if (proposals_out) *proposals_out = total_proposals;
    return GR_OK;
}

}  // namespace gr
