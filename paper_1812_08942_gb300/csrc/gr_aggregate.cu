// Node aggregation by algebraic distance (Sec. 3.2.2).
//
// Edges are ordered by the key (d, edge id), a strict total order.  A pass
// computes the greedy matching of the current cluster graph in that order by
// rounds of a lock-free handshake: every free cluster points at the free
// neighbouring cluster across its smallest key; mutual pointers merge.  With
// a strict total order this is the unique locally-dominant matching, equal to
// the sequential greedy one (Preis 1999; Manne & Bisseling 2007).  A pass that
// would exceed the allowed merge count keeps its smallest keys, which equals
// stopping the greedy scan early.  Clusters are identified by their smallest
// fine node; a cluster's members form a linked list starting there.
#include "gr_internal.cuh"

namespace gr {

enum : uint8_t { ST_FREE = 0, ST_MATCHED = 1, ST_DEAD = 2 };

struct Key {
    uint64_t hi;
    uint32_t lo;
};
__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// FP32 distance: (float bits << 32 | id) in hi.  FP64: double bits in hi, id in lo.
template <bool D64>
__device__ __forceinline__ Key make_key(const void* __restrict__ d, int32_t e, int32_t* err) {
    Key k;
    if constexpr (D64) {
        double x = __ldg((const double*)d + e);
        if (!(x >= 0.0)) atomicExch(err, 1);
        k.hi = x == 0.0 ? 0ull : (uint64_t)__double_as_longlong(x);
        k.lo = (uint32_t)e;
    } else {
        float x = __ldg((const float*)d + e);
        if (!(x >= 0.f)) atomicExch(err, 1);
        uint64_t b = x == 0.f ? 0ull : (uint64_t)(uint32_t)__float_as_int(x);
        k.hi = (b << 32) | (uint64_t)(uint32_t)e;
        k.lo = 0u;
    }
    return k;
}

struct AggState {
    int32_t* cl;       // n: cluster (smallest member) of each fine node
    int32_t* nxt;      // n: next member in the cluster list, -1 ends
    int32_t* tail;     // n: last member (valid for cluster heads)
    uint8_t* status;   // n: per cluster head
    int32_t* best;     // n: best neighbouring cluster, -1 none
    uint64_t* bhi;     // n
    uint32_t* blo;     // n
    int32_t* wl[2];    // worklists of free clusters
    int32_t* pc;       // matched pairs: smaller head
    int32_t* pb;       //                larger head
    uint64_t* phi;     //                key
    uint32_t* plo;
    int32_t* keep;     // per pair
    int32_t* flags;    // n: label scan input
    int32_t* lab;      // n
    uint64_t* tk_hi;   // n * TOPK cached candidate keys
    uint32_t* tk_lo;   // n * TOPK
    int32_t* tk_nb;    // n * TOPK cached candidate clusters
    uint8_t* tk_cnt;   // n: number of cached candidates
    uint64_t* keys;    // 2m per-slot keys (FP32 distances), else unused
    int32_t* ctr;      // [0],[1] worklist counts, [2] pair count, [3] [4] error flags
};

__global__ void k_agg_init(int64_t n, int32_t* __restrict__ cl, int32_t* __restrict__ nxt,
                           int32_t* __restrict__ tail) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cl[i] = (int32_t)i;
    nxt[i] = -1;
    tail[i] = (int32_t)i;
}

// Append `item` to a worklist when `keep`: one atomic per warp, entries of a
// warp stay contiguous and in lane order (keeps neighbouring rows together).
__device__ __forceinline__ void warp_append(bool keep, int32_t item, int32_t* __restrict__ list,
                                            int32_t* __restrict__ count) {
    const unsigned active = __activemask();
    const unsigned ball = __ballot_sync(active, keep);
    if (!ball) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ball) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(ball));
    base = __shfl_sync(active, base, leader);
    if (keep) list[base + __popc(ball & ((1u << lane) - 1u))] = item;
}

// start of a pass: every cluster head becomes free and joins the worklist
__global__ void k_pass_init(int64_t n, const int32_t* __restrict__ cl, uint8_t* __restrict__ status,
                            int32_t* __restrict__ best, int32_t* __restrict__ wl,
                            int32_t* __restrict__ ctr) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    best[i] = -1;
    status[i] = ST_FREE;
    warp_append(cl[i] == (int32_t)i, (int32_t)i, wl, &ctr[0]);
}

// Per-slot keys for FP32 distances: (float bits << 32 | edge id) of the slot's
// edge, so every round reads one coalesced 8-byte key per slot.
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

constexpr int TOPK = 1;  // cached candidates per cluster (1 measured best: deeper caches cost more than the rescans they save)

__device__ __forceinline__ Key key_inf() {
    Key k;
    k.hi = ~0ull;
    k.lo = ~0u;
    return k;
}

// Each free cluster finds its smallest key towards another free cluster.
// LPC lanes per cluster walk the members' CSR rows and keep the TOPK smallest
// candidates (neighbours only ever leave the free set, so the first cached
// candidate that is still free is the current best; a cluster rescans only
// when all TOPK cached candidates are gone).  In the first pass every node is
// its own cluster, so the cluster-id gather is skipped; in the first round of
// a pass every cluster is free, so the status gather is skipped too.
template <bool D64, int LPC, bool FIRST_PASS>
__device__ __forceinline__ void propose_one(
    const int32_t c, const int l, const unsigned gmask, const int gbase_lane, const int64_t* __restrict__ rowptr,
    const int32_t* __restrict__ col, const int32_t* __restrict__ eid, const uint64_t* __restrict__ keys,
    const void* __restrict__ d, const int32_t* __restrict__ cl, const int32_t* __restrict__ nxt,
    uint8_t* __restrict__ status, int32_t* __restrict__ best, uint64_t* __restrict__ bhi, uint32_t* __restrict__ blo,
    uint64_t* __restrict__ tk_hi, uint32_t* __restrict__ tk_lo, int32_t* __restrict__ tk_nb,
    uint8_t* __restrict__ tk_cnt, const int first_round, int32_t* __restrict__ err) {
    // 1) cached candidates
    const int cnt = first_round ? 0 : tk_cnt[c];
    if (cnt > 0) {
        bool fr = false;
        if (l < cnt) fr = status[tk_nb[(int64_t)c * TOPK + l]] == ST_FREE;
        const unsigned ball = __ballot_sync(gmask, fr) >> gbase_lane;
        if (ball) {
            const int f = __ffs(ball) - 1;
            if (l == 0) {
                best[c] = tk_nb[(int64_t)c * TOPK + f];
                bhi[c] = tk_hi[(int64_t)c * TOPK + f];
                blo[c] = tk_lo[(int64_t)c * TOPK + f];
            }
            return;
        }
        if (cnt < TOPK) {  // every free neighbour the scan saw is gone
            if (l == 0) status[c] = ST_DEAD;
            return;
        }
    }
    // 2) scan: per-lane sorted lists of the TOPK smallest candidates
    Key lk[TOPK];
    int32_t ln[TOPK];
#pragma unroll
    for (int t = 0; t < TOPK; ++t) {
        lk[t] = key_inf();
        ln[t] = -1;
    }
    for (int32_t p = c; p >= 0; p = FIRST_PASS ? -1 : nxt[p]) {
        const int64_t e_end = rowptr[p + 1];
        for (int64_t j = rowptr[p] + l; j < e_end; j += LPC) {
            const int32_t cq = FIRST_PASS ? col[j] : cl[col[j]];
            if (!FIRST_PASS && cq == c) continue;
            if (!first_round && status[cq] != ST_FREE) continue;
            Key k;
            if constexpr (D64) {
                k = make_key<true>(d, eid[j], err);
            } else {
                k.hi = keys[j];
                k.lo = 0u;
            }
            if (key_less(k, lk[TOPK - 1])) {
                lk[TOPK - 1] = k;
                ln[TOPK - 1] = cq;
#pragma unroll
                for (int t = TOPK - 1; t > 0; --t)
                    if (key_less(lk[t], lk[t - 1])) {
                        Key tk = lk[t];
                        lk[t] = lk[t - 1];
                        lk[t - 1] = tk;
                        int32_t tn = ln[t];
                        ln[t] = ln[t - 1];
                        ln[t - 1] = tn;
                    }
            }
        }
    }
    // 3) merge the lanes' lists: TOPK rounds of group argmin over list heads
    int found = 0;
#pragma unroll
    for (int t = 0; t < TOPK; ++t) {
        Key bk = lk[0];
        int bl = l;
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) {
            Key ok;
            ok.hi = __shfl_xor_sync(gmask, bk.hi, o, LPC);
            ok.lo = __shfl_xor_sync(gmask, bk.lo, o, LPC);
            const int ol = __shfl_xor_sync(gmask, bl, o, LPC);
            if (key_less(ok, bk) || (ok.hi == bk.hi && ok.lo == bk.lo && ol < bl)) {
                bk = ok;
                bl = ol;
            }
        }
        const int32_t bnb = __shfl_sync(gmask, ln[0], bl, LPC);
        if (bk.hi == ~0ull && bk.lo == ~0u) break;  // uniform across the group
        if (l == 0) {
            tk_hi[(int64_t)c * TOPK + t] = bk.hi;
            tk_lo[(int64_t)c * TOPK + t] = bk.lo;
            tk_nb[(int64_t)c * TOPK + t] = bnb;
            if (t == 0) {
                best[c] = bnb;
                bhi[c] = bk.hi;
                blo[c] = bk.lo;
            }
        }
        if (l == bl) {  // pop the winner's head
#pragma unroll
            for (int u = 0; u < TOPK - 1; ++u) {
                lk[u] = lk[u + 1];
                ln[u] = ln[u + 1];
            }
            lk[TOPK - 1] = key_inf();
            ln[TOPK - 1] = -1;
        }
        ++found;
    }
    if (l == 0) {
        tk_cnt[c] = (uint8_t)found;
        if (found == 0) status[c] = ST_DEAD;  // no free neighbour now, none later in this pass
    }
}


template <bool D64, int LPC, bool FIRST_PASS>
__global__ void k_propose(const int32_t* __restrict__ wl, const int32_t* __restrict__ wl_count,
                          int32_t* __restrict__ next_count, const int64_t* __restrict__ rowptr,
                          const int32_t* __restrict__ col, const int32_t* __restrict__ eid,
                          const uint64_t* __restrict__ keys, const void* __restrict__ d,
                          const int32_t* __restrict__ cl, const int32_t* __restrict__ nxt,
                          uint8_t* __restrict__ status, int32_t* __restrict__ best, uint64_t* __restrict__ bhi,
                          uint32_t* __restrict__ blo, uint64_t* __restrict__ tk_hi, uint32_t* __restrict__ tk_lo,
                          int32_t* __restrict__ tk_nb, uint8_t* __restrict__ tk_cnt, int first_round,
                          int32_t* __restrict__ err) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *next_count = 0;
    const int l = threadIdx.x % LPC;
    const unsigned gmask = LPC == 32 ? 0xffffffffu : (((1u << LPC) - 1u) << ((threadIdx.x & 31) / LPC * LPC));
    const int gbase_lane = (threadIdx.x & 31) / LPC * LPC;
    const int count = *wl_count;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / LPC;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPC; g < count; g += groups)
        propose_one<D64, LPC, FIRST_PASS>(wl[g], l, gmask, gbase_lane, rowptr, col, eid, keys, d, cl, nxt, status,
                                          best, bhi, blo, tk_hi, tk_lo, tk_nb, tk_cnt, first_round, err);
}

// Mutual best pointers merge; the rest stays on the worklist.
__global__ void k_accept(const int32_t* __restrict__ wl, const int32_t* __restrict__ wl_count,
                         int32_t* __restrict__ wl_next, int32_t* __restrict__ next_count,
                         uint8_t* __restrict__ status, const int32_t* __restrict__ best,
                         const uint64_t* __restrict__ bhi, const uint32_t* __restrict__ blo,
                         int32_t* __restrict__ pc, int32_t* __restrict__ pb,
                         uint64_t* __restrict__ phi, uint32_t* __restrict__ plo,
                         int32_t* __restrict__ npairs) {
    const int count = *wl_count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const int32_t c = wl[i];
        if (status[c] != ST_FREE) continue;  // dead this round
        const int32_t b = best[c];
        const bool matched = best[b] == c;
        if (matched) {
            status[c] = ST_MATCHED;
            if (c < b) {
                int32_t k = atomicAdd(npairs, 1);
                pc[k] = c;
                pb[k] = b;
                phi[k] = bhi[c];
                plo[k] = blo[c];
            }
        }
        warp_append(!matched, c, wl_next, next_count);
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
static void launch_propose(gr_ctx* c, AggState& S, int r, int64_t bound, const void* d) {
    const int64_t threads = bound * LPC;
    int64_t want = threads > 0 ? ceil_div(threads, 256) : 1;
    const int64_t cap = (int64_t)c->num_sms * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    k_propose<D64, LPC, FIRST_PASS><<<grid, 256, 0, c->stream>>>(
        S.wl[r & 1], S.ctr + (r & 1), S.ctr + ((r + 1) & 1), c->rowptr, c->col, c->eid, S.keys, d, S.cl, S.nxt,
        S.status, S.best, S.bhi, S.blo, S.tk_hi, S.tk_lo, S.tk_nb, S.tk_cnt, r == 0 ? 1 : 0, S.ctr + 3);
    count_launch();
}

template <bool D64, int LPC>
static void launch_propose_pass(gr_ctx* c, AggState& S, int r, int64_t bound, const void* d, bool first_pass) {
    if (first_pass) launch_propose<D64, LPC, true>(c, S, r, bound, d);
    else launch_propose<D64, LPC, false>(c, S, r, bound, d);
}

gr_status aggregate_impl(gr_ctx* c, const void* d, int d_is_f64, int64_t target_nc, int passes,
                         int max_rounds, int32_t* agg, int64_t* nc_out, int32_t* rounds_out) {
    const int64_t n = c->n;
    cudaStream_t s = c->stream;
    if (max_rounds <= 0) max_rounds = (int)(n < (1 << 30) ? n + 64 : (1 << 30));
    // scratch
    size_t need = 0;
    auto add = [&](size_t bytes) {
        size_t off = need;
        need += (bytes + 255) & ~size_t(255);
        return off;
    };
    const size_t o_cl = add(4 * n), o_nxt = add(4 * n), o_tail = add(4 * n), o_st = add(n),
                 o_best = add(4 * n), o_bhi = add(8 * n), o_blo = add(4 * n), o_wl0 = add(4 * n),
                 o_wl1 = add(4 * n), o_pc = add(4 * n), o_pb = add(4 * n), o_phi = add(8 * n),
                 o_plo = add(4 * n), o_keep = add(4 * n), o_flags = add(4 * n), o_lab = add(4 * n),
                 o_tkhi = add(8 * TOPK * n), o_tklo = add(4 * TOPK * n), o_tknb = add(4 * TOPK * n),
                 o_tkcnt = add(n), o_keys = add(d_is_f64 ? 8 : 8 * 2 * c->m), o_ctr = add(64);
    void* base;
    GR_TRY_CUDA(c, c->ws.get(WS_AGG_STATE, need, &base), "aggregate scratch");
    char* B = (char*)base;
    AggState S;
    S.cl = (int32_t*)(B + o_cl);
    S.nxt = (int32_t*)(B + o_nxt);
    S.tail = (int32_t*)(B + o_tail);
    S.status = (uint8_t*)(B + o_st);
    S.best = (int32_t*)(B + o_best);
    S.bhi = (uint64_t*)(B + o_bhi);
    S.blo = (uint32_t*)(B + o_blo);
    S.wl[0] = (int32_t*)(B + o_wl0);
    S.wl[1] = (int32_t*)(B + o_wl1);
    S.pc = (int32_t*)(B + o_pc);
    S.pb = (int32_t*)(B + o_pb);
    S.phi = (uint64_t*)(B + o_phi);
    S.plo = (uint32_t*)(B + o_plo);
    S.keep = (int32_t*)(B + o_keep);
    S.flags = (int32_t*)(B + o_flags);
    S.lab = (int32_t*)(B + o_lab);
    S.tk_hi = (uint64_t*)(B + o_tkhi);
    S.tk_lo = (uint32_t*)(B + o_tklo);
    S.tk_nb = (int32_t*)(B + o_tknb);
    S.tk_cnt = (uint8_t*)(B + o_tkcnt);
    S.keys = (uint64_t*)(B + o_keys);
    S.ctr = (int32_t*)(B + o_ctr);
    int64_t* hs = host_scratch();
    if (!hs) return set_error(c, GR_ENOMEM, "aggregate: pinned scratch unavailable");
    int32_t* hctr = (int32_t*)hs;  // pinned: [0..3] counters

    const unsigned gn = (unsigned)ceil_div(n > 0 ? n : 1, 256);
    k_agg_init<<<gn, 256, 0, s>>>(n, S.cl, S.nxt, S.tail); count_launch();
    GR_TRY_CUDA(c, cudaMemsetAsync(S.ctr, 0, 64, s), "memset");
    if (!d_is_f64 && c->m > 0) {
        k_slot_keys<<<(unsigned)ceil_div(2 * c->m, 256), 256, 0, s>>>(2 * c->m, c->eid, (const float*)d, S.keys,
                                                                       S.ctr + 4);
        count_launch();
    }
    const double avg = n > 0 ? 2.0 * (double)c->m / (double)n : 0.0;
    const int lpc = avg >= 24 ? 32 : (avg >= 6 ? 8 : 4);

    int64_t n_cur = n;
    int total_rounds = 0;
    for (int pass = 0; pass < passes; ++pass) {
        if (n_cur <= target_nc) break;
        const int64_t allowed = n_cur - target_nc;
        GR_TRY_CUDA(c, cudaMemsetAsync(S.ctr, 0, 16, s), "memset");
        k_pass_init<<<gn, 256, 0, s>>>(n, S.cl, S.status, S.best, S.wl[0], S.ctr); count_launch();
        int64_t nlive = n_cur;
        int r = 0;
        while (nlive > 0) {
            const int batch = 6;  // rounds between readbacks; a round on an empty list is two tiny launches
            for (int bi = 0; bi < batch; ++bi, ++r) {
                const bool fp = pass == 0;
                if (d_is_f64) {
                    if (lpc == 32) launch_propose_pass<true, 32>(c, S, r, nlive, d, fp);
                    else if (lpc == 8) launch_propose_pass<true, 8>(c, S, r, nlive, d, fp);
                    else launch_propose_pass<true, 4>(c, S, r, nlive, d, fp);
                } else {
                    if (lpc == 32) launch_propose_pass<false, 32>(c, S, r, nlive, d, fp);
                    else if (lpc == 8) launch_propose_pass<false, 8>(c, S, r, nlive, d, fp);
                    else launch_propose_pass<false, 4>(c, S, r, nlive, d, fp);
                }
                const int64_t acap = (int64_t)c->num_sms * 8, awant = ceil_div(nlive, 256);
                k_accept<<<(unsigned)(awant < acap ? awant : acap), 256, 0, s>>>(
                    S.wl[r & 1], S.ctr + (r & 1), S.wl[(r + 1) & 1], S.ctr + ((r + 1) & 1), S.status,
                    S.best, S.bhi, S.blo, S.pc, S.pb, S.phi, S.plo, S.ctr + 2); count_launch();
            }
            GR_TRY_CUDA(c, cudaGetLastError(), "aggregate rounds");
            GR_TRY_CUDA(c, cudaMemcpyAsync(hctr, S.ctr, 32, cudaMemcpyDeviceToHost, s), "readback");
            GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
            if (hctr[3] || hctr[4]) return set_error(c, GR_EINVAL, "aggregate: distances must be >= 0 and not NaN");
            const int64_t prev = nlive;
            nlive = hctr[r & 1];
            // every round removes at least the pair across the smallest free-free key
            if (nlive > 0 && nlive >= prev)
                return set_error(c, GR_ECUDA, "aggregate: a handshake round made no progress");
            if (r > max_rounds && nlive > 0) {
                total_rounds += r;
                if (rounds_out) *rounds_out = total_rounds;
                return set_error(c, GR_ETIMEOUT, "aggregate: handshake round limit exceeded");
            }
        }
        total_rounds += r;
        const int32_t npairs = hctr[2];
        if (npairs == 0) break;
        const unsigned gp = (unsigned)ceil_div(npairs, 256);
        if ((int64_t)npairs > allowed) {
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
    // labels: rank of each cluster head (= its smallest member)
    k_head_flags<<<gn, 256, 0, s>>>(n, S.cl, S.flags); count_launch();
    GR_TRY_CUDA(c, scan_exclusive_i32(S.flags, S.lab, n, c->ws, s), "scan labels");
    k_labels<<<gn, 256, 0, s>>>(n, S.cl, S.lab, S.flags, agg, hs + 2); count_launch();
    GR_TRY_CUDA(c, cudaGetLastError(), "labels");
    GR_TRY_CUDA(c, cudaStreamSynchronize(s), "sync");
    *nc_out = hs[2];
    if (*nc_out != n_cur) return set_error(c, GR_ECUDA, "aggregate: internal count mismatch");
    if (rounds_out) *rounds_out = total_rounds;
    return GR_OK;
}

}  // namespace gr
