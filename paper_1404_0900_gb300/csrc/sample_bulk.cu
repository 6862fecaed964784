// sample_bulk.cu -- third tier of the IC RR sampler for the heaviest sets: a batched,
// level-synchronous reverse BFS (Section 3.1 "Implementation") over many RR sets at
// once.
//
// The warp-per-set tiers (sample.cu) give up on a set whose members outgrow their
// queues; such sets are rare but can be very large. Here S of them are expanded
// together, one BFS level per launch sequence:
//   - the level's frontier is a list of (slot, node) items (nodes with in-edges only);
//   - each item's in-list is cut into 4-aligned groups of in-CSR positions and an
//     exclusive scan over the items gives every group a global index (an in-list
//     under the geometric-skip rule of common.cuh gets one placeholder group, since
//     the group-to-item mapping needs every item to own a group; one warp per such
//     item draws its live in-edges in bulk_skip_kernel);
//   - warps take contiguous ranges of 32 groups, so a hub's in-list is spread over the
//     whole GPU; each lane draws one Philox block (4 coin words, keyed on set id and
//     in-CSR position, as in the first pass) and loads 4 thresholds with one 16-byte
//     load;
//   - a live in-edge whose source is new (test-and-set in the slot's visited bitmap)
//     adds the source to the slot's members and, if it has in-edges, to the next
//     frontier (warp-aggregated appends).
// After the last level, each slot's set is reduced (kappa), counted (cover) or copied
// into the RR-set store (emit), and the visited bits are cleared through the member
// list.
//
// The levels of a batch run in one persistent cooperative launch (bulk_levels_kernel):
// per level, (A) every block computes the group counts of a contiguous range of items
// and their sum, (B) every block turns its range into global group offsets from the sums
// of the blocks before it, (C) all warps expand the level; a bounded grid barrier
// separates the phases, so a level costs three barriers instead of a launch sequence
// and a host round trip. Frontier items, group offsets and block sums written during
// the launch are read with __ldcg (L2, not the SM's L1, which other SMs' writes do not
// update). Without cooperative launch support the same phases run as separate kernels
// stepped by the host.
#include <algorithm>

#include "common.cuh"

namespace {

struct BulkScalars {
    unsigned long long f_count;  // frontier items appended (all levels)
    unsigned long long m_count;  // members appended
    unsigned long long live;     // live in-edges followed
    unsigned long long exam;     // in-edges whose own coin was drawn
    // persistent launch, block 0: levels and nanoseconds in phases A + B, in C, at barriers
    unsigned long long levels, ns_offsets, ns_expand, ns_wait;
    int err;                     // bit 0: F overflow, bit 1: M overflow
    int pad;
};

struct BulkArgs {
    const uint64_t* rowptr;
    const uint32_t* src;
    const uint32_t* thr;
    const unsigned long long* node_thr;  // per-node shared threshold (bit 32: shared)
    const unsigned long long* qtab;      // gap tables of skip-rule nodes
    uint64_t n, m;
    PhiloxKeys K;
    uint64_t sid0;
    int flags, k;
    const uint32_t* seed_mark;
    const uint32_t* list;  // heavy set indices (relative to sid0)
    uint32_t base, S;      // this batch: slots s in [0, S) hold list[base + s]
    const uint32_t* hand;  // pass 2's state of the set at list position i < hcap (or null)
    uint32_t hcap, hw;
    uint32_t* bitmap;
    uint64_t words;
    unsigned long long* slot_width;
    uint32_t* slot_cnt;
    uint32_t* slot_flag;
    unsigned long long* slot_start;
    uint32_t* slot_cursor;
    uint4* F;  // frontier items: (in-list begin, end, set slot | skip flag << 31, node)
    uint64_t fcap;
    uint2* M;
    uint64_t mcap;
    BulkScalars* bs;
    uint64_t lvl_lo, lvl_n;  // current level: F[lvl_lo .. lvl_lo + lvl_n)
    uint32_t* ng;        // group count of each item of the level (bit 31: skip-rule item)
    uint64_t* gp;        // exclusive group prefix of the level, gp[lvl_n] = total
    unsigned long long* bsum;  // persistent launch: one group sum per block
    GridBarrier* bar;          // persistent launch: grid barrier, zeroed before the launch
    unsigned wait_limit;       // polls per barrier wait
    // outputs shared with the first pass
    DevScalars* ds;
    uint32_t* pool;
    uint32_t* pool_sid;
    uint64_t pool_cap;
    uint64_t* set_start;
    uint32_t* set_len;
    uint64_t* set_width;
};

__device__ __forceinline__ bool marked(const uint32_t* mark, uint32_t u) {
    return (__ldg(mark + (u >> 5)) >> (u & 31)) & 1u;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t pick4(uint4 v, int c) {
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}

// Warp-aggregated append of (slot, node) to one of the lists; returns nothing.
__device__ __forceinline__ void warp_append(bool pred, uint32_t s, uint32_t u,
                                            unsigned long long* counter, uint2* list,
                                            uint64_t cap, int* err, int errbit, int lane) {
    const uint32_t bal = __ballot_sync(0xffffffffu, pred);
    if (!bal) return;
    const int leader = __ffs(bal) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) {
        const unsigned long long pos = base + __popc(bal & ((1u << lane) - 1u));
        if (pos < cap)
            list[pos] = make_uint2(s, u);
        else
            atomicOr(err, errbit);
    }
}

// Warp-aggregated append of a frontier item to F.
__device__ __forceinline__ void warp_append_f(bool pred, uint4 item, unsigned long long* counter,
                                              uint4* list, uint64_t cap, int* err, int lane) {
    const uint32_t bal = __ballot_sync(0xffffffffu, pred);
    if (!bal) return;
    const int leader = __ffs(bal) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) {
        const unsigned long long pos = base + __popc(bal & ((1u << lane) - 1u));
        if (pos < cap)
            list[pos] = item;
        else
            atomicOr(err, 1);
    }
}

// The state pass 2 handed over for list position li, or null.
__device__ __forceinline__ const uint32_t* bulk_hand(const BulkArgs& a, uint64_t li) {
    if (!a.hand || li >= a.hcap) return nullptr;
    const uint32_t* hs = a.hand + li * (uint64_t)a.hw;
    const uint32_t t0 = hs[0];
    return t0 > 0 && t0 + 4 <= a.hw ? hs : nullptr;
}

// One thread per slot: a set without handed-over state starts from its root; a set with
// it gets its counters (width 0, its members' count) for bulk_hand_kernel to fill.
__global__ void bulk_init_kernel(BulkArgs a) {
    const bool cover = a.flags & SAMPLE_COVER;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < a.S; s += gridDim.x * blockDim.x) {
        const uint64_t li = (uint64_t)a.base + s;
        const uint32_t* hs = bulk_hand(a, li);
        a.slot_cursor[s] = 0;
        if (hs) {
            // the width pass 2 counted for the members before the batch it stopped at;
            // bulk_hand_kernel adds the in-degrees of the rest
            a.slot_width[s] = (unsigned long long)hs[2] | ((unsigned long long)hs[3] << 32);
            a.slot_cnt[s] = hs[0];
            a.slot_flag[s] = 0u;
            continue;
        }
        const uint32_t j = a.list[li];
        const uint64_t sid = a.sid0 + j;
        const uint32_t root = rr_root(sid, a.n, a.K);
        atomicOr(&a.bitmap[(uint64_t)s * a.words + (root >> 5)], 1u << (root & 31));
        const uint64_t beg = a.rowptr[root], end = a.rowptr[root + 1];
        a.slot_width[s] = end - beg;
        a.slot_cnt[s] = 1;
        const bool cov = cover && marked(a.seed_mark, root);
        a.slot_flag[s] = cov ? 1u : 0u;
        unsigned long long pm = atomicAdd(&a.bs->m_count, 1ull);
        if (pm < a.mcap)
            a.M[pm] = make_uint2(s, root);
        else
            atomicOr(&a.bs->err, 2);
        if (end > beg && !cov) {
            unsigned long long pf = atomicAdd(&a.bs->f_count, 1ull);
            const bool sk = tim_skip_rule(a.node_thr[root], end - beg);
            if (pf < a.fcap)
                a.F[pf] = make_uint4((uint32_t)beg, (uint32_t)end, s | (sk ? 0x80000000u : 0u),
                                     root);
            else
                atomicOr(&a.bs->err, 1);
        }
    }
}

// The members pass 2 found before it handed a set over, 32 per warp item over the whole
// grid (item = slot x 32-member chunk): visited bits, member list, the seed test (cover),
// and the members from the batch pass 2 was at on: their in-degrees into the set's
// width (pass 2 handed over the sum for the members before them) and, with in-edges,
// into the frontier (a covered set's frontier items are skipped when the level is
// expanded).
__global__ void bulk_hand_kernel(BulkArgs a, uint32_t chunks_per_slot) {
    const int lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const bool cover = a.flags & SAMPLE_COVER;
    const uint64_t items = (uint64_t)a.S * chunks_per_slot;
    for (uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; w < items; w += nw) {
        const uint32_t s = (uint32_t)(w / chunks_per_slot);
        const uint32_t c = (uint32_t)(w % chunks_per_slot);
        const uint32_t* hs = bulk_hand(a, (uint64_t)a.base + s);
        if (!hs) continue;
        const uint32_t t0 = hs[0];
        if (c * 32u >= t0) continue;
        const uint32_t h0 = min(hs[1], t0);
        const uint32_t i = c * 32u + lane;
        const bool h = i < t0;
        const uint32_t u = h ? hs[4 + i] : 0u;
        uint64_t beg = 0, end = 0;
        bool cov = false;
        if (h) {
            atomicOr(&a.bitmap[(uint64_t)s * a.words + (u >> 5)], 1u << (u & 31));
            if (i >= h0) {  // not yet expanded: its in-degree is not in the width yet
                beg = a.rowptr[u];
                end = a.rowptr[u + 1];
            }
            cov = cover && marked(a.seed_mark, u);
        }
        warp_append(h, s, u, &a.bs->m_count, a.M, a.mcap, &a.bs->err, 2, lane);
        const unsigned long long wsum = __reduce_add_sync(0xffffffffu, (unsigned)(end - beg));
        if (lane == 0 && wsum) atomicAdd(&a.slot_width[s], wsum);
        if (__any_sync(0xffffffffu, cov) && lane == 0) a.slot_flag[s] = 1u;
        const bool push = h && i >= h0 && end > beg;
        const uint4 item = make_uint4((uint32_t)beg, (uint32_t)end,
                                      s | (push && tim_skip_rule(a.node_thr[u], end - beg)
                                               ? 0x80000000u : 0u), u);
        warp_append_f(push, item, &a.bs->f_count, a.F, a.fcap, &a.bs->err, lane);
    }
}

constexpr uint32_t NG_SKIP = 0x80000000u;

// Groups of frontier item F[lo + i]: the 4-aligned groups of its in-list, or one
// placeholder group (flagged NG_SKIP) for a list under the skip rule.
__device__ __forceinline__ uint32_t item_groups(const BulkArgs& a, uint64_t lo, uint64_t i) {
    const uint4 it = __ldcg(&a.F[lo + i]);
    return (it.z >> 31) ? (1u | NG_SKIP) : ((it.y - 1) >> 2) - (it.x >> 2) + 1u;  // y > x
}

// Host-stepped path: group counts of the level without the skip flag (the scan input).
__global__ void bulk_ng_kernel(BulkArgs a) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.lvl_n;
         i += (uint64_t)gridDim.x * blockDim.x)
        a.ng[i] = item_groups(a, a.lvl_lo, i) & ~NG_SKIP;
}

// Appends of one warp staged in shared memory and copied to the global list in runs of
// up to WSTAGE items with one atomic on the list's counter (one address for the whole
// GPU, so one atomic per warp and step there would serialise): a warp flushes its
// buffer when the next append would not fit and when it leaves the expand phase.
constexpr uint32_t WSTAGE = 128;
// live in-edges (position, set slot) a warp queues in expand_level before it resolves
// them; one step adds at most 4 chunks x 32 lanes x 4 in-edges = 512
constexpr uint32_t LBUF = 768;
// groups of a super-chunk (8 chunks of 32), the unit of the expand phase
constexpr uint64_t SCG = 256;
// dynamic shared memory of the expand kernels: per warp, the two stages, the live queue
// and the boundary mask of a super-chunk
constexpr size_t EXPAND_SMEM =
    8 * (WSTAGE * (sizeof(uint2) + sizeof(uint4)) + LBUF * sizeof(uint2) + 8 * 4);
#ifndef LEVELS_MIN_BLOCKS
#define LEVELS_MIN_BLOCKS 2  // resident blocks per SM the persistent launch is built for
#endif

template <class T>
struct WarpStage {
    T* buf;      // WSTAGE entries in shared memory
    uint32_t n;  // entries held (the same on every lane)
};

template <class T>
__device__ __forceinline__ void wstage_flush(WarpStage<T>& ws, unsigned long long* counter,
                                             T* list, uint64_t cap, int* err, int errbit,
                                             int lane) {
    __syncwarp();
    if (ws.n) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(counter, (unsigned long long)ws.n);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (uint32_t i = lane; i < ws.n; i += 32) {
            if (base + i < cap)
                list[base + i] = ws.buf[i];
            else
                atomicOr(err, errbit);
        }
        ws.n = 0;
    }
    __syncwarp();
}

// Add the in-degrees and the number of a lane's new members (cnt, all of set slot s)
// to the set, one atomic pair per set and warp.
__device__ __forceinline__ void slot_add(bool fresh, uint32_t s, uint64_t deg, uint32_t cnt,
                                         const BulkArgs& a, int lane) {
    const uint32_t fm = __ballot_sync(0xffffffffu, fresh);
    if (!fresh) return;
    const uint32_t grp = __match_any_sync(fm, s);
    // the group's members are distinct nodes of one set: their in-degrees sum below m
    const unsigned dsum = __reduce_add_sync(grp, (unsigned)deg);
    const unsigned csum = __reduce_add_sync(grp, cnt);
    if (lane == __ffs(grp) - 1) {
        atomicAdd(&a.slot_width[s], (unsigned long long)dsum);
        atomicAdd(&a.slot_cnt[s], csum);
    }
}

// Append up to 4 items per lane (items[k] for bit k of bits) to the warp's stage: one
// warp scan, no atomic unless the stage has to be flushed first.
template <class T>
__device__ __forceinline__ void wstage_append4(uint32_t bits, const T* items, WarpStage<T>& ws,
                                               unsigned long long* counter, T* list,
                                               uint64_t cap, int* err, int errbit, int lane) {
    const uint32_t cnt = __popc(bits);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);  // <= 128 = WSTAGE
    if (total == 0) return;
    if (ws.n + total > WSTAGE) wstage_flush(ws, counter, list, cap, err, errbit, lane);
    uint32_t pos = ws.n + incl - cnt;
#pragma unroll
    for (int c = 0; c < 4; c++)
        if ((bits >> c) & 1u) ws.buf[pos++] = items[c];
    ws.n += total;
}

// Expand the level F[lo .. lo + nl) over its G = gp[nl] groups. Warp wid of nw takes a
// contiguous range of super-chunks (SCG groups). Per super-chunk the warp loads the
// group offsets of the 256 items after its first one (8 independent loads per lane)
// and marks the item starts in a 256-bit mask, so that every group finds its item and
// the item's first group by popcounts; then, four chunks at a time, every lane loads
// its group's item record, its 4 thresholds and draws its 4 coins, and the live
// in-edges are queued as (position, set slot). The queue is resolved in two sweeps:
// sources and visited-bit atomics, eight per lane in flight, then the new members'
// in-lists, four per lane in flight.
// Appends go through the warp's stages (members, frontier).
__device__ __forceinline__ void expand_level(const BulkArgs& a, uint64_t lo, uint64_t nl,
                                             uint2* mbuf, uint4* fbuf, uint2* lb,
                                             uint32_t* mwords, uint64_t wid, uint64_t nw,
                                             int lane) {
    WarpStage<uint2> wm{mbuf, 0u};
    WarpStage<uint4> wf{fbuf, 0u};
    const uint64_t G = __ldcg(a.gp + nl);
    const uint64_t nsc = (G + SCG - 1) / SCG;
    const uint64_t per = (nsc + nw - 1) / nw;
    const uint64_t sc0 = min(wid * per, nsc), sc1 = min(sc0 + per, nsc);
    const bool cover = a.flags & SAMPLE_COVER;
    uint32_t live_acc = 0, exam_acc = 0, nbuf = 0;
    auto drain = [&]() {
        __syncwarp();
        // sources and visited bits of every queued live in-edge, eight per lane in
        // flight; each entry becomes (source, slot | new << 31) (slots are below 2^16)
        for (uint32_t i0 = 0; i0 < nbuf; i0 += 256) {
            uint32_t u[8], old[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint32_t idx = i0 + 32u * q + lane;
                u[q] = idx < nbuf ? __ldg(a.src + lb[idx].x) : 0u;
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint32_t idx = i0 + 32u * q + lane;
                old[q] = idx < nbuf ? atomicOr(&a.bitmap[(uint64_t)lb[idx].y * a.words + (u[q] >> 5)],
                                               1u << (u[q] & 31))
                                    : 0u;
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const uint32_t idx = i0 + 32u * q + lane;
                if (idx < nbuf) {
                    const bool fresh = !(old[q] & (1u << (u[q] & 31)));
                    lb[idx] = make_uint2(u[q], lb[idx].y | (fresh ? 0x80000000u : 0u));
                }
            }
        }
        __syncwarp();
        // the new members: their in-lists and node words, four per lane in flight, then
        // the member and frontier appends
        for (uint32_t i = 0; i < nbuf; i += 128) {
            uint32_t u[4], sv[4], fr = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t idx = i + 32u * q + lane;
                const uint2 e = idx < nbuf ? lb[idx] : make_uint2(0u, 0u);
                u[q] = e.x;
                sv[q] = e.y & 0x7FFFFFFFu;
                if (e.y >> 31) fr |= 1u << q;
            }
            uint64_t d[4] = {0, 0, 0, 0};
            uint32_t push = 0;
            uint4 fi[4];
            uint2 mi[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                mi[q] = make_uint2(sv[q], u[q]);
                if ((fr >> q) & 1u) {
                    const uint64_t ub = __ldg(a.rowptr + u[q]), ue = __ldg(a.rowptr + u[q] + 1);
                    const unsigned long long nt = __ldg(a.node_thr + u[q]);
                    d[q] = ue - ub;
                    if (d[q]) push |= 1u << q;
                    fi[q] = make_uint4((uint32_t)ub, (uint32_t)ue,
                                       sv[q] | (tim_skip_rule(nt, ue - ub) ? 0x80000000u : 0u),
                                       u[q]);
                    if (cover && marked(a.seed_mark, u[q])) a.slot_flag[sv[q]] = 1u;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; q++) slot_add((fr >> q) & 1u, sv[q], d[q], 1u, a, lane);
            wstage_append4(fr, mi, wm, &a.bs->m_count, a.M, a.mcap, &a.bs->err, 2, lane);
            if (cover) {
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (((push >> q) & 1u) && a.slot_flag[sv[q]]) push &= ~(1u << q);
            }
            wstage_append4(push, fi, wf, &a.bs->f_count, a.F, a.fcap, &a.bs->err, 1, lane);
        }
        nbuf = 0;
        __syncwarp();
    };
    if (sc0 < sc1) {
        // the item holding group sc0 * SCG: the last i with gp[i] <= x, by a 32-ary
        // search of the warp (gp[0] = 0 <= x < gp[nl] = G, gp non-decreasing)
        uint64_t i0;
        {
            const uint64_t x = sc0 * SCG;
            uint64_t l = 0, h = nl;  // gp[l] <= x < gp[h]
            for (int guard = 0; guard < 16 && h - l > 1; guard++) {
                const uint64_t stride = (h - l + 31) >> 5;
                const uint64_t pr = l + (uint64_t)lane * stride;
                const bool le = pr < h && __ldcg(a.gp + pr) <= x;
                const uint32_t bl = __ballot_sync(0xffffffffu, le);  // lanes 0 .. k-1 hold
                const int k = 32 - __clz(bl);                         // bl has bit 0 set
                const uint64_t nl2 = l + (uint64_t)(k - 1) * stride;
                h = min(h, nl2 + stride);
                l = nl2;
            }
            i0 = l;
        }
        const uint32_t below = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
        for (uint64_t sc = sc0; sc < sc1; sc++) {
            const uint64_t S0 = sc * SCG;  // gp[i0] <= S0 < gp[i0 + 1]
            if (lane < 8) mwords[lane] = 0u;
            __syncwarp();
            uint32_t adv = 0;  // item starts in (S0, S0 + SCG]: the next super-chunk's i0
            uint64_t b[8];
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const uint64_t idx = i0 + 1 + (uint64_t)lane + 32ull * k;
                b[k] = idx <= nl ? __ldcg(a.gp + idx) : ~0ull;
            }
            const uint64_t gs0 = __ldcg(a.gp + i0);
#pragma unroll
            for (int k = 0; k < 8; k++) {
                if (b[k] <= S0 + SCG) adv++;
                if (b[k] < S0 + SCG)  // > S0: offsets after i0 exceed S0
                    atomicOr(&mwords[(uint32_t)(b[k] - S0) >> 5], 1u << ((uint32_t)(b[k] - S0) & 31));
            }
            adv = __reduce_add_sync(0xffffffffu, adv);
            __syncwarp();
            uint32_t mw[8];
#pragma unroll
            for (int k = 0; k < 8; k++) mw[k] = mwords[k];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                uint4 inf[4];
                uint64_t gof[4];  // group offset inside the item
                bool act[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int c = 4 * h + k;
                    const uint64_t t = S0 + (uint64_t)(c * 32 + lane);
                    act[k] = t < G;
                    // q = item starts at or before this group, pos = the last of them
                    const uint32_t cur = mw[c] & below;
                    uint32_t q = __popc(cur);
                    int pos = cur ? c * 32 + 31 - __clz(cur) : -1;
#pragma unroll
                    for (int w = 7; w >= 0; w--) {  // words below, highest first
                        if (w >= c) continue;
                        q += __popc(mw[w]);
                        if (pos < 0 && mw[w]) pos = w * 32 + 31 - __clz(mw[w]);
                    }
                    gof[k] = t - (q ? S0 + (uint64_t)pos : gs0);
                    inf[k] = act[k] ? __ldcg(&a.F[lo + i0 + q]) : make_uint4(0u, 0u, 0u, 0u);
                }
                uint4 tv[4];
                uint64_t g[4];
                uint32_t jj[4];
                bool wk[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    g[k] = ((uint64_t)inf[k].x >> 2) + gof[k];
                    const uint32_t sl = inf[k].z & 0x7FFFFFFFu;
                    wk[k] = act[k] && !(inf[k].z >> 31) &&
                            !(cover && *(volatile uint32_t*)&a.slot_flag[sl]);
                    tv[k] = wk[k] ? __ldg(reinterpret_cast<const uint4*>(a.thr) + g[k])
                                  : make_uint4(0u, 0u, 0u, 0u);
                    jj[k] = wk[k] ? __ldg(a.list + a.base + sl) : 0u;
                }
                uint32_t lm = 0;  // bit 4k + cc: position 4 g[k] + cc is live
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (!wk[k]) continue;
                    const uint64_t sid = a.sid0 + jj[k];
                    const uint4 x = philox4x32_10((uint32_t)sid, (uint32_t)(sid >> 32),
                                                  (uint32_t)g[k], TIM_TAG_IC, a.K);
#pragma unroll
                    for (int cc = 0; cc < 4; cc++) {
                        const uint64_t p = (g[k] << 2) + cc;
                        const uint32_t th = pick4(tv[k], cc);
                        if (p >= inf[k].x && p < inf[k].y) {
                            exam_acc++;
                            if (th == 0xFFFFFFFFu || pick4(x, cc) < th) lm |= 1u << (4 * k + cc);
                        }
                    }
                }
                const uint32_t cnt = __popc(lm);
                uint32_t incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                uint32_t qpos = nbuf + incl - cnt;
#pragma unroll
                for (int k = 0; k < 4; k++)
#pragma unroll
                    for (int cc = 0; cc < 4; cc++)
                        if ((lm >> (4 * k + cc)) & 1u)
                            lb[qpos++] = make_uint2((uint32_t)((g[k] << 2) + cc),
                                                    inf[k].z & 0x7FFFFFFFu);
                nbuf += __shfl_sync(0xffffffffu, incl, 31);
                live_acc += cnt;
                if (nbuf > LBUF - 512) drain();
            }
            i0 += adv;
        }
    }
    drain();
    wstage_flush(wm, &a.bs->m_count, a.M, a.mcap, &a.bs->err, 2, lane);
    wstage_flush(wf, &a.bs->f_count, a.F, a.fcap, &a.bs->err, 1, lane);
    live_acc = __reduce_add_sync(0xffffffffu, live_acc);
    exam_acc = __reduce_add_sync(0xffffffffu, exam_acc);
    if (lane == 0 && live_acc) atomicAdd(&a.bs->live, (unsigned long long)live_acc);
    if (lane == 0 && exam_acc) atomicAdd(&a.bs->exam, (unsigned long long)exam_acc);
}

// Shared memory of one warp in the expand kernels: member stage, frontier stage, live
// queue, boundary mask.
struct ExpandSmem {
    uint2* m;
    uint4* f;
    uint2* lb;
    uint32_t* mw;
};

__device__ __forceinline__ ExpandSmem expand_smem(unsigned char* dsm, int w) {
    ExpandSmem e;
    e.f = reinterpret_cast<uint4*>(dsm) + w * WSTAGE;
    e.m = reinterpret_cast<uint2*>(dsm + 8 * WSTAGE * sizeof(uint4)) + w * WSTAGE;
    e.lb = reinterpret_cast<uint2*>(dsm + 8 * WSTAGE * (sizeof(uint4) + sizeof(uint2))) + w * LBUF;
    e.mw = reinterpret_cast<uint32_t*>(dsm + 8 * WSTAGE * (sizeof(uint4) + sizeof(uint2)) +
                                       8 * LBUF * sizeof(uint2)) + w * 8;
    return e;
}

__global__ void __launch_bounds__(256) bulk_expand_kernel(BulkArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const ExpandSmem e = expand_smem(dsm, threadIdx.x >> 5);
    expand_level(a, a.lvl_lo, a.lvl_n, e.m, e.f, e.lb, e.mw,
                 (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5,
                 ((uint64_t)gridDim.x * blockDim.x) >> 5, threadIdx.x & 31);
}

// The level's items under the skip rule (flag of their frontier record), one warp per
// item; the lanes screen 32 items at a time.
__device__ __forceinline__ void skip_level(const BulkArgs& a, uint64_t lo, uint64_t nl,
                                           uint64_t wid, uint64_t nw, int lane) {
    const bool cover = a.flags & SAMPLE_COVER;
    uint32_t live_acc = 0;
    for (uint64_t base = wid * 32; base < nl; base += nw * 32) {
        const bool sk = base + lane < nl && (__ldcg(&a.F[lo + base + lane]).z >> 31);
        uint32_t todo = __ballot_sync(0xffffffffu, sk);
        while (todo) {
        const uint64_t i = base + (uint64_t)(__ffs(todo) - 1);
        todo &= todo - 1;
        const uint4 it = __ldcg(&a.F[lo + i]);
        const uint32_t s = it.z & 0x7FFFFFFFu, v = it.w;
        const uint64_t beg = it.x, end = it.y;
        const unsigned long long nt = __ldg(a.node_thr + v);
        if (cover && *(volatile uint32_t*)&a.slot_flag[s]) continue;
        const uint64_t sid = a.sid0 + __ldg(a.list + a.base + s);
        skip_live_warp((uint32_t)sid, (uint32_t)(sid >> 32), a.K, (uint32_t)beg,
                       (uint32_t)(end - beg), skip_table(a.qtab, nt), lane, [&](uint32_t p) {
                           bool fresh = false;
                           uint32_t u = 0;
                           uint64_t ub = 0, ue = 0;
                           unsigned long long unt = 0;
                           if (lane == 0) {
                               live_acc++;
                               u = __ldg(a.src + p);
                               const uint32_t b = 1u << (u & 31);
                               const uint32_t old =
                                   atomicOr(&a.bitmap[(uint64_t)s * a.words + (u >> 5)], b);
                               fresh = !(old & b);
                               if (fresh) {
                                   ub = __ldg(a.rowptr + u);
                                   ue = __ldg(a.rowptr + u + 1);
                                   unt = __ldg(a.node_thr + u);
                                   atomicAdd(&a.slot_width[s], ue - ub);
                                   atomicAdd(&a.slot_cnt[s], 1u);
                                   if (cover && marked(a.seed_mark, u)) a.slot_flag[s] = 1u;
                               }
                           }
                           warp_append(fresh, s, u, &a.bs->m_count, a.M, a.mcap, &a.bs->err, 2,
                                       lane);
                           const bool push = fresh && ue > ub && !(cover && a.slot_flag[s]);
                           const uint4 item = make_uint4(
                               (uint32_t)ub, (uint32_t)ue,
                               s | (tim_skip_rule(unt, ue - ub) ? 0x80000000u : 0u), u);
                           warp_append_f(push, item, &a.bs->f_count, a.F, a.fcap, &a.bs->err,
                                         lane);
                           return false;
                       });
        }
    }
    live_acc = __reduce_add_sync(0xffffffffu, live_acc);
    if (lane == 0 && live_acc) atomicAdd(&a.bs->live, (unsigned long long)live_acc);
}

__global__ void __launch_bounds__(256) bulk_skip_kernel(BulkArgs a) {
    skip_level(a, a.lvl_lo, a.lvl_n, (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5,
               ((uint64_t)gridDim.x * blockDim.x) >> 5, threadIdx.x & 31);
}

// Sum of v over the block (every thread gets it). blockDim.x is a multiple of 32, <= 1024.
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v,
                                                        unsigned long long* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    unsigned long long t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
    return t;
}

// Exclusive scan of x over the block; *total = the block's sum. Same conditions.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long x,
                                                              unsigned long long* red,
                                                              unsigned long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();
    if (lane == 31) red[w] = inc;
    __syncthreads();
    unsigned long long before = 0, all = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
        if (i < w) before += red[i];
        all += red[i];
    }
    *total = all;
    return before + inc - x;
}

// All levels of a batch in one cooperative launch (see the file comment). Every block
// reads the level bounds from f_count after the barrier that ends a level, before any
// block appends to F again, so all blocks agree on them; on a timeout or a full list
// every block leaves at the same barrier or the next one.
__global__ void __launch_bounds__(256, LEVELS_MIN_BLOCKS) bulk_levels_kernel(BulkArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ unsigned long long red[32];
    const int lane = threadIdx.x & 31;
    const uint64_t wid = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    int* err = &a.bs->err;
    uint64_t lo = 0, hi = __ldcg(&a.bs->f_count);
    if (__ldcg(err)) return;
    // block 0 accounts where its time goes (phases and barrier waits)
    const bool clerk = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_prev = clerk ? globaltimer_ns() : 0ull, ns_off = 0, ns_exp = 0,
                       ns_wait = 0, nlev = 0;
    auto lap = [&](unsigned long long& acc) {
        if (clerk) {
            const unsigned long long t = globaltimer_ns();
            acc += t - t_prev;
            t_prev = t;
        }
    };
    auto account = [&]() {
        if (clerk) {
            a.bs->levels += nlev;
            a.bs->ns_offsets += ns_off;
            a.bs->ns_expand += ns_exp;
            a.bs->ns_wait += ns_wait;
        }
    };
    for (int level = 0; level < (1 << 26) && hi > lo; level++) {
        nlev++;
        const uint64_t nl = hi - lo;
        if (nl > a.fcap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, 1);
            return;
        }
        // (A) group counts of this block's items and their sum
        const uint64_t per = (nl + gridDim.x - 1) / gridDim.x;
        const uint64_t ib = min((uint64_t)blockIdx.x * per, nl), ie = min(ib + per, nl);
        unsigned long long sum = 0;
        for (uint64_t i = ib + threadIdx.x; i < ie; i += blockDim.x) {
            const uint32_t g = item_groups(a, lo, i);
            a.ng[i] = g;
            sum += g & ~NG_SKIP;
        }
        sum = block_sum(sum, red);
        if (threadIdx.x == 0) a.bsum[blockIdx.x] = sum;
        lap(ns_off);
        if (!grid_barrier(a.bar, err, a.wait_limit)) return;
        lap(ns_wait);
        // (B) global group offsets of this block's items
        unsigned long long before = 0, all = 0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
            const unsigned long long x = __ldcg(a.bsum + b);
            if (b < blockIdx.x) before += x;
            all += x;
        }
        before = block_sum(before, red);
        all = block_sum(all, red);
        for (uint64_t c = ib; c < ie; c += blockDim.x) {
            const uint64_t i = c + threadIdx.x;
            const unsigned long long g = i < ie ? (a.ng[i] & ~NG_SKIP) : 0u;
            unsigned long long tot;
            const unsigned long long ex = block_excl_scan(g, red, &tot);
            if (i < ie) a.gp[i] = before + ex;
            before += tot;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.gp[nl] = all;
        lap(ns_off);
        if (!grid_barrier(a.bar, err, a.wait_limit)) return;
        lap(ns_wait);
        // (C) expand: in-lists by groups over all warps, skip-rule lists by one warp each
        {
            const ExpandSmem e = expand_smem(dsm, threadIdx.x >> 5);
            expand_level(a, lo, nl, e.m, e.f, e.lb, e.mw, wid, nw, lane);
        }
        skip_level(a, lo, nl, wid, nw, lane);
        lap(ns_exp);
        if (!grid_barrier(a.bar, err, a.wait_limit)) return;
        lap(ns_wait);
        lo = hi;
        hi = __ldcg(&a.bs->f_count);
        if (__ldcg(err)) {
            account();
            return;
        }
    }
    account();
}

__global__ void bulk_finalize_kernel(BulkArgs a) {
    const bool emit = a.flags & SAMPLE_EMIT, kap = a.flags & SAMPLE_KAPPA,
               cover = a.flags & SAMPLE_COVER;
    unsigned long long k_lo = 0, k_hi = 0, wsum = 0, cov = 0, memb = 0;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < a.S; s += gridDim.x * blockDim.x) {
        const uint32_t j = a.list[a.base + s];
        const unsigned long long w = a.slot_width[s];
        const uint32_t cnt = a.slot_cnt[s];
        wsum += w;
        memb += cnt;
        if (cover && a.slot_flag[s]) cov++;
        if (kap) {
            const unsigned long long kf = kappa_fixed(kappa_fp64(w, a.m, a.k));
            k_lo += kf;
            if (k_lo < kf) k_hi++;
        }
        if (emit) {
            const unsigned long long st = atomicAdd(&a.ds->pool_used, (unsigned long long)cnt);
            a.slot_start[s] = st;
            if (st + cnt <= a.pool_cap) {
                a.set_start[j] = st;
                a.set_len[j] = cnt;
                a.set_width[j] = w;
            } else {
                atomicOr(&a.ds->err, TIM_DEV_ERR_POOL);
            }
        }
    }
    if (kap && (k_lo || k_hi)) atomic_add_u128(&a.ds->ksum_lo, &a.ds->ksum_hi, k_lo, k_hi);
    if (wsum) {
        atomicAdd(&a.ds->wsum, wsum);
        atomicAdd(&a.ds->width[2], wsum);
    }
    if (cov) atomicAdd(&a.ds->covered, cov);
    if (memb) atomicAdd(&a.ds->memb[2], memb);
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.bs->exam) atomicAdd(&a.ds->exam[2], a.bs->exam);
}

// Copy members into the store (emit) and clear the visited bits, one member each.
__global__ void bulk_emit_clear_kernel(BulkArgs a, unsigned long long mcount, int emit) {
    const int lane = threadIdx.x & 31;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < mcount;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 it = a.M[e];
        if (emit) {
            // one cursor atomic per set and warp (staged appends keep a set's members
            // together)
            const uint32_t grp = __match_any_sync(__activemask(), it.x);
            const int leader = __ffs(grp) - 1;
            const unsigned long long st = a.slot_start[it.x];
            const uint32_t cnt = a.slot_cnt[it.x];
            uint32_t base = 0;
            if (lane == leader && st + cnt <= a.pool_cap)
                base = atomicAdd(&a.slot_cursor[it.x], (unsigned)__popc(grp));
            base = __shfl_sync(grp, base, leader);
            if (st + cnt <= a.pool_cap) {
                const uint32_t pos = base + __popc(grp & ((1u << lane) - 1u));
                a.pool[st + pos] = it.y;
                a.pool_sid[st + pos] = a.list[a.base + it.x];
            }
        }
        a.bitmap[(uint64_t)it.x * a.words + (it.y >> 5)] = 0u;
    }
}

}  // namespace

// Heavy IC sets listed in ctx->ovf_list[0 .. count): expand them in batches.
int tim_bulk_ic(tim_ctx* ctx, const SampleRequest& req, const uint32_t* list, uint32_t count,
                uint32_t* pool, uint32_t* pool_sid, uint64_t pool_cap, DevScalars* ds,
                uint64_t* live_out, const uint32_t* hand, uint32_t hcap, uint32_t hw) {
    if (count == 0) return TIM_OK;
    const uint64_t n = (uint64_t)ctx->n;
    const uint64_t words = (n + 31) / 32 + 1;
    // slots: one visited bitmap of n bits per set of a batch, at most 16 GiB of them in
    // all (a quarter of the device memory free at the context's first heavy pass, if
    // that is less), at least 32; the buffers grow to the next power of two of the sets
    // a call lists. Larger batches mean fewer levels for the same sets (TIM+ on a
    // 41.6M-node, 1.4B-edge Chung-Lu graph: 32 batches and ~1,460 levels per run with
    // 2 GiB of bitmaps, TIM+ 263 -> 246 ms with 16 GiB).
    if (ctx->bulk_budget == 0) {
        size_t fr = 0, tot = 0;
        ctx->bulk_budget = 16ull << 30;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
            ctx->bulk_budget = std::min<uint64_t>(ctx->bulk_budget, fr / 4);
        else
            cudaGetLastError();
    }
    uint64_t smax = std::max<uint64_t>(32, ctx->bulk_budget / (words * 4));
    smax = std::min<uint64_t>(smax, 65536);
    uint64_t slots = 32;
    while (slots < count && slots < smax) slots <<= 1;
    smax = std::min<uint64_t>(slots, smax);
    uint32_t S = (uint32_t)std::min<uint64_t>(smax, count);
    void* prev_bitmap = ctx->bulk_bitmap.p;
    TIM_TRY(tim_ensure(ctx, ctx->bulk_bitmap, (size_t)smax * words * 4));
    if (ctx->bulk_bitmap.p != prev_bitmap) ctx->bulk_bitmap_clean = false;
    if (!ctx->bulk_bitmap_clean) {
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->bulk_bitmap.p, 0, ctx->bulk_bitmap.bytes, ctx->stream));
        ctx->bulk_bitmap_clean = true;
    }
    TIM_TRY(tim_ensure(ctx, ctx->bulk_slot, (size_t)smax * 40));
    if (ctx->bulk_fcap == 0) ctx->bulk_fcap = 1 << 22;
    if (ctx->bulk_mcap == 0) ctx->bulk_mcap = 1 << 22;
    TIM_TRY(tim_ensure(ctx, ctx->bulk_F, ctx->bulk_fcap * sizeof(uint4)));
    TIM_TRY(tim_ensure(ctx, ctx->bulk_M, ctx->bulk_mcap * sizeof(uint2)));
    TIM_TRY(tim_ensure(ctx, ctx->bulk_ng, ctx->bulk_fcap * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->bulk_gp, (ctx->bulk_fcap + 1) * sizeof(uint64_t)));
    TIM_TRY(tim_ensure(ctx, ctx->bulk_scal, sizeof(BulkScalars)));
    CUDA_TRY(ctx, cudaFuncSetAttribute(bulk_levels_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)EXPAND_SMEM));
    CUDA_TRY(ctx, cudaFuncSetAttribute(bulk_expand_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)EXPAND_SMEM));
    // persistent launch: co-resident blocks (at most 4 per SM), their sums and a barrier
    int coop = 0, nb = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (!ctx->bulk_stepped && coop &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bulk_levels_kernel, 256, EXPAND_SMEM) !=
            cudaSuccess) {
        cudaGetLastError();
        nb = 0;
    }
    const bool persistent = !ctx->bulk_stepped && coop && nb > 0;
    const unsigned GP = (unsigned)(ctx->num_sms * std::min(nb, 4));
    if (persistent) {
        TIM_TRY(tim_ensure(ctx, ctx->bulk_bsum, (size_t)GP * sizeof(unsigned long long)));
        TIM_TRY(tim_ensure(ctx, ctx->bulk_bar, sizeof(GridBarrier)));
    }

    BulkArgs a;
    a.rowptr = (const uint64_t*)ctx->rowptr.p;
    a.src = (const uint32_t*)ctx->src.p;
    a.thr = (const uint32_t*)ctx->thr.p;
    a.node_thr = (const unsigned long long*)ctx->node_thr.p;
    a.qtab = (const unsigned long long*)ctx->qtab.p;
    a.n = n;
    a.m = (uint64_t)ctx->m;
    a.K = tim_philox_keys(req.seed);
    a.sid0 = req.sid0;
    a.flags = req.flags;
    a.k = req.k;
    a.seed_mark = req.seed_mark;
    a.list = list;
    a.hand = hand;
    a.hcap = hand ? hcap : 0u;
    a.hw = hw;
    a.bitmap = (uint32_t*)ctx->bulk_bitmap.p;
    a.words = words;
    char* sl = (char*)ctx->bulk_slot.p;
    a.slot_width = (unsigned long long*)sl;
    a.slot_start = (unsigned long long*)(sl + smax * 8);
    a.slot_cnt = (uint32_t*)(sl + smax * 16);
    a.slot_flag = (uint32_t*)(sl + smax * 20);
    a.slot_cursor = (uint32_t*)(sl + smax * 24);
    a.bs = (BulkScalars*)ctx->bulk_scal.p;
    a.ds = ds;
    a.pool = pool;
    a.pool_sid = pool_sid;
    a.pool_cap = pool_cap;
    a.set_start = (uint64_t*)ctx->set_start.p;
    a.set_len = (uint32_t*)ctx->set_len.p;
    a.set_width = (uint64_t*)ctx->set_width.p;
    a.bsum = (unsigned long long*)ctx->bulk_bsum.p;
    a.bar = (GridBarrier*)ctx->bulk_bar.p;
    a.wait_limit = ctx->wait_limit;
    BulkScalars hb;
    const unsigned GX = (unsigned)(ctx->num_sms * 4);
    uint32_t done = 0;
    uint64_t live = 0;
    while (done < count) {
        const uint32_t bs = std::min<uint32_t>(S, count - done);
        a.base = done;
        a.S = bs;
        a.F = (uint4*)ctx->bulk_F.p;
        a.M = (uint2*)ctx->bulk_M.p;
        a.fcap = ctx->bulk_fcap;
        a.mcap = ctx->bulk_mcap;
        a.ng = (uint32_t*)ctx->bulk_ng.p;
        a.gp = (uint64_t*)ctx->bulk_gp.p;
        CUDA_TRY(ctx, cudaMemsetAsync(a.bs, 0, sizeof(BulkScalars), ctx->stream));
        bulk_init_kernel<<<(bs + 255) / 256, 256, 0, ctx->stream>>>(a);
        LAUNCH_CHECK(ctx, "bulk_init_kernel");
        if (a.hand) {
            bulk_hand_kernel<<<(unsigned)(ctx->num_sms * 8), 256, 0, ctx->stream>>>(
                a, (hw > 4 ? hw - 4 + 31 : 0) / 32);
            LAUNCH_CHECK(ctx, "bulk_hand_kernel");
        }
        uint64_t lo = 0, hi = 0;
        bool overflow = false;
        if (persistent) {
            CUDA_TRY(ctx, cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), ctx->stream));
            void* args[] = {&a};
            cudaEventRecord(ctx->bev[0], ctx->stream);
            CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)bulk_levels_kernel, dim3(GP),
                                                      dim3(256), args, EXPAND_SMEM,
                                                      ctx->stream));
            LAUNCH_CHECK(ctx, "bulk_levels_kernel");
            cudaEventRecord(ctx->bev[1], ctx->stream);
            CUDA_TRY(ctx, cudaMemcpyAsync(&hb, a.bs, sizeof hb, cudaMemcpyDeviceToHost,
                                          ctx->stream));
            TIM_TRY(tim_sync(ctx));
            float kms = 0.f;
            cudaEventElapsedTime(&kms, ctx->bev[0], ctx->bev[1]);
            ctx->prof.pass3_ms_kernel += kms;
            if (hb.err & TIM_DEV_ERR_TIMEOUT) {
                ctx->bulk_bitmap_clean = false;
                return tim_fail(ctx, TIM_ERR_TIMEOUT, "heavy-set grid barrier timed out");
            }
            overflow = hb.err != 0;
        } else {
            CUDA_TRY(ctx, cudaMemcpyAsync(&hb, a.bs, sizeof hb, cudaMemcpyDeviceToHost,
                                          ctx->stream));
            TIM_TRY(tim_sync(ctx));
            hi = hb.f_count;
            overflow = hb.err != 0;
        }
        for (int level = 0; !persistent && !overflow && hi > lo && level < (1 << 26); level++) {
            a.lvl_lo = lo;
            a.lvl_n = hi - lo;
            if (a.lvl_n > ctx->bulk_fcap) {
                overflow = true;
                break;
            }
            bulk_ng_kernel<<<GX * 2, 256, 0, ctx->stream>>>(a);
            LAUNCH_CHECK(ctx, "bulk_ng_kernel");
            TIM_TRY(tim_scan_u32_to_u64(ctx, (const uint32_t*)ctx->bulk_ng.p,
                                        (uint64_t*)ctx->bulk_gp.p, a.lvl_n));
            bulk_expand_kernel<<<GX * 4, 256, EXPAND_SMEM, ctx->stream>>>(a);
            LAUNCH_CHECK(ctx, "bulk_expand_kernel");
            bulk_skip_kernel<<<GX * 2, 256, 0, ctx->stream>>>(a);
            LAUNCH_CHECK(ctx, "bulk_skip_kernel");
            CUDA_TRY(ctx, cudaMemcpyAsync(&hb, a.bs, sizeof hb, cudaMemcpyDeviceToHost, ctx->stream));
            TIM_TRY(tim_sync(ctx));
            if (hb.err) overflow = true;
            lo = hi;
            hi = hb.f_count;
        }
        if (overflow) {
            // grow the lists and redo this batch from scratch
            CUDA_TRY(ctx, cudaMemsetAsync(ctx->bulk_bitmap.p, 0, ctx->bulk_bitmap.bytes, ctx->stream));
            if (hb.err & 1 || hi - lo > ctx->bulk_fcap) ctx->bulk_fcap *= 2;
            if (hb.err & 2) ctx->bulk_mcap *= 2;
            if (ctx->bulk_fcap > (1ull << 31) || ctx->bulk_mcap > (1ull << 31))
                return tim_fail(ctx, TIM_ERR_OOM, "heavy-set lists exceed 2^31 entries");
            tim_free(ctx->bulk_F);
            tim_free(ctx->bulk_M);
            tim_free(ctx->bulk_ng);
            tim_free(ctx->bulk_gp);
            TIM_TRY(tim_ensure(ctx, ctx->bulk_F, ctx->bulk_fcap * sizeof(uint4)));
            TIM_TRY(tim_ensure(ctx, ctx->bulk_M, ctx->bulk_mcap * sizeof(uint2)));
            TIM_TRY(tim_ensure(ctx, ctx->bulk_ng, ctx->bulk_fcap * sizeof(uint32_t)));
                    TIM_TRY(tim_ensure(ctx, ctx->bulk_gp, (ctx->bulk_fcap + 1) * sizeof(uint64_t)));
            continue;
        }
        bulk_finalize_kernel<<<(bs + 255) / 256, 256, 0, ctx->stream>>>(a);
        LAUNCH_CHECK(ctx, "bulk_finalize_kernel");
        const unsigned long long mc = hb.m_count;
        bulk_emit_clear_kernel<<<GX * 2, 256, 0, ctx->stream>>>(a, mc,
                                                               (req.flags & SAMPLE_EMIT) ? 1 : 0);
        LAUNCH_CHECK(ctx, "bulk_emit_clear_kernel");
        live += hb.live;
        done += bs;
        if (persistent) {
            tim_profile& P = ctx->prof;
            P.pass3_batches += 1;
            P.pass3_levels += hb.levels;
            P.pass3_ms_offsets += hb.ns_offsets * 1e-6;
            P.pass3_ms_expand += hb.ns_expand * 1e-6;
            P.pass3_ms_wait += hb.ns_wait * 1e-6;
        }
    }
    if (live_out) *live_out = live;
    return TIM_OK;
}
