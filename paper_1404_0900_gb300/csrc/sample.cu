// sample.cu -- random RR sets on the GPU (Definitions 1-2; randomised BFS of Section
// 3.1 "Implementation" for IC; the triggering-model BFS of Section 4.2 with the LT
// triggering distribution of Section 6).
//
// Every coin is keyed on (seed, set id, in-CSR position) and every LT draw on (seed,
// set id, node), so a set does not depend on which kernel expands it, in what order,
// or on how many threads: the three tiers below give identical sets.
//
// Tier 1: a persistent kernel with one warp per RR set; the set's BFS queue (which is
//   also its member list) and a visited hash live in shared memory. A frontier of up
//   to 32 nodes is expanded at once: their in-lists are cut into 4-aligned groups of
//   in-CSR positions, spread over the lanes, and each lane draws one Philox block (4
//   coin words) and loads 4 thresholds with one 16-byte load. A set whose members
//   outgrow the queue, or (IC) whose examined in-edges would pass a budget, is listed
//   for tier 2. This keeps the kernel's tail short: light sets are most sets.
// An IC set that tier 1 gives up on is handed over with its state (the queue so far,
//   the frontier batch to redo, the width before it), and tier 2 goes on from there
//   instead of starting again from the root (the coins are keyed, so the set is the same).
// Tier 2: the same code with a 32x larger queue and hash in global memory (one arena
//   slot per team; the queue tail and status stay in shared memory, since every new
//   member takes a tail atomic) and no edge budget, run by teams of T warps per set: T = 1 when the
//   listed sets are many (parallelism across sets fills the GPU), up to 8 when they are
//   few (the team splits each in-list, so one heavy set does not leave the GPU idle).
// In-lists of at least BIG_GROUPS groups (hubs) are streamed by the whole team one at
// a time with two groups in flight per lane; the rest of a frontier is flattened.
// Tier 3: sets beyond tier 2's queue: IC goes to the batched level-synchronous pass of
//   sample_bulk.cu; LT (a chain) is walked by one warp per set with a visited bitmap; a
//   general triggering model's set is expanded level by level by one block per set.
//
// Per set the kernels can (flags): EMIT the members into the RR-set store, sum KAPPA
// (Eq. 6) in 2^-63 fixed point, and test COVER (does the set meet a given seed set;
// the coverage test of Algorithm 3; the BFS stops at the first member in the seed set).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr int ST_OVERFLOW = 1;
constexpr int ST_COVERED = 2;
constexpr int WARPS = 8;          // warps per CTA (tiers 1 and 2)
constexpr int BIG_THREADS = 256;  // tier 3 LT CTA size

// Queue capacity Q and hash size 2^LOG2H (>= 2Q) of one warp's set.
template <int QQ, int LG>
struct Cap {
    static constexpr int Q = QQ;
    static constexpr int LOG2H = LG;
    static constexpr int H = 1 << LG;
    // hash[H] u32, queue[Q] u32, slot[Q] u16, ctl[4] int
    static constexpr int WORDS = (1 << LG) + QQ + QQ / 2 + 4;
};
using Tier1 = Cap<256, 9>;
// the other first-pass capacities the autotuner may choose for IC
using Tier1S = Cap<128, 8>;
using Tier1L = Cap<512, 10>;
using Tier2 = Cap<8192, 14>;

struct SampleArgs {
    const uint64_t* rowptr;
    const uint32_t* src;
    const uint32_t* thr;
    const unsigned long long* node_thr;  // IC: per-node shared threshold (bit 32: shared)
    const unsigned long long* qtab;      // IC: gap tables of skip-rule nodes
    uint64_t n, m;
    PhiloxKeys K;
    uint64_t sid0, count;
    int flags, k;
    const uint32_t* seed_mark;
    uint32_t* pool;
    uint32_t* pool_sid;
    uint64_t pool_cap;
    uint64_t* set_start;
    uint32_t* set_len;
    uint64_t* set_width;
    DevScalars* ds;
    uint32_t* list1;   // tier 1 -> tier 2
    uint32_t* list2;   // tier 2 -> tier 3
    uint32_t list_cap;
    uint32_t* arena;   // tier 2 per-warp storage
    uint32_t* big_bitmap;  // tier 3 LT
    uint32_t* big_queue;
    uint64_t big_words;
    unsigned long long width_budget;  // tier 1 IC: in-edges one warp may examine per set
    unsigned long long width_budget2; // tier 2 IC: in-edges one team may examine per set
    int chunk;                        // sets claimed per work-counter increment
    uint32_t* lt_col;                 // tier 1 LT: per-thread member columns
    // IC: the state pass 1 hands to pass 2 for the set at list1 position i < hcap, hw
    // words at hand + i hw: queue length, resume position, width so far (2 words), queue
    uint32_t* hand;
    uint32_t hcap, hw;
    // IC: the state pass 2 hands to the heavy pass for the set at list2 position i < h2cap,
    // h2w words at hand2 + i h2w: queue length, resume position, width before it (2
    // words), queue
    uint32_t* hand2;
    uint32_t h2cap, h2w;
    // triggering model: options of each node, their cumulative thresholds, their in-edges
    const uint64_t* node_opt;
    const uint32_t* opt_cum;
    const uint64_t* opt_off;
    const uint32_t* opt_pos;
};

__device__ __forceinline__ uint4 draw(const SampleArgs& a, uint64_t sid, uint32_t elem,
                                      uint32_t tag) {
    return philox4x32_10((uint32_t)sid, (uint32_t)(sid >> 32), elem, tag, a.K);
}

__device__ __forceinline__ bool marked(const uint32_t* mark, uint32_t u) {
    return (__ldg(mark + (u >> 5)) >> (u & 31)) & 1u;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Visited set of one RR set: insert u. Returns INS_NEW, INS_OLD, or INS_FULL when the
// queue or the hash is full (the set then moves to the next tier). Bounded probing.
constexpr int INS_OLD = 0, INS_NEW = 1, INS_FULL = 2;

template <class C>
__device__ __forceinline__ int set_insert(uint32_t* hash, uint32_t* queue, uint16_t* slot,
                                          int* ctl, uint32_t u) {
    uint32_t h = (u * 0x9E3779B1u) >> (32 - C::LOG2H);
    for (int probe = 0; probe < C::H; probe++) {
        uint32_t old = atomicCAS(&hash[h], EMPTY, u);
        if (old == EMPTY) {
            int pos = atomicAdd(&ctl[0], 1);
            if (pos < C::Q) {
                queue[pos] = u;
                slot[pos] = (uint16_t)h;
                return INS_NEW;
            }
            atomicOr(&ctl[1], ST_OVERFLOW);
            return INS_FULL;
        }
        if (old == u) return INS_OLD;
        h = (h + 1) & (C::H - 1);
    }
    atomicOr(&ctl[1], ST_OVERFLOW);
    return INS_FULL;
}

// First position j in [lo, hi) with thr[j] > x (thr non-decreasing), or hi.
// 32-ary search by the whole warp.
__device__ __forceinline__ uint64_t warp_lt_search(const uint32_t* __restrict__ thr, uint64_t lo,
                                                   uint64_t hi, uint32_t x, int lane) {
    for (int it = 0; it < 16 && hi - lo > 32; it++) {
        uint64_t stride = (hi - lo + 31) >> 5;
        uint64_t p = lo + (uint64_t)(lane + 1) * stride - 1;
        bool valid = p < hi;
        bool pred = valid && __ldg(thr + p) > x;
        uint32_t b = __ballot_sync(0xffffffffu, pred);
        if (b) {
            int f = __ffs(b) - 1;
            uint64_t nlo = lo + (uint64_t)f * stride;
            hi = nlo + stride;
            lo = nlo;
        } else {
            lo += (uint64_t)__popc(__ballot_sync(0xffffffffu, valid)) * stride;
        }
    }
    uint64_t p = lo + lane;
    bool pred = p < hi && __ldg(thr + p) > x;
    uint32_t b = __ballot_sync(0xffffffffu, pred);
    return b ? lo + (uint64_t)(__ffs(b) - 1) : hi;
}

// ------------------------------------------------------------ tiers 1 and 2

// Barrier over the T warps of a team (T = 1: the warp itself). Named barrier ids
// 1..8 are one per team of the block; 0 stays free for __syncthreads.
template <int T>
__device__ __forceinline__ void team_sync(int team) {
    if (T == 1)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(T * 32) : "memory");
}

// Which of the in-CSR positions 4g .. 4g+3 lie in [beg, end) (bit c = position 4g+c).
// Positions are 32-bit: the graph loader rejects m >= 2^32.
__device__ __forceinline__ uint32_t range_mask(uint32_t g, uint32_t beg, uint32_t end) {
    const uint32_t p0 = g << 2;
    if (p0 >= beg && p0 + 4u <= end) return 0xFu;
    const uint32_t lo = beg > p0 ? beg - p0 : 0u;
    const uint32_t hi = end < p0 + 4u ? end - p0 : 4u;
    return ((1u << hi) - 1u) & ~((1u << lo) - 1u);
}

// Live coins of one group whose 4 in-edges share threshold t (0 < t < 0xFFFFFFFF).
__device__ __forceinline__ uint32_t live_mask_shared(uint4 x, uint32_t t) {
    return (x.x < t ? 1u : 0u) | (x.y < t ? 2u : 0u) | (x.z < t ? 4u : 0u) |
           (x.w < t ? 8u : 0u);
}

// Live coins of one group: bit c set iff word c < thr c, or thr c marks p >= 1.
__device__ __forceinline__ uint32_t live_mask(uint4 x, uint4 t) {
    return ((x.x < t.x) | (t.x == 0xFFFFFFFFu) ? 1u : 0u) |
           ((x.y < t.y) | (t.y == 0xFFFFFFFFu) ? 2u : 0u) |
           ((x.z < t.z) | (t.z == 0xFFFFFFFFu) ? 4u : 0u) |
           ((x.w < t.w) | (t.w == 0xFFFFFFFFu) ? 8u : 0u);
}

// Follow the live in-edges of group g given their mask: insert each source. Returns
// bit 0 if the set overflowed, bit 1 if it met the seed set.
template <class C, class A>
__device__ __forceinline__ int follow_live(const A& a, uint32_t g, uint32_t mask,
                                        uint32_t* hash, uint32_t* queue, uint16_t* slot,
                                        int* ctl) {
    int f = 0;
    while (mask) {
        const int c = __ffs(mask) - 1;
        mask &= mask - 1;
        const uint32_t u = __ldg(a.src + ((g << 2) + c));
        const int r = set_insert<C>(hash, queue, slot, ctl, u);
        if (r == INS_FULL) {
            f |= 1;
        } else if (r == INS_NEW && (a.flags & SAMPLE_COVER) && marked(a.seed_mark, u)) {
            atomicOr(&ctl[1], ST_COVERED);
            f |= 2;
        }
    }
    return f;
}

// In-lists with at least this many 4-edge groups are expanded one at a time by the
// whole team (no ownership search, two groups in flight per lane).
constexpr uint32_t BIG_GROUPS = 32;

// Where an IC expansion stopped: the queue position of the frontier batch to process
// next and the width of the members before it.
struct Resume {
    int head;
    unsigned long long width;
};

// Expand one RR set with a team of T warps (wt = warp index in the team, team = team
// index in the block). IC only: with `in` the queue, hash and ctl already hold a set
// that an earlier pass stopped (queue[0 .. ctl[0])), and the expansion goes on from
// in->head with width in->width; with `out`, an expansion that stops records where. Returns the status bits; *width_out = w(R) (Eq. 1); *live_out
// counts live in-edges followed (per lane).
template <int MODEL, class C, int T, class A>
__device__ __forceinline__ int team_rr(const A& a, const PhiloxKeys& K, uint64_t sid, uint32_t* hash,
                                       uint32_t* queue, uint16_t* slot, int* ctl,
                                       unsigned long long budget, int wt, int team,
                                       unsigned long long* width_out,
                                       unsigned long long* live_out,
                                       unsigned long long* exam_out,
                                       const Resume* in = nullptr, Resume* out = nullptr) {
    const int lane = threadIdx.x & 31;
    volatile int* vctl = ctl;
    const bool cover = a.flags & SAMPLE_COVER;
    const uint32_t root = rr_root(sid, a.n, K);
    if (!in && wt == 0 && lane == 0) {
        uint32_t h = (root * 0x9E3779B1u) >> (32 - C::LOG2H);
        hash[h] = root;
        queue[0] = root;
        slot[0] = (uint16_t)h;
        ctl[0] = 1;
        ctl[1] = (cover && marked(a.seed_mark, root)) ? ST_COVERED : 0;
    }
    team_sync<T>(team);
    unsigned long long width = in ? in->width : 0, live = 0, work = 0, exam = 0;
    if constexpr (MODEL == TIM_IC) {
        const uint32_t s0 = (uint32_t)sid, s1 = (uint32_t)(sid >> 32);
        const uint4* thr4 = reinterpret_cast<const uint4*>(a.thr);
        int head = in ? in->head : 0;
        int bh = head;                // the batch being processed and the width before it
        unsigned long long bw = width;
        for (int guard = 0; guard < C::Q + 1; guard++) {
            // a consistent snapshot of (tail, status) for the whole team
            int tail, stat;
            if (T == 1) {
                tail = __shfl_sync(0xffffffffu, vctl[0], 0);
                stat = __shfl_sync(0xffffffffu, vctl[1], 0);
            } else {
                tail = vctl[0];
                stat = vctl[1];
                team_sync<T>(team);
            }
            if (stat || head >= tail) break;
            bh = head;
            bw = width;
            const int nb = min(32, tail - head);
            uint64_t beg = 0, end = 0;
            // a node's in-edges often share one threshold (weighted cascade: p = 1/indeg);
            // then no threshold is loaded, t = 0 needs no coins, t = 2^32-1 (p >= 1)
            // makes every in-edge live without a draw, and a long list is sampled by
            // geometric skipping
            unsigned long long nt = 0;
            if (lane < nb) {
                const uint32_t v = queue[head + lane];
                beg = __ldg(a.rowptr + v);
                end = __ldg(a.rowptr + v + 1);
                nt = __ldg(a.node_thr + v);
            }
            const bool skip_list = lane < nb && tim_skip_rule(nt, end - beg);
            // the frontier's nodes are distinct, so these sums stay below m < 2^32
            const unsigned long long dw = __reduce_add_sync(0xffffffffu, (unsigned)(end - beg));
            // the budget counts in-edges that take a coin; a skipped list counts as at
            // most 64
            const unsigned long long dx = __reduce_add_sync(
                0xffffffffu, (unsigned)(skip_list ? min(end - beg, (uint64_t)64) : end - beg));
            if (work + dx > budget) {
                // too heavy for this tier: list the set for the next one
                if (wt == 0 && lane == 0) ctl[1] |= ST_OVERFLOW;
                break;
            }
            work += dx;
            width += dw;
            // examined in-edges: every in-edge of a list outside the skip rule (the live
            // ones the rule finds are added as they are found)
            const unsigned long long dt =
                __reduce_add_sync(0xffffffffu, (unsigned)(skip_list ? 0ull : end - beg));
            if (wt == 0 && lane == 0) exam += dt;
            // 32-bit in-CSR positions (m < 2^32)
            const uint32_t b32 = (uint32_t)beg, e32 = (uint32_t)end;
            const uint32_t ng = e32 > b32 ? ((e32 - 1) >> 2) - (b32 >> 2) + 1 : 0u;
            const bool big = ng >= BIG_GROUPS;
            int flags = 0;
            // hubs first: the whole team strides over one in-list at a time, two groups in
            // flight per lane; only the in-list's first and last group need a range mask
            uint32_t bigmask = __ballot_sync(0xffffffffu, big);
            int hubi = 0;  // hubs under the skip rule go to the team's warps in turn
            while (bigmask && !(flags & 3)) {
                const int b = __ffs(bigmask) - 1;
                bigmask &= bigmask - 1;
                const uint32_t bb = __shfl_sync(0xffffffffu, b32, b);
                const uint32_t be = __shfl_sync(0xffffffffu, e32, b);
                const unsigned long long bt = __shfl_sync(0xffffffffu, nt, b);
                const bool shared = (bt >> 32) != 0;
                const uint32_t t = (uint32_t)bt;
                if (shared && t == 0u) continue;
                if (tim_skip_rule(bt, be - bb)) {
                    // geometric skipping: one step per live in-edge, by one warp of the team
                    if (hubi++ % T == wt) {
                        int f = 0;
                        skip_live_warp(s0, s1, K, bb, be - bb, skip_table(a.qtab, bt), lane,
                                       [&](uint32_t j) {
                            if (lane == 0) {
                                live++;
                                exam++;
                                const uint32_t u = __ldg(a.src + j);
                                const int r = set_insert<C>(hash, queue, slot, ctl, u);
                                if (r == INS_FULL) {
                                    f |= 1;
                                } else if (r == INS_NEW && cover && marked(a.seed_mark, u)) {
                                    atomicOr(&ctl[1], ST_COVERED);
                                    f |= 2;
                                }
                            }
                            f = __shfl_sync(0xffffffffu, f, 0);
                            return (f & 3) != 0;
                        });
                        flags |= f;
                    }
                    continue;
                }
                const uint32_t gfirst = bb >> 2, glast = (be - 1) >> 2;
                for (uint32_t gb = gfirst + (uint32_t)(wt * 32); gb <= glast; gb += 64u * T) {
                    const uint32_t g0 = gb + lane, g1 = gb + 32u * T + lane;
                    const bool v0 = g0 <= glast, v1 = g1 <= glast;
                    uint32_t m0 = 0, m1 = 0;
                    if (shared) {
                        if (t == 0xFFFFFFFFu) {
                            m0 = v0 ? 0xFu : 0u;
                            m1 = v1 ? 0xFu : 0u;
                        } else {
                            if (v0) m0 = live_mask_shared(philox4x32_10(s0, s1, g0, TIM_TAG_IC, K), t);
                            if (v1) m1 = live_mask_shared(philox4x32_10(s0, s1, g1, TIM_TAG_IC, K), t);
                        }
                    } else {
                        if (v0) {
                            const uint4 x = philox4x32_10(s0, s1, g0, TIM_TAG_IC, K);
                            m0 = live_mask(x, __ldg(thr4 + g0));
                        }
                        if (v1) {
                            const uint4 x = philox4x32_10(s0, s1, g1, TIM_TAG_IC, K);
                            m1 = live_mask(x, __ldg(thr4 + g1));
                        }
                    }
                    if (__any_sync(0xffffffffu, (m0 | m1) != 0u)) {
                        if (m0 && (g0 == gfirst || g0 == glast)) m0 &= range_mask(g0, bb, be);
                        if (m1 && (g1 == gfirst || g1 == glast)) m1 &= range_mask(g1, bb, be);
                        live += __popc(m0) + __popc(m1);
                        if (m0) flags |= follow_live<C, A>(a, g0, m0, hash, queue, slot, ctl);
                        if (m1) flags |= follow_live<C, A>(a, g1, m1, hash, queue, slot, ctl);
                        if (__any_sync(0xffffffffu, flags & 3)) break;
                    }
                }
                flags = __reduce_or_sync(0xffffffffu, flags);
            }
            // the rest, flattened over the lanes: lane -> (owner node, group)
            const uint32_t ngs = big ? 0u : ng;  // lists under the skip rule are big
            uint32_t incl = ngs;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - ngs;
            for (uint32_t base = wt * 32; base < total && !(flags & 3); base += 32 * T) {
                const uint32_t t = base + lane;
                int own = 0;  // number of lanes whose inclusive count is <= t
#pragma unroll
                for (int sft = 16; sft > 0; sft >>= 1) {
                    const uint32_t ic = __shfl_sync(0xffffffffu, incl, own + sft - 1);
                    if (ic <= t) own += sft;
                }
                const uint32_t o_beg = __shfl_sync(0xffffffffu, b32, own);
                const uint32_t o_end = __shfl_sync(0xffffffffu, e32, own);
                const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, own);
                const unsigned long long o_nt = __shfl_sync(0xffffffffu, nt, own);
                uint32_t m = 0, g = 0;
                if (t < total) {
                    g = (o_beg >> 2) + (t - o_excl);
                    const uint32_t ot = (uint32_t)o_nt;
                    if (!(o_nt >> 32))
                        m = live_mask(philox4x32_10(s0, s1, g, TIM_TAG_IC, K), __ldg(thr4 + g));
                    else if (ot == 0xFFFFFFFFu)
                        m = 0xFu;
                    else if (ot != 0u)
                        m = live_mask_shared(philox4x32_10(s0, s1, g, TIM_TAG_IC, K), ot);
                    if (m) m &= range_mask(g, o_beg, o_end);
                }
                if (__any_sync(0xffffffffu, m != 0u)) {
                    live += __popc(m);
                    if (m) flags |= follow_live<C, A>(a, g, m, hash, queue, slot, ctl);
                    flags = __reduce_or_sync(0xffffffffu, flags);
                }
            }
            team_sync<T>(team);
            head += nb;
        }
        if (out) {  // meaningful when the set stopped: the batch to (re)process
            out->head = bh;
            out->width = bw;
        }
    } else if constexpr (MODEL == TIM_TRIG) {
        // a general triggering model (Section 4.2): every reached node picks one option
        // with the LT draw (the first whose cumulative threshold exceeds it) and the
        // option's in-edges are followed, flattened over the lanes
        const uint32_t s0 = (uint32_t)sid, s1 = (uint32_t)(sid >> 32);
        int head = 0;
        for (int guard = 0; guard < C::Q + 1; guard++) {
            int tail, stat;
            if (T == 1) {
                tail = __shfl_sync(0xffffffffu, vctl[0], 0);
                stat = __shfl_sync(0xffffffffu, vctl[1], 0);
            } else {
                tail = vctl[0];
                stat = vctl[1];
                team_sync<T>(team);
            }
            if (stat || head >= tail) break;
            const int nb = min(32, tail - head);
            uint64_t beg = 0, end = 0, ob = 0, oe = 0;
            if (lane < nb) {
                const uint32_t v = queue[head + lane];
                beg = __ldg(a.rowptr + v);
                end = __ldg(a.rowptr + v + 1);
                const uint64_t o0 = __ldg(a.node_opt + v), o1 = __ldg(a.node_opt + v + 1);
                if (o1 > o0) {
                    const uint32_t x = philox4x32_10(s0, s1, v, TIM_TAG_LT, K).x;
                    const uint64_t o = lane_lt_search(a.opt_cum, o0, o1, x);
                    if (o < o1) {
                        ob = __ldg(a.opt_off + o);
                        oe = __ldg(a.opt_off + o + 1);
                    }
                }
            }
            width += __reduce_add_sync(0xffffffffu, (unsigned)(end - beg));
            const uint32_t ne = (uint32_t)(oe - ob);
            uint32_t incl = ne;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - ne;
            if (wt == 0 && lane == 0) exam += total;
            int flags = 0;
            for (uint32_t base = wt * 32; base < total && !(flags & 3); base += 32 * T) {
                const uint32_t t = base + lane;
                int own = 0;  // number of lanes whose inclusive count is <= t
#pragma unroll
                for (int sft = 16; sft > 0; sft >>= 1) {
                    const uint32_t ic = __shfl_sync(0xffffffffu, incl, own + sft - 1);
                    if (ic <= t) own += sft;
                }
                const uint64_t o_b = __shfl_sync(0xffffffffu, ob, own);
                const uint32_t o_x = __shfl_sync(0xffffffffu, excl, own);
                if (t < total) {
                    live++;
                    const uint32_t u = __ldg(a.src + __ldg(a.opt_pos + o_b + (t - o_x)));
                    const int r = set_insert<C>(hash, queue, slot, ctl, u);
                    if (r == INS_FULL) {
                        flags |= 1;
                    } else if (r == INS_NEW && cover && marked(a.seed_mark, u)) {
                        atomicOr(&ctl[1], ST_COVERED);
                        flags |= 2;
                    }
                }
                flags = __reduce_or_sync(0xffffffffu, flags);
            }
            team_sync<T>(team);
            head += nb;
        }
    } else if (wt == 0) {
        // an LT set is a chain: one warp walks it, the team's other warps wait
        uint32_t v = root;
        for (int guard = 0; guard < C::Q + 1; guard++) {
            if (__shfl_sync(0xffffffffu, vctl[1], 0)) break;
            const uint64_t beg = __ldg(a.rowptr + v), end = __ldg(a.rowptr + v + 1);
            width += end - beg;
            if (beg == end) break;
            const uint32_t x =
                philox4x32_10((uint32_t)sid, (uint32_t)(sid >> 32), v, TIM_TAG_LT, K).x;
            const unsigned long long nt = __ldg(a.node_thr + v);
            const uint64_t j = (nt >> 32) ? lt_uniform_pick(nt, beg, end, x)
                                          : warp_lt_search(a.thr, beg, end, x, lane);
            if (j >= end) break;
            const uint32_t u = __ldg(a.src + j);
            int fresh = 0;
            if (lane == 0) {
                live++;
                fresh = set_insert<C>(hash, queue, slot, ctl, u) == INS_NEW ? 1 : 0;
                if (fresh && cover && marked(a.seed_mark, u)) atomicOr(&ctl[1], ST_COVERED);
            }
            fresh = __shfl_sync(0xffffffffu, fresh, 0);
            __syncwarp();
            if (!fresh) break;
            v = u;
        }
    }
    team_sync<T>(team);
    *width_out = width;
    *live_out += live;
    *exam_out += exam;
    return T == 1 ? __shfl_sync(0xffffffffu, vctl[1], 0) : vctl[1];
}

// kappa (Eq. 6) of the sets whose widths lanes 0 .. cnt-1 hold, one set per lane: the
// FP64 operations of 32 sets share one warp instruction each (GB300's FP64 rate is a
// small fraction of its FP32 rate, and one set per warp instruction cost several ms per
// run of Algorithm 2 on the largest graphs). Each lane adds into its own 128-bit sum.
__device__ __forceinline__ void kappa_lanes(unsigned long long w, unsigned cnt, int lane,
                                            unsigned long long m, int k, unsigned long long& lo,
                                            unsigned long long& hi) {
    if ((unsigned)lane < cnt) {
        const unsigned long long kf = kappa_fixed(kappa_fp64(w, m, k));
        lo += kf;
        if (lo < kf) hi++;
    }
}

// TIER 1: teams of one warp, storage in shared memory, every set index of [0, count),
// in-edge budget (IC); listed sets go to list1. TIER 2: teams of T warps, storage in
// the global arena, the sets of list1, no budget; listed sets go to list2.
// Tier 1 is bound by integer arithmetic (coins), tier 2 by latency: tier 2 trades
// registers for resident warps.
template <int MODEL, class C, int TIER, int T>
__global__ void __launch_bounds__(WARPS * 32, TIER == 1 ? 4 : 6) rr_team_kernel(SampleArgs a) {
    extern __shared__ uint32_t smem[];
    __shared__ unsigned long long s_claim[WARPS];
    __shared__ int s_ctl[WARPS][4];  // tier 2: a team's tail and status (shared atomics)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int wt = wid % T, team = wid / T;
    const int tl = wt * 32 + lane;  // thread index inside the team
    uint32_t* hash;
    if (TIER == 1) {
        hash = smem + team * C::WORDS;
        for (int i = tl; i < C::H; i += 32 * T) hash[i] = EMPTY;
    } else {
        // the arena's hash regions are all EMPTY between sets
        const uint64_t slot_id = (uint64_t)blockIdx.x * (WARPS / T) + team;
        hash = a.arena + slot_id * C::WORDS;
    }
    team_sync<T>(team);
    uint32_t* queue = hash + C::H;
    uint16_t* slot = reinterpret_cast<uint16_t*>(queue + C::Q);
    int* ctl = TIER == 1 ? reinterpret_cast<int*>(queue + C::Q + C::Q / 2) : s_ctl[team];
    const unsigned long long budget =
        MODEL != TIM_IC ? ~0ull : TIER == 1 ? a.width_budget : a.width_budget2;
    unsigned long long* counter = TIER == 1 ? &a.ds->next_set : &a.ds->next2;
    const uint64_t items =
        TIER == 1 ? a.count : (uint64_t)min(((volatile unsigned*)&a.ds->cnt1)[0], a.list_cap);
    uint32_t* out_list = TIER == 1 ? a.list1 : a.list2;
    unsigned* out_cnt = TIER == 1 ? &a.ds->cnt1 : &a.ds->cnt2;
    unsigned long long k_lo = 0, k_hi = 0, wsum = 0, cov = 0, live = 0, memb = 0, exam = 0;
    const bool emit = a.flags & SAMPLE_EMIT, kap = a.flags & SAMPLE_KAPPA;
    const bool leader = wt == 0 && lane == 0;
    // widths of completed sets waiting for their kappa (warp 0 of the team; lane i holds
    // the i-th, kcnt is the same on every lane)
    unsigned long long kw = 0;
    unsigned kcnt = 0;
    for (;;) {
        unsigned long long i0 = 0;
        if (leader) i0 = atomicAdd(counter, (unsigned long long)a.chunk);
        if (T == 1) {
            i0 = __shfl_sync(0xffffffffu, i0, 0);
        } else {
            if (leader) s_claim[team] = i0;
            team_sync<T>(team);
            i0 = s_claim[team];
            team_sync<T>(team);
        }
        if (i0 >= items) break;
        const unsigned long long i1 = min(i0 + (unsigned long long)a.chunk, (unsigned long long)items);
        for (unsigned long long it = i0; it < i1; it++) {
            const uint64_t j = TIER == 1 ? it : a.list1[it];
            unsigned long long width;
            // IC: pass 2 goes on with a set where pass 1 stopped, from the state pass 1
            // handed over (its queue, the batch to redo, the width before it)
            constexpr bool HAND = MODEL == TIM_IC;
            Resume rin{0, 0ull}, rout{0, 0ull};
            bool resumed = false;
            if (HAND && TIER == 2 && a.hand && it < a.hcap) {
                const uint32_t* hs = a.hand + it * (uint64_t)a.hw;
                const uint32_t t0 = hs[0];
                if (t0 > 0 && t0 <= (uint32_t)C::Q) {
                    if (leader) {
                        ctl[0] = (int)t0;
                        ctl[1] = 0;
                    }
                    team_sync<T>(team);
                    for (uint32_t i = tl; i < t0; i += 32 * T) {
                        const uint32_t u = hs[4 + i];
                        queue[i] = u;
                        // the members are distinct: each takes the first empty slot it finds
                        uint32_t h = (u * 0x9E3779B1u) >> (32 - C::LOG2H);
                        for (int probe = 0; probe < C::H; probe++) {
                            if (atomicCAS(&hash[h], EMPTY, u) == EMPTY) break;
                            h = (h + 1) & (C::H - 1);
                        }
                        slot[i] = (uint16_t)h;
                        // a member in the seed set found in the batch that overflowed pass
                        // 1's queue: the set is covered (as a fresh expansion would find)
                        if ((a.flags & SAMPLE_COVER) && marked(a.seed_mark, u))
                            atomicOr(&ctl[1], ST_COVERED);
                    }
                    rin.head = (int)min(hs[1], t0);
                    rin.width = (unsigned long long)hs[2] | ((unsigned long long)hs[3] << 32);
                    resumed = true;
                }
                team_sync<T>(team);
            }
            const int st = team_rr<MODEL, C, T, SampleArgs>(
                a, a.K, a.sid0 + j, hash, queue, slot, ctl, budget, wt, team, &width, &live,
                &exam, resumed ? &rin : nullptr,
                (HAND && ((TIER == 1 && a.hand) || (TIER == 2 && a.hand2))) ? &rout : nullptr);
            const int tail = min(T == 1 ? __shfl_sync(0xffffffffu, ((volatile int*)ctl)[0], 0)
                                        : ((volatile int*)ctl)[0],
                                 C::Q);
            team_sync<T>(team);
            if (st & ST_OVERFLOW) {
                unsigned idx = 0;
                if (leader) {
                    idx = atomicAdd(out_cnt, 1u);
                    if (idx < a.list_cap)
                        out_list[idx] = (uint32_t)j;
                    else
                        atomicOr(&a.ds->err, TIM_DEV_ERR_OVF_LIST);
                }
                if (HAND && TIER == 1 && T == 1 && a.hand) {  // hand the state to pass 2
                    idx = __shfl_sync(0xffffffffu, idx, 0);
                    if (idx < a.hcap) {
                        uint32_t* hs = a.hand + idx * (uint64_t)a.hw;
                        for (int i = lane; i < tail; i += 32) hs[4 + i] = queue[i];
                        if (lane == 0) {
                            hs[0] = (uint32_t)tail;
                            hs[1] = (uint32_t)rout.head;
                            hs[2] = (uint32_t)rout.width;
                            hs[3] = (uint32_t)(rout.width >> 32);
                        }
                    }
                }
                if (HAND && TIER == 2 && a.hand2) {  // hand the state to the heavy pass
                    if (T == 1) {
                        idx = __shfl_sync(0xffffffffu, idx, 0);
                    } else {
                        if (leader) s_claim[team] = idx;
                        team_sync<T>(team);
                        idx = (unsigned)s_claim[team];
                    }
                    if (idx < a.h2cap) {
                        uint32_t* hs = a.hand2 + idx * (uint64_t)a.h2w;
                        for (int i = tl; i < tail; i += 32 * T) hs[4 + i] = queue[i];
                        if (leader) {
                            hs[0] = (uint32_t)tail;
                            hs[1] = (uint32_t)min(rout.head, tail);
                            hs[2] = (uint32_t)rout.width;  // in-degrees of queue[0 .. hs[1])
                            hs[3] = (uint32_t)(rout.width >> 32);
                        }
                    }
                    team_sync<T>(team);
                }
                for (int i = tl; i < C::H; i += 32 * T) hash[i] = EMPTY;
                team_sync<T>(team);
                continue;
            }
            if (leader) {
                wsum += width;
                memb += tail;
                if (st & ST_COVERED) cov++;
            }
            if (kap && wt == 0) {  // width is the same on every lane
                if ((unsigned)lane == kcnt) kw = width;
                if (++kcnt == 32) {
                    kappa_lanes(kw, kcnt, lane, a.m, a.k, k_lo, k_hi);
                    kcnt = 0;
                }
            }
            if (emit) {
                unsigned long long base = 0;
                if (leader) base = atomicAdd(&a.ds->pool_used, (unsigned long long)tail);
                if (T == 1) {
                    base = __shfl_sync(0xffffffffu, base, 0);
                } else {
                    if (leader) s_claim[team] = base;
                    team_sync<T>(team);
                    base = s_claim[team];
                }
                if (base + tail <= a.pool_cap) {
                    for (int i = tl; i < tail; i += 32 * T) {
                        a.pool[base + i] = queue[i];
                        a.pool_sid[base + i] = (uint32_t)j;
                    }
                    if (leader) {
                        a.set_start[j] = base;
                        a.set_len[j] = (uint32_t)tail;
                        a.set_width[j] = width;
                    }
                } else if (leader) {
                    atomicOr(&a.ds->err, TIM_DEV_ERR_POOL);
                }
            }
            for (int i = tl; i < tail; i += 32 * T) hash[slot[i]] = EMPTY;
            team_sync<T>(team);
        }
    }
    live = warp_sum_u64(live);
    if (lane == 0 && live) atomicAdd(&a.ds->live[TIER - 1], live);
    if (lane == 0 && exam) atomicAdd(&a.ds->exam[TIER - 1], exam);
    if (kap && wt == 0) {
        kappa_lanes(kw, kcnt, lane, a.m, a.k, k_lo, k_hi);
        if (k_lo || k_hi) atomic_add_u128(&a.ds->ksum_lo, &a.ds->ksum_hi, k_lo, k_hi);
    }
    if (leader) {
        if (wsum) {
            atomicAdd(&a.ds->wsum, wsum);
            atomicAdd(&a.ds->width[TIER - 1], wsum);
        }
        if (cov) atomicAdd(&a.ds->covered, cov);
        if (memb) atomicAdd(&a.ds->memb[TIER - 1], memb);
    }
}

// ------------------------------------------------- tier 1 for LT: a chain per lane
//
// An LT RR set is a chain (Section 4.2: each node keeps at most one live in-edge), so
// its walk has no parallelism of its own: every thread walks one chain. The members go
// to the thread's column of a global array (member k at k * lanes + thread, so a warp's
// stores are contiguous); a 1024-bit Bloom filter per thread in shared memory screens
// the revisit test, which scans the column only on a filter hit. Chains longer than
// LT_CAP go to tier 2 (list1). Idle lanes claim sets together (one atomic per warp) at
// the top of every step, and finished lanes reserve store space together, so a warp
// keeps all 32 chains moving.
constexpr int LT_THREADS = 128;
constexpr int LT_CAP = 1024;                 // members per chain in this pass
constexpr int LT_BLOOM_WORDS = 32;           // 1024 bits per thread
constexpr size_t LT_SMEM = (size_t)LT_BLOOM_WORDS * LT_THREADS * sizeof(uint32_t);

__device__ __forceinline__ void lt_bloom_bits(uint32_t u, uint32_t& w1, uint32_t& m1, uint32_t& w2,
                                              uint32_t& m2) {
    const uint32_t h = u * 0x9E3779B1u;
    const uint32_t b1 = h >> 22, b2 = (h >> 12) & 1023u;
    w1 = b1 >> 5;
    m1 = 1u << (b1 & 31);
    w2 = b2 >> 5;
    m2 = 1u << (b2 & 31);
}

__device__ __forceinline__ void lane_bloom_add(uint32_t* bloom, uint32_t u) {
    uint32_t w1, m1, w2, m2;
    lt_bloom_bits(u, w1, m1, w2, m2);
    bloom[w1 * LT_THREADS] |= m1;
    bloom[w2 * LT_THREADS] |= m2;
}

__device__ __forceinline__ bool lane_bloom_test(const uint32_t* bloom, uint32_t u) {
    uint32_t w1, m1, w2, m2;
    lt_bloom_bits(u, w1, m1, w2, m2);
    return (bloom[w1 * LT_THREADS] & m1) && (bloom[w2 * LT_THREADS] & m2);
}

// Revisit test of the lanes with hit set: does lane l's column (the warp's columns
// start at wcol; member k of lane l at wcol[k * lanes + l]) hold u among its first len
// members? All lanes scan each such column together. Warp-collective.
__device__ __forceinline__ bool lane_cols_contain(const uint32_t* wcol, uint64_t lanes, int lane,
                                                  bool hit, uint32_t u, int len) {
    bool seen = false;
    for (unsigned hm = __ballot_sync(0xffffffffu, hit); hm; hm &= hm - 1) {
        const int l = __ffs(hm) - 1;
        const uint32_t ul = __shfl_sync(0xffffffffu, u, l);
        const int ll = __shfl_sync(0xffffffffu, len, l);
        bool f = false;
        for (int k = lane; k < ll; k += 32) f |= wcol[(uint64_t)k * lanes + l] == ul;
        f = __any_sync(0xffffffffu, f);
        if (lane == l) seen = f;
    }
    return seen;
}

__global__ void __launch_bounds__(LT_THREADS) rr_lt_lane_kernel(SampleArgs a) {
    extern __shared__ uint32_t bloom_all[];
    const int tid = threadIdx.x, lane = tid & 31;
    uint32_t* bloom = bloom_all + tid;  // word w at bloom[w * LT_THREADS]
    for (int w = 0; w < LT_BLOOM_WORDS; w++) bloom[w * LT_THREADS] = 0u;
    const uint64_t lanes = (uint64_t)gridDim.x * LT_THREADS;
    // member k of lane l of this warp's columns: wcol[k * lanes + l]
    uint32_t* wcol = a.lt_col + (uint64_t)blockIdx.x * LT_THREADS + (tid & ~31);
    uint32_t* col = wcol + lane;
    const bool emit = a.flags & SAMPLE_EMIT, kap = a.flags & SAMPLE_KAPPA,
               cover = a.flags & SAMPLE_COVER;
    unsigned long long k_lo = 0, k_hi = 0, wsum = 0, cov = 0, live = 0, memb = 0;
    bool has = false, exhausted = false;
    uint64_t j = 0, sid = 0;
    uint32_t v = 0;
    int len = 0, status = 0;
    unsigned long long width = 0;
    // bounded: every step either advances a chain (at most LT_CAP steps each) or
    // finishes it, and the lanes take at most count sets between them
    const uint64_t steps = (a.count + 1) * (uint64_t)(LT_CAP + 2) + 64;
    for (uint64_t guard = 0; guard < steps; guard++) {
        // idle lanes claim the next sets, one atomic for the warp
        const bool need = !has && !exhausted;
        const unsigned nm = __ballot_sync(0xffffffffu, need);
        if (nm) {
            const int leader = __ffs(nm) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(&a.ds->next_set, (unsigned long long)__popc(nm));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (need) {
                const unsigned long long mine = base + __popc(nm & ((1u << lane) - 1u));
                if (mine < a.count) {
                    j = mine;
                    sid = a.sid0 + j;
                    v = rr_root(sid, a.n, a.K);
                    col[0] = v;
                    len = 1;
                    width = 0;
                    uint32_t w1, m1, w2, m2;
                    lt_bloom_bits(v, w1, m1, w2, m2);
                    bloom[w1 * LT_THREADS] |= m1;
                    bloom[w2 * LT_THREADS] |= m2;
                    status = (cover && marked(a.seed_mark, v)) ? ST_COVERED : 0;
                    has = true;
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, has)) break;
        // one step of every lane's chain: the next member u, if any
        bool fin = false, cand = false;
        uint32_t u = 0;
        if (has) {
            if (status) {
                fin = true;
            } else {
                const uint64_t beg = __ldg(a.rowptr + v), end = __ldg(a.rowptr + v + 1);
                const unsigned long long nt = __ldg(a.node_thr + v);
                width += end - beg;
                uint64_t jj = end;
                if (beg < end) {
                    const uint32_t x =
                        philox4x32_10((uint32_t)sid, (uint32_t)(sid >> 32), v, TIM_TAG_LT, a.K).x;
                    jj = (nt >> 32) ? lt_uniform_pick(nt, beg, end, x)
                                    : lane_lt_search(a.thr, beg, end, x);
                }
                if (jj >= end) {
                    fin = true;
                } else {
                    u = __ldg(a.src + jj);
                    live++;
                    cand = true;
                }
            }
        }
        // revisit test: the filter first; on a hit the whole warp scans that column
        uint32_t w1 = 0, m1 = 0, w2 = 0, m2 = 0;
        bool hit = false;
        if (cand) {
            lt_bloom_bits(u, w1, m1, w2, m2);
            hit = (bloom[w1 * LT_THREADS] & m1) && (bloom[w2 * LT_THREADS] & m2);
        }
        bool seen = false;
        for (unsigned hm = __ballot_sync(0xffffffffu, hit); hm; hm &= hm - 1) {
            const int l = __ffs(hm) - 1;
            const uint32_t ul = __shfl_sync(0xffffffffu, u, l);
            const int ll = __shfl_sync(0xffffffffu, len, l);
            bool f = false;
            for (int k = lane; k < ll; k += 32) f |= wcol[(uint64_t)k * lanes + l] == ul;
            f = __any_sync(0xffffffffu, f);
            if (lane == l) seen = f;
        }
        bool ovf = false;
        if (cand) {
            if (seen) {
                fin = true;
            } else if (len == LT_CAP) {
                fin = ovf = true;
            } else {
                col[(uint64_t)len * lanes] = u;
                len++;
                bloom[w1 * LT_THREADS] |= m1;
                bloom[w2 * LT_THREADS] |= m2;
                if (cover && marked(a.seed_mark, u)) status |= ST_COVERED;
                v = u;
            }
        }
        if (fin && ovf) {
            const unsigned idx = atomicAdd(&a.ds->cnt1, 1u);
            if (idx < a.list_cap)
                a.list1[idx] = (uint32_t)j;
            else
                atomicOr(&a.ds->err, TIM_DEV_ERR_OVF_LIST);
        } else if (fin) {
            wsum += width;
            memb += len;
            if (status & ST_COVERED) cov++;
            if (kap) {
                const unsigned long long kf = kappa_fixed(kappa_fp64(width, a.m, a.k));
                k_lo += kf;
                if (k_lo < kf) k_hi++;
            }
        }
        // finished chains reserve their store space together and the warp copies each
        // one's column with all its lanes
        const bool put = emit && fin && !ovf;
        const unsigned pm = __ballot_sync(0xffffffffu, put);
        if (pm) {
            unsigned incl = put ? (unsigned)len : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&a.ds->pool_used, (unsigned long long)total);
            base = __shfl_sync(0xffffffffu, base, 0);
            const unsigned long long st = base + incl - (put ? (unsigned)len : 0u);
            const bool fits = base + total <= a.pool_cap;
            if (put) {
                if (fits) {
                    a.set_start[j] = st;
                    a.set_len[j] = (uint32_t)len;
                    a.set_width[j] = width;
                } else {
                    atomicOr(&a.ds->err, TIM_DEV_ERR_POOL);
                }
            }
            if (fits) {
                for (unsigned m = pm; m; m &= m - 1) {
                    const int l = __ffs(m) - 1;
                    const unsigned long long sl = __shfl_sync(0xffffffffu, st, l);
                    const int ll = __shfl_sync(0xffffffffu, len, l);
                    const uint32_t jl = (uint32_t)__shfl_sync(0xffffffffu, j, l);
                    for (int k = lane; k < ll; k += 32) {
                        a.pool[sl + k] = wcol[(uint64_t)k * lanes + l];
                        a.pool_sid[sl + k] = jl;
                    }
                }
            }
        }
        if (fin) {
            for (int w = 0; w < LT_BLOOM_WORDS; w++) bloom[w * LT_THREADS] = 0u;
            has = false;
        }
    }
    live = warp_sum_u64(live);
    wsum = warp_sum_u64(wsum);
    memb = warp_sum_u64(memb);
    cov = warp_sum_u64(cov);
    if (lane == 0) {
        if (live) atomicAdd(&a.ds->live[0], live);
        if (wsum) {
            atomicAdd(&a.ds->wsum, wsum);
            atomicAdd(&a.ds->width[0], wsum);
        }
        if (memb) atomicAdd(&a.ds->memb[0], memb);
        if (cov) atomicAdd(&a.ds->covered, cov);
    }
    if (kap && (k_lo || k_hi)) atomic_add_u128(&a.ds->ksum_lo, &a.ds->ksum_hi, k_lo, k_hi);
}

// ---------------------------------------------------------- tier 3 (LT chains)

// One CTA per listed set; warp 0 walks the chain with a visited bitmap and a queue of
// up to n members in global memory.
__global__ void __launch_bounds__(BIG_THREADS) rr_lt_chain_kernel(SampleArgs a) {
    __shared__ unsigned long long s_j;
    __shared__ int s_tail, s_status;
    __shared__ unsigned long long s_width, s_base;
    const int tid = threadIdx.x, lane = tid & 31;
    uint32_t* bitmap = a.big_bitmap + (uint64_t)blockIdx.x * a.big_words;
    uint32_t* queue = a.big_queue + (uint64_t)blockIdx.x * a.n;
    const bool emit = a.flags & SAMPLE_EMIT, kap = a.flags & SAMPLE_KAPPA,
               cover = a.flags & SAMPLE_COVER;
    unsigned long long k_lo = 0, k_hi = 0, wsum = 0, cov = 0, live = 0, memb = 0;
    const unsigned nlist = min(((volatile unsigned*)&a.ds->cnt2)[0], a.list_cap);
    for (;;) {
        if (tid == 0) s_j = atomicAdd(&a.ds->next3, 1ull);
        __syncthreads();
        unsigned long long idx = s_j;
        if (idx >= nlist) break;
        uint64_t j = a.list2[idx];
        uint64_t sid = a.sid0 + j;
        uint32_t root = rr_root(sid, a.n, a.K);
        if (tid == 0) {
            atomicOr(&bitmap[root >> 5], 1u << (root & 31));
            queue[0] = root;
            s_tail = 1;
            s_status = (cover && marked(a.seed_mark, root)) ? ST_COVERED : 0;
            s_width = 0;
        }
        __syncthreads();
        if (tid < 32) {
            uint32_t v = root;
            unsigned long long width = 0;
            int tail = 1;
            int status = s_status;
            for (uint64_t guard = 0; guard <= a.n && !status; guard++) {
                uint64_t beg = __ldg(a.rowptr + v), end = __ldg(a.rowptr + v + 1);
                width += end - beg;
                if (beg == end) break;
                uint32_t x = draw(a, sid, v, TIM_TAG_LT).x;
                const unsigned long long nt = __ldg(a.node_thr + v);
                uint64_t jj = (nt >> 32) ? lt_uniform_pick(nt, beg, end, x)
                                         : warp_lt_search(a.thr, beg, end, x, lane);
                if (jj >= end) break;
                uint32_t u = __ldg(a.src + jj);
                int fresh = 0;
                if (lane == 0) {
                    live++;
                    uint32_t bit = 1u << (u & 31);
                    uint32_t old = atomicOr(&bitmap[u >> 5], bit);
                    fresh = !(old & bit);
                    if (fresh) queue[tail] = u;
                }
                fresh = __shfl_sync(0xffffffffu, fresh, 0);
                if (!fresh) break;
                tail++;
                if (cover && marked(a.seed_mark, u)) status |= ST_COVERED;
                v = u;
            }
            __syncwarp();
            if (lane == 0) {
                s_width = width;
                s_tail = tail;
                s_status = status;
            }
        }
        __syncthreads();
        const int tail = s_tail;
        const unsigned long long width = s_width;
        if (tid == 0) {
            wsum += width;
            memb += tail;
            if (s_status & ST_COVERED) cov++;
            if (kap) {
                unsigned long long kf = kappa_fixed(kappa_fp64(width, a.m, a.k));
                k_lo += kf;
                if (k_lo < kf) k_hi++;
            }
            if (emit) s_base = atomicAdd(&a.ds->pool_used, (unsigned long long)tail);
        }
        __syncthreads();
        if (emit) {
            unsigned long long base = s_base;
            if (base + tail <= a.pool_cap) {
                for (int i = tid; i < tail; i += BIG_THREADS) {
                    a.pool[base + i] = queue[i];
                    a.pool_sid[base + i] = (uint32_t)j;
                }
                if (tid == 0) {
                    a.set_start[j] = base;
                    a.set_len[j] = (uint32_t)tail;
                    a.set_width[j] = width;
                }
            } else if (tid == 0) {
                atomicOr(&a.ds->err, TIM_DEV_ERR_POOL);
            }
        }
        for (int i = tid; i < tail; i += BIG_THREADS) {
            uint32_t u = queue[i];
            atomicAnd(&bitmap[u >> 5], ~(1u << (u & 31)));
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (kap && (k_lo || k_hi)) atomic_add_u128(&a.ds->ksum_lo, &a.ds->ksum_hi, k_lo, k_hi);
        if (wsum) {
            atomicAdd(&a.ds->wsum, wsum);
            atomicAdd(&a.ds->width[2], wsum);
        }
        if (cov) atomicAdd(&a.ds->covered, cov);
        if (memb) atomicAdd(&a.ds->memb[2], memb);
        if (live) atomicAdd(&a.ds->live[2], live);
    }
}

// ------------------------------------------------- tier 3 (triggering model)

// One CTA per listed set, level-synchronous: the warps claim 32 queued nodes of the
// current level at a time, each lane draws its node's option, and the options' in-edges
// are flattened over the lanes; a new member sets its bit in the slot's visited bitmap
// (n bits) and takes the next entry of the slot's queue (n entries). A level ends when
// every warp has drained it; the set ends at an empty level (or, COVER, at the first
// member in the seed set).
__global__ void __launch_bounds__(BIG_THREADS) rr_trig_big_kernel(SampleArgs a) {
    __shared__ unsigned long long s_j, s_base;
    __shared__ unsigned long long s_width[BIG_THREADS / 32];
    __shared__ unsigned s_head, s_tail;
    __shared__ int s_status;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint32_t* bitmap = a.big_bitmap + (uint64_t)blockIdx.x * a.big_words;
    uint32_t* queue = a.big_queue + (uint64_t)blockIdx.x * a.n;
    const bool emit = a.flags & SAMPLE_EMIT, kap = a.flags & SAMPLE_KAPPA,
               cover = a.flags & SAMPLE_COVER;
    volatile int* vstatus = &s_status;
    unsigned long long k_lo = 0, k_hi = 0, wsum = 0, cov = 0, live = 0, memb = 0;
    const unsigned nlist = min(((volatile unsigned*)&a.ds->cnt2)[0], a.list_cap);
    for (;;) {
        if (tid == 0) s_j = atomicAdd(&a.ds->next3, 1ull);
        __syncthreads();
        const unsigned long long idx = s_j;
        if (idx >= nlist) break;
        const uint64_t j = a.list2[idx];
        const uint64_t sid = a.sid0 + j;
        const uint32_t root = rr_root(sid, a.n, a.K);
        if (tid == 0) {
            atomicOr(&bitmap[root >> 5], 1u << (root & 31));
            queue[0] = root;
            s_tail = 1;
            s_head = 0;
            s_status = (cover && marked(a.seed_mark, root)) ? ST_COVERED : 0;
        }
        __syncthreads();
        unsigned long long width = 0;
        unsigned lvl_end = 1;
        // at most n levels: every level but the last adds a member
        for (uint64_t level = 0; level <= a.n; level++) {
            for (;;) {
                unsigned h0 = 0;
                if (lane == 0) h0 = atomicAdd(&s_head, 32u);
                h0 = __shfl_sync(0xffffffffu, h0, 0);
                if (h0 >= lvl_end || *vstatus) break;
                const unsigned nb = min(32u, lvl_end - h0);
                uint64_t beg = 0, end = 0, ob = 0, oe = 0;
                if (lane < nb) {
                    const uint32_t v = queue[h0 + lane];
                    beg = __ldg(a.rowptr + v);
                    end = __ldg(a.rowptr + v + 1);
                    const uint64_t o0 = __ldg(a.node_opt + v), o1 = __ldg(a.node_opt + v + 1);
                    if (o1 > o0) {
                        const uint32_t x = draw(a, sid, v, TIM_TAG_LT).x;
                        const uint64_t o = lane_lt_search(a.opt_cum, o0, o1, x);
                        if (o < o1) {
                            ob = __ldg(a.opt_off + o);
                            oe = __ldg(a.opt_off + o + 1);
                        }
                    }
                }
                width += __reduce_add_sync(0xffffffffu, (unsigned)(end - beg));
                const uint32_t ne = (uint32_t)(oe - ob);
                uint32_t incl = ne;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
                const uint32_t excl = incl - ne;
                for (uint32_t base = 0; base < total; base += 32) {
                    const uint32_t t = base + lane;
                    int own = 0;
#pragma unroll
                    for (int sft = 16; sft > 0; sft >>= 1) {
                        const uint32_t ic = __shfl_sync(0xffffffffu, incl, own + sft - 1);
                        if (ic <= t) own += sft;
                    }
                    const uint64_t o_b = __shfl_sync(0xffffffffu, ob, own);
                    const uint32_t o_x = __shfl_sync(0xffffffffu, excl, own);
                    if (t < total) {
                        live++;
                        const uint32_t u = __ldg(a.src + __ldg(a.opt_pos + o_b + (t - o_x)));
                        const uint32_t bit = 1u << (u & 31);
                        if (!(atomicOr(&bitmap[u >> 5], bit) & bit)) {
                            queue[atomicAdd(&s_tail, 1u)] = u;
                            if (cover && marked(a.seed_mark, u)) atomicOr(&s_status, ST_COVERED);
                        }
                    }
                }
            }
            __syncthreads();
            const unsigned next_end = s_tail;
            const bool done = s_status || next_end == lvl_end;
            __syncthreads();  // every thread has read s_tail and s_status
            if (done) break;
            if (tid == 0) s_head = lvl_end;
            lvl_end = next_end;
            __syncthreads();
        }
        if (lane == 0) s_width[wid] = width;
        __syncthreads();
        const unsigned tail = s_tail;
        if (tid == 0) {
            width = 0;
            for (int w = 0; w < BIG_THREADS / 32; w++) width += s_width[w];
            s_width[0] = width;
            wsum += width;
            memb += tail;
            if (s_status & ST_COVERED) cov++;
            if (kap) {
                const unsigned long long kf = kappa_fixed(kappa_fp64(width, a.m, a.k));
                k_lo += kf;
                if (k_lo < kf) k_hi++;
            }
            if (emit) s_base = atomicAdd(&a.ds->pool_used, (unsigned long long)tail);
        }
        __syncthreads();
        if (emit) {
            const unsigned long long base = s_base;
            if (base + tail <= a.pool_cap) {
                for (unsigned i = tid; i < tail; i += BIG_THREADS) {
                    a.pool[base + i] = queue[i];
                    a.pool_sid[base + i] = (uint32_t)j;
                }
                if (tid == 0) {
                    a.set_start[j] = base;
                    a.set_len[j] = tail;
                    a.set_width[j] = s_width[0];
                }
            } else if (tid == 0) {
                atomicOr(&a.ds->err, TIM_DEV_ERR_POOL);
            }
        }
        for (unsigned i = tid; i < tail; i += BIG_THREADS) {
            const uint32_t u = queue[i];
            atomicAnd(&bitmap[u >> 5], ~(1u << (u & 31)));
        }
        __syncthreads();
    }
    live = warp_sum_u64(live);
    if (lane == 0 && live) atomicAdd(&a.ds->live[2], live);
    if (tid == 0) {
        if (kap && (k_lo || k_hi)) atomic_add_u128(&a.ds->ksum_lo, &a.ds->ksum_hi, k_lo, k_hi);
        if (wsum) {
            atomicAdd(&a.ds->wsum, wsum);
            atomicAdd(&a.ds->width[2], wsum);
        }
        if (cov) atomicAdd(&a.ds->covered, cov);
        if (memb) atomicAdd(&a.ds->memb[2], memb);
    }
}

template <int MODEL, class C, int TIER, int T>
int occupancy(size_t smem) {
    int nb = 0;
    auto k = rr_team_kernel<MODEL, C, TIER, T>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, WARPS * 32, smem) != cudaSuccess ||
        nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

int launch_tier1(tim_ctx* ctx, const SampleArgs& a, unsigned grid, size_t smem) {
    if (ctx->model == TIM_IC) {
        if (ctx->cap1 == 128)
            rr_team_kernel<TIM_IC, Tier1S, 1, 1><<<grid, WARPS * 32, smem, ctx->stream>>>(a);
        else if (ctx->cap1 == 512)
            rr_team_kernel<TIM_IC, Tier1L, 1, 1><<<grid, WARPS * 32, smem, ctx->stream>>>(a);
        else
            rr_team_kernel<TIM_IC, Tier1, 1, 1><<<grid, WARPS * 32, smem, ctx->stream>>>(a);
        LAUNCH_CHECK(ctx, "rr_team_kernel (tier 1)");
    } else if (ctx->model == TIM_TRIG) {
        rr_team_kernel<TIM_TRIG, Tier1, 1, 1><<<grid, WARPS * 32, smem, ctx->stream>>>(a);
        LAUNCH_CHECK(ctx, "rr_team_kernel (tier 1, triggering)");
    } else {
        int nb = 0;
        CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rr_lt_lane_kernel,
                                                                    LT_THREADS, LT_SMEM));
        const unsigned g = (unsigned)(ctx->num_sms * std::max(nb, 1));
        SampleArgs b = a;
        TIM_TRY(tim_ensure(ctx, ctx->lt_col,
                           (size_t)g * LT_THREADS * LT_CAP * sizeof(uint32_t)));
        b.lt_col = (uint32_t*)ctx->lt_col.p;
        rr_lt_lane_kernel<<<g, LT_THREADS, LT_SMEM, ctx->stream>>>(b);
        LAUNCH_CHECK(ctx, "rr_lt_lane_kernel (tier 1)");
    }
    return TIM_OK;
}

int launch_tier2(tim_ctx* ctx, const SampleArgs& a, unsigned grid, int T) {
    if (ctx->model != TIM_IC || T == 1) {
        if (ctx->model == TIM_IC)
            rr_team_kernel<TIM_IC, Tier2, 2, 1><<<grid, WARPS * 32, 0, ctx->stream>>>(a);
        else if (ctx->model == TIM_TRIG)
            rr_team_kernel<TIM_TRIG, Tier2, 2, 1><<<grid, WARPS * 32, 0, ctx->stream>>>(a);
        else
            rr_team_kernel<TIM_LT, Tier2, 2, 1><<<grid, WARPS * 32, 0, ctx->stream>>>(a);
    } else if (T == 2) {
        rr_team_kernel<TIM_IC, Tier2, 2, 2><<<grid, WARPS * 32, 0, ctx->stream>>>(a);
    } else if (T == 4) {
        rr_team_kernel<TIM_IC, Tier2, 2, 4><<<grid, WARPS * 32, 0, ctx->stream>>>(a);
    } else {
        rr_team_kernel<TIM_IC, Tier2, 2, 8><<<grid, WARPS * 32, 0, ctx->stream>>>(a);
    }
    LAUNCH_CHECK(ctx, "rr_team_kernel (tier 2)");
    return TIM_OK;
}


// ------------------------------------------------------- several queries at once

// One query of a multi-query launch (device memory).
struct QueryDesc {
    const uint64_t* rowptr;
    const uint32_t* src;
    const uint32_t* thr;
    const unsigned long long* node_thr;
    const unsigned long long* qtab;
    uint64_t n, m;
    uint64_t sid0, count;
    int model, flags, k, pad;
    const uint32_t* seed_mark;
    uint32_t* pool;
    uint32_t* pool_sid;
    uint64_t pool_cap;
    uint64_t* set_start;
    uint32_t* set_len;
    uint64_t* set_width;
    DevScalars* ds;
    unsigned long long width_budget, width_budget2;
};

struct MultiArgs {
    PhiloxKeys K;
    const QueryDesc* q;
    const unsigned long long* prefix;  // prefix[i] = sets of queries before i; [nq] = total
    int nq;
    int chunk;
    unsigned long long* next;  // [0] tier-1, [1] tier-2 work counters
    unsigned* cnt;             // [0] sets listed for tier 2, [1] for tier 3
    int* err;
    uint2* list1;  // (query, set index)
    uint2* list2;
    uint32_t list_cap;
    uint32_t* arena;
    // IC: pass-1 state handed to pass 2 for list1 position i < hcap (as in SampleArgs)
    uint32_t* hand;
    uint32_t hcap, hw;
};

// What team_rr reads of one query: its graph and flags, plus the launch's keys.
struct QArgs {
    const uint64_t* rowptr;
    const uint32_t* src;
    const uint32_t* thr;
    const unsigned long long* node_thr;
    const unsigned long long* qtab;
    uint64_t n, m;
    int flags, k;
    const uint32_t* seed_mark;
};

constexpr int MAXQ = 256;  // queries per multi-query launch

struct QAcc {
    unsigned long long k_lo, k_hi, wsum, cov, live, memb, exam;
};

template <int TIER>
__device__ __forceinline__ void flush_acc(const QueryDesc* qd, int qi, QAcc& acc, int lane) {
    const unsigned long long lv = warp_sum_u64(acc.live);
    if (qi >= 0 && lane == 0) {
        DevScalars* ds = qd[qi].ds;
        if (acc.k_lo || acc.k_hi) atomic_add_u128(&ds->ksum_lo, &ds->ksum_hi, acc.k_lo, acc.k_hi);
        if (acc.wsum) {
            atomicAdd(&ds->wsum, acc.wsum);
            atomicAdd(&ds->width[TIER - 1], acc.wsum);
        }
        if (acc.cov) atomicAdd(&ds->covered, acc.cov);
        if (lv) atomicAdd(&ds->live[TIER - 1], lv);
        if (acc.memb) atomicAdd(&ds->memb[TIER - 1], acc.memb);
        if (acc.exam) atomicAdd(&ds->exam[TIER - 1], acc.exam);
    }
    acc = QAcc{0, 0, 0, 0, 0, 0, 0};
}

// TIER 1: shared-memory sets of every query (global set index across queries); TIER 2:
// the listed (query, set) pairs with a global arena and teams of T warps.
template <class C, int TIER, int T>
__global__ void __launch_bounds__(WARPS * 32, 3) rr_multi_kernel(MultiArgs ma) {
    extern __shared__ uint32_t smem[];
    __shared__ unsigned long long s_claim[WARPS];
    __shared__ unsigned long long s_prefix[MAXQ + 1];
    __shared__ int s_ctl[WARPS][4];  // tier 2: a team's tail and status (shared atomics)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int wt = wid % T, team = wid / T;
    const int tl = wt * 32 + lane;
    for (int i = threadIdx.x; i <= ma.nq; i += blockDim.x) s_prefix[i] = ma.prefix[i];
    __syncthreads();
    uint32_t* hash;
    if (TIER == 1) {
        hash = smem + team * C::WORDS;
        for (int i = tl; i < C::H; i += 32 * T) hash[i] = EMPTY;
    } else {
        const uint64_t slot_id = (uint64_t)blockIdx.x * (WARPS / T) + team;
        hash = ma.arena + slot_id * C::WORDS;
    }
    team_sync<T>(team);
    uint32_t* queue = hash + C::H;
    uint16_t* slot = reinterpret_cast<uint16_t*>(queue + C::Q);
    int* ctl = TIER == 1 ? reinterpret_cast<int*>(queue + C::Q + C::Q / 2) : s_ctl[team];
    unsigned long long* counter = &ma.next[TIER - 1];
    const uint64_t items = TIER == 1 ? s_prefix[ma.nq]
                                     : (uint64_t)min(((volatile unsigned*)ma.cnt)[0], ma.list_cap);
    uint2* out_list = TIER == 1 ? ma.list1 : ma.list2;
    unsigned* out_cnt = TIER == 1 ? &ma.cnt[0] : &ma.cnt[1];
    const bool leader = wt == 0 && lane == 0;
    QAcc acc{0, 0, 0, 0, 0, 0, 0};
    int cur_q = -1;
    // kappa of the current query's completed sets, 32 at a time, one per lane (warp 0 of
    // the team): pending widths, the query's m and k, and each lane's 128-bit sum
    unsigned long long kw = 0, km = 0, klo = 0, khi = 0;
    unsigned kcnt = 0;
    int kk = 0;
    auto kflush = [&](int qi) {
        kappa_lanes(kw, kcnt, lane, km, kk, klo, khi);
        kcnt = 0;
        if (qi >= 0 && (klo || khi))
            atomic_add_u128(&ma.q[qi].ds->ksum_lo, &ma.q[qi].ds->ksum_hi, klo, khi);
        klo = khi = 0;
    };
    for (;;) {
        unsigned long long i0 = 0;
        if (leader) i0 = atomicAdd(counter, (unsigned long long)ma.chunk);
        if (T == 1) {
            i0 = __shfl_sync(0xffffffffu, i0, 0);
        } else {
            if (leader) s_claim[team] = i0;
            team_sync<T>(team);
            i0 = s_claim[team];
            team_sync<T>(team);
        }
        if (i0 >= items) break;
        const unsigned long long i1 = min(i0 + (unsigned long long)ma.chunk, (unsigned long long)items);
        for (unsigned long long it = i0; it < i1; it++) {
            int qi;
            uint64_t j;
            if (TIER == 1) {
                int lo = 0, hi = ma.nq;  // s_prefix[lo] <= it < s_prefix[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s_prefix[mid] <= it)
                        lo = mid;
                    else
                        hi = mid;
                }
                qi = lo;
                j = it - s_prefix[lo];
            } else {
                const uint2 e = ma.list1[it];
                qi = (int)e.x;
                j = e.y;
            }
            if (qi != cur_q) {
                if (wt == 0) kflush(cur_q);
                flush_acc<TIER>(ma.q, cur_q, acc, lane);
                cur_q = qi;
            }
            const QueryDesc& d = ma.q[qi];
            const QArgs qa{d.rowptr, d.src, d.thr, d.node_thr, d.qtab,
                           d.n,      d.m,   d.flags, d.k,     d.seed_mark};
            const int model = d.model;
            const unsigned long long budget =
                model != TIM_IC ? ~0ull : TIER == 1 ? d.width_budget : d.width_budget2;
            unsigned long long width;
            int st;
            // IC: pass 2 goes on from the state pass 1 handed over (see rr_team_kernel)
            Resume rin{0, 0ull}, rout{0, 0ull};
            bool resumed = false;
            if (TIER == 2 && model == TIM_IC && ma.hand && it < ma.hcap) {
                const uint32_t* hs = ma.hand + it * (uint64_t)ma.hw;
                const uint32_t t0 = hs[0];
                if (t0 > 0 && t0 <= (uint32_t)C::Q) {
                    if (leader) {
                        ctl[0] = (int)t0;
                        ctl[1] = 0;
                    }
                    team_sync<T>(team);
                    for (uint32_t i = tl; i < t0; i += 32 * T) {
                        const uint32_t u = hs[4 + i];
                        queue[i] = u;
                        uint32_t h = (u * 0x9E3779B1u) >> (32 - C::LOG2H);
                        for (int probe = 0; probe < C::H; probe++) {
                            if (atomicCAS(&hash[h], EMPTY, u) == EMPTY) break;
                            h = (h + 1) & (C::H - 1);
                        }
                        slot[i] = (uint16_t)h;
                        if ((d.flags & SAMPLE_COVER) && marked(d.seed_mark, u))
                            atomicOr(&ctl[1], ST_COVERED);
                    }
                    rin.head = (int)min(hs[1], t0);
                    rin.width = (unsigned long long)hs[2] | ((unsigned long long)hs[3] << 32);
                    resumed = true;
                }
                team_sync<T>(team);
            }
            if (model == TIM_IC)
                st = team_rr<TIM_IC, C, T, QArgs>(qa, ma.K, d.sid0 + j, hash, queue, slot, ctl,
                                                  budget, wt, team, &width, &acc.live,
                                                  &acc.exam, resumed ? &rin : nullptr,
                                                  (TIER == 1 && ma.hand) ? &rout : nullptr);
            else
                st = team_rr<TIM_LT, C, T, QArgs>(qa, ma.K, d.sid0 + j, hash, queue, slot, ctl,
                                                  budget, wt, team, &width, &acc.live,
                                                  &acc.exam);
            const int tail = min(T == 1 ? __shfl_sync(0xffffffffu, ((volatile int*)ctl)[0], 0)
                                        : ((volatile int*)ctl)[0],
                                 C::Q);
            team_sync<T>(team);
            if (st & ST_OVERFLOW) {
                unsigned idx = 0;
                if (leader) {
                    idx = atomicAdd(out_cnt, 1u);
                    if (idx < ma.list_cap)
                        out_list[idx] = make_uint2((uint32_t)qi, (uint32_t)j);
                    else
                        atomicOr(ma.err, TIM_DEV_ERR_OVF_LIST);
                }
                if (TIER == 1 && T == 1 && model == TIM_IC && ma.hand) {
                    idx = __shfl_sync(0xffffffffu, idx, 0);
                    if (idx < ma.hcap) {
                        uint32_t* hs = ma.hand + idx * (uint64_t)ma.hw;
                        for (int i = lane; i < tail; i += 32) hs[4 + i] = queue[i];
                        if (lane == 0) {
                            hs[0] = (uint32_t)tail;
                            hs[1] = (uint32_t)rout.head;
                            hs[2] = (uint32_t)rout.width;
                            hs[3] = (uint32_t)(rout.width >> 32);
                        }
                    }
                }
                for (int i = tl; i < C::H; i += 32 * T) hash[i] = EMPTY;
                team_sync<T>(team);
                continue;
            }
            if (leader) {
                acc.wsum += width;
                acc.memb += tail;
                if (st & ST_COVERED) acc.cov++;
            }
            if ((d.flags & SAMPLE_KAPPA) && wt == 0) {  // width is the same on every lane
                if ((unsigned)lane == kcnt) kw = width;
                km = d.m;
                kk = d.k;
                if (++kcnt == 32) {
                    kappa_lanes(kw, kcnt, lane, km, kk, klo, khi);
                    kcnt = 0;
                }
            }
            if (d.flags & SAMPLE_EMIT) {
                unsigned long long base = 0;
                if (leader) base = atomicAdd(&d.ds->pool_used, (unsigned long long)tail);
                if (T == 1) {
                    base = __shfl_sync(0xffffffffu, base, 0);
                } else {
                    if (leader) s_claim[team] = base;
                    team_sync<T>(team);
                    base = s_claim[team];
                }
                if (base + tail <= d.pool_cap) {
                    for (int i = tl; i < tail; i += 32 * T) {
                        d.pool[base + i] = queue[i];
                        d.pool_sid[base + i] = (uint32_t)j;
                    }
                    if (leader) {
                        d.set_start[j] = base;
                        d.set_len[j] = (uint32_t)tail;
                        d.set_width[j] = width;
                    }
                } else if (leader) {
                    atomicOr(&d.ds->err, TIM_DEV_ERR_POOL);
                }
            }
            for (int i = tl; i < tail; i += 32 * T) hash[slot[i]] = EMPTY;
            team_sync<T>(team);
        }
    }
    if (wt == 0) kflush(cur_q);
    flush_acc<TIER>(ma.q, cur_q, acc, lane);
}

// Tier 1 of the LT queries of a multi-query launch: one chain per thread as in
// rr_lt_lane_kernel, over the set index space of the LT queries (lt_prefix; IC queries
// have no sets there). Each thread keeps its query's totals and flushes them when it
// moves to another query; store space is reserved per set; chains longer than LT_CAP
// join the tier-2 list of the launch.
__global__ void __launch_bounds__(LT_THREADS)
rr_lt_lane_multi_kernel(MultiArgs ma, const unsigned long long* lt_prefix,
                        unsigned long long* lt_next, uint32_t* lt_col) {
    extern __shared__ uint32_t bloom_all[];
    __shared__ unsigned long long s_prefix[MAXQ + 1];
    const int tid = threadIdx.x, lane = tid & 31;
    for (int i = tid; i <= ma.nq; i += blockDim.x) s_prefix[i] = lt_prefix[i];
    uint32_t* bloom = bloom_all + tid;
    for (int w = 0; w < LT_BLOOM_WORDS; w++) bloom[w * LT_THREADS] = 0u;
    __syncthreads();
    const uint64_t total = s_prefix[ma.nq];
    const uint64_t lanes = (uint64_t)gridDim.x * LT_THREADS;
    uint32_t* wcol = lt_col + (uint64_t)blockIdx.x * LT_THREADS + (tid & ~31);
    uint32_t* col = wcol + lane;
    QAcc acc{0, 0, 0, 0, 0, 0, 0};
    int cur_q = -1;
    bool has = false, exhausted = false;
    int qi = -1, flags = 0, kk = 0, len = 0, status = 0;
    uint64_t j = 0, sid = 0, n = 0, m = 0;
    const uint64_t* rowptr = nullptr;
    const uint32_t* src = nullptr;
    const uint32_t* thr = nullptr;
    const unsigned long long* node_thr = nullptr;
    const uint32_t* seed_mark = nullptr;
    uint32_t v = 0;
    unsigned long long width = 0;
    const uint64_t steps = (total + 1) * (uint64_t)(LT_CAP + 2) + 64;
    for (uint64_t guard = 0; guard < steps; guard++) {
        const bool need = !has && !exhausted;
        const unsigned nm = __ballot_sync(0xffffffffu, need);
        if (nm) {
            const int leader = __ffs(nm) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(lt_next, (unsigned long long)__popc(nm));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (need) {
                const unsigned long long mine = base + __popc(nm & ((1u << lane) - 1u));
                if (mine < total) {
                    int lo = 0, hi = ma.nq;  // s_prefix[lo] <= mine < s_prefix[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (s_prefix[mid] <= mine)
                            lo = mid;
                        else
                            hi = mid;
                    }
                    if (lo != cur_q) {
                        if (cur_q >= 0) {
                            DevScalars* ds = ma.q[cur_q].ds;
                            if (acc.k_lo || acc.k_hi)
                                atomic_add_u128(&ds->ksum_lo, &ds->ksum_hi, acc.k_lo, acc.k_hi);
                            if (acc.wsum) {
                                atomicAdd(&ds->wsum, acc.wsum);
                                atomicAdd(&ds->width[0], acc.wsum);
                            }
                            if (acc.cov) atomicAdd(&ds->covered, acc.cov);
                            if (acc.live) atomicAdd(&ds->live[0], acc.live);
                            if (acc.memb) atomicAdd(&ds->memb[0], acc.memb);
                        }
                        acc = QAcc{0, 0, 0, 0, 0, 0, 0};
                        cur_q = lo;
                        const QueryDesc& d = ma.q[lo];
                        rowptr = d.rowptr;
                        src = d.src;
                        thr = d.thr;
                        node_thr = d.node_thr;
                        seed_mark = d.seed_mark;
                        n = d.n;
                        m = d.m;
                        flags = d.flags;
                        kk = d.k;
                    }
                    qi = lo;
                    j = mine - s_prefix[lo];
                    sid = ma.q[lo].sid0 + j;
                    v = rr_root(sid, n, ma.K);
                    col[0] = v;
                    len = 1;
                    width = 0;
                    lane_bloom_add(bloom, v);
                    status = ((flags & SAMPLE_COVER) && marked(seed_mark, v)) ? ST_COVERED : 0;
                    has = true;
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(0xffffffffu, has)) break;
        bool fin = false, cand = false;
        uint32_t u = 0;
        if (has) {
            if (status) {
                fin = true;
            } else {
                const uint64_t beg = __ldg(rowptr + v), end = __ldg(rowptr + v + 1);
                const unsigned long long nt = __ldg(node_thr + v);
                width += end - beg;
                uint64_t jj = end;
                if (beg < end) {
                    const uint32_t x =
                        philox4x32_10((uint32_t)sid, (uint32_t)(sid >> 32), v, TIM_TAG_LT, ma.K).x;
                    jj = (nt >> 32) ? lt_uniform_pick(nt, beg, end, x)
                                    : lane_lt_search(thr, beg, end, x);
                }
                if (jj >= end) {
                    fin = true;
                } else {
                    u = __ldg(src + jj);
                    acc.live++;
                    cand = true;
                }
            }
        }
        const bool seen =
            lane_cols_contain(wcol, lanes, lane, cand && lane_bloom_test(bloom, u), u, len);
        bool ovf = false;
        if (cand) {
            if (seen) {
                fin = true;
            } else if (len == LT_CAP) {
                fin = ovf = true;
            } else {
                col[(uint64_t)len * lanes] = u;
                len++;
                lane_bloom_add(bloom, u);
                if ((flags & SAMPLE_COVER) && marked(seed_mark, u)) status |= ST_COVERED;
                v = u;
            }
        }
        bool put = false;
        unsigned long long st = 0;
        uint32_t* pool = nullptr;
        uint32_t* pool_sid = nullptr;
        if (fin && ovf) {
            const unsigned idx = atomicAdd(&ma.cnt[0], 1u);
            if (idx < ma.list_cap)
                ma.list1[idx] = make_uint2((uint32_t)qi, (uint32_t)j);
            else
                atomicOr(ma.err, TIM_DEV_ERR_OVF_LIST);
        } else if (fin) {
            acc.wsum += width;
            acc.memb += len;
            if (status & ST_COVERED) acc.cov++;
            if (flags & SAMPLE_KAPPA) {
                const unsigned long long kf = kappa_fixed(kappa_fp64(width, m, kk));
                acc.k_lo += kf;
                if (acc.k_lo < kf) acc.k_hi++;
            }
            if (flags & SAMPLE_EMIT) {
                const QueryDesc& d = ma.q[qi];
                st = atomicAdd(&d.ds->pool_used, (unsigned long long)len);
                if (st + (unsigned)len <= d.pool_cap) {
                    put = true;
                    pool = d.pool;
                    pool_sid = d.pool_sid;
                    d.set_start[j] = st;
                    d.set_len[j] = (uint32_t)len;
                    d.set_width[j] = width;
                } else {
                    atomicOr(&d.ds->err, TIM_DEV_ERR_POOL);
                }
            }
        }
        // the warp copies each stored chain's column with all its lanes
        for (unsigned pm = __ballot_sync(0xffffffffu, put); pm; pm &= pm - 1) {
            const int l = __ffs(pm) - 1;
            const unsigned long long sl = __shfl_sync(0xffffffffu, st, l);
            const int ll = __shfl_sync(0xffffffffu, len, l);
            const uint32_t jl = (uint32_t)__shfl_sync(0xffffffffu, (unsigned long long)j, l);
            uint32_t* pl = (uint32_t*)__shfl_sync(0xffffffffu, (unsigned long long)pool, l);
            uint32_t* psl = (uint32_t*)__shfl_sync(0xffffffffu, (unsigned long long)pool_sid, l);
            for (int k = lane; k < ll; k += 32) {
                pl[sl + k] = wcol[(uint64_t)k * lanes + l];
                psl[sl + k] = jl;
            }
        }
        if (fin) {
            for (int w = 0; w < LT_BLOOM_WORDS; w++) bloom[w * LT_THREADS] = 0u;
            has = false;
        }
    }
    if (cur_q >= 0) {
        DevScalars* ds = ma.q[cur_q].ds;
        if (acc.k_lo || acc.k_hi) atomic_add_u128(&ds->ksum_lo, &ds->ksum_hi, acc.k_lo, acc.k_hi);
        if (acc.wsum) {
            atomicAdd(&ds->wsum, acc.wsum);
            atomicAdd(&ds->width[0], acc.wsum);
        }
        if (acc.cov) atomicAdd(&ds->covered, acc.cov);
        if (acc.live) atomicAdd(&ds->live[0], acc.live);
        if (acc.memb) atomicAdd(&ds->memb[0], acc.memb);
    }
}

int launch_multi(tim_ctx* owner, const MultiArgs& ma, int tier, int T, unsigned grid,
                 size_t smem) {
    if (tier == 1) {
        if (owner->cap1 == 128)
            rr_multi_kernel<Tier1S, 1, 1><<<grid, WARPS * 32, smem, owner->stream>>>(ma);
        else if (owner->cap1 == 512)
            rr_multi_kernel<Tier1L, 1, 1><<<grid, WARPS * 32, smem, owner->stream>>>(ma);
        else
            rr_multi_kernel<Tier1, 1, 1><<<grid, WARPS * 32, smem, owner->stream>>>(ma);
    } else if (T == 1) {
        rr_multi_kernel<Tier2, 2, 1><<<grid, WARPS * 32, 0, owner->stream>>>(ma);
    } else if (T == 2) {
        rr_multi_kernel<Tier2, 2, 2><<<grid, WARPS * 32, 0, owner->stream>>>(ma);
    } else if (T == 4) {
        rr_multi_kernel<Tier2, 2, 4><<<grid, WARPS * 32, 0, owner->stream>>>(ma);
    } else {
        rr_multi_kernel<Tier2, 2, 8><<<grid, WARPS * 32, 0, owner->stream>>>(ma);
    }
    LAUNCH_CHECK(owner, tier == 1 ? "rr_multi_kernel (tier 1)" : "rr_multi_kernel (tier 2)");
    return TIM_OK;
}

template <class C, int TIER, int T>
int multi_occupancy(size_t smem) {
    int nb = 0;
    auto k = rr_multi_kernel<C, TIER, T>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, WARPS * 32, smem) != cudaSuccess ||
        nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

}  // namespace

int tim_sample(tim_ctx* ctx, const SampleRequest& req, SampleResult* res) {
    if (!ctx->have_graph) return tim_fail(ctx, TIM_ERR_STATE, "no graph loaded");
    const uint64_t count = req.count;
    const bool emit = req.flags & SAMPLE_EMIT;
    if (count > 0xFFFFFFF0ull) return tim_fail(ctx, TIM_ERR_ARG, "too many RR sets in one call");
    // per-set arrays grow to the next power of two so that the doubling rounds of
    // Algorithm 2 do not reallocate every round
    uint64_t cap_sets = 1024;
    while (cap_sets < count + 1) cap_sets <<= 1;
    if (emit) {
        TIM_TRY(tim_ensure(ctx, ctx->set_start, cap_sets * sizeof(uint64_t)));
        TIM_TRY(tim_ensure(ctx, ctx->set_len, cap_sets * sizeof(uint32_t)));
        TIM_TRY(tim_ensure(ctx, ctx->set_width, cap_sets * sizeof(uint64_t)));
        uint64_t want = cap_sets * 8 + 4096;
        if (ctx->pool.bytes < want * sizeof(uint32_t)) {
            TIM_TRY(tim_ensure(ctx, ctx->pool, want * sizeof(uint32_t)));
            TIM_TRY(tim_ensure(ctx, ctx->pool_sid, want * sizeof(uint32_t)));
        }
    }
    const uint32_t list_cap = (uint32_t)(count + 1);
    TIM_TRY(tim_ensure(ctx, ctx->ovf_list, (size_t)cap_sets * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->ovf_list2, (size_t)cap_sets * sizeof(uint32_t)));

    // tier 2 arena: one slot per resident warp, hash regions kept EMPTY between sets
    const int cap1 = ctx->model == TIM_IC ? ctx->cap1 : 256;
    const size_t smem1 = (size_t)WARPS * sizeof(uint32_t) *
                         (cap1 == 128 ? Tier1S::WORDS : cap1 == 512 ? Tier1L::WORDS : Tier1::WORDS);
    const int nb1 = ctx->model == TIM_IC
                        ? (cap1 == 128   ? occupancy<TIM_IC, Tier1S, 1, 1>(smem1)
                           : cap1 == 512 ? occupancy<TIM_IC, Tier1L, 1, 1>(smem1)
                                         : occupancy<TIM_IC, Tier1, 1, 1>(smem1))
                    : ctx->model == TIM_TRIG ? occupancy<TIM_TRIG, Tier1, 1, 1>(smem1)
                                             : occupancy<TIM_LT, Tier1, 1, 1>(smem1);
    const int nb2 = ctx->model == TIM_IC     ? occupancy<TIM_IC, Tier2, 2, 1>(0)
                    : ctx->model == TIM_TRIG ? occupancy<TIM_TRIG, Tier2, 2, 1>(0)
                                             : occupancy<TIM_LT, Tier2, 2, 1>(0);
    const unsigned grid1 = (unsigned)(ctx->num_sms * nb1);
    const unsigned grid2 = (unsigned)(ctx->num_sms * nb2);
    const size_t arena_bytes = (size_t)grid2 * WARPS * Tier2::WORDS * sizeof(uint32_t);
    void* prev_arena = ctx->arena.p;
    TIM_TRY(tim_ensure(ctx, ctx->arena, arena_bytes));
    if (ctx->arena.p != prev_arena || !ctx->arena_clean) {
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->arena.p, 0xFF, ctx->arena.bytes, ctx->stream));
        ctx->arena_clean = true;
    }
    // tier 3 LT and triggering slots: a bitmap of n bits and a queue of n entries each,
    // at most ~2 GiB
    const uint64_t words = (uint64_t)(ctx->n + 31) / 32 + 1;
    int slots = 0;
    if (ctx->model != TIM_IC) {
        const uint64_t per_slot = (words + (uint64_t)ctx->n) * sizeof(uint32_t);
        slots = ctx->num_sms;
        const uint64_t budget = 2ull << 30;
        if ((uint64_t)slots * per_slot > budget)
            slots = (int)std::max<uint64_t>(1, budget / per_slot);
        void* prev_bm = ctx->big_bitmap.p;
        TIM_TRY(tim_ensure(ctx, ctx->big_bitmap, (size_t)slots * words * sizeof(uint32_t)));
        TIM_TRY(tim_ensure(ctx, ctx->big_queue,
                           (size_t)slots * (uint64_t)ctx->n * sizeof(uint32_t)));
        if (ctx->big_bitmap.p != prev_bm || !ctx->big_bitmap_clean) {
            CUDA_TRY(ctx, cudaMemsetAsync(ctx->big_bitmap.p, 0, ctx->big_bitmap.bytes, ctx->stream));
            ctx->big_bitmap_clean = true;
        }
    }
    SampleArgs a;
    a.rowptr = (const uint64_t*)ctx->rowptr.p;
    a.src = (const uint32_t*)ctx->src.p;
    a.thr = (const uint32_t*)ctx->thr.p;
    a.node_thr = (const unsigned long long*)ctx->node_thr.p;
    a.qtab = (const unsigned long long*)ctx->qtab.p;
    a.n = (uint64_t)ctx->n;
    a.m = (uint64_t)ctx->m;
    a.K = tim_philox_keys(req.seed);
    a.sid0 = req.sid0;
    a.count = count;
    a.flags = req.flags;
    a.k = req.k;
    a.seed_mark = req.seed_mark;
    a.ds = tim_dscal(ctx);
    a.list1 = (uint32_t*)ctx->ovf_list.p;
    a.list2 = (uint32_t*)ctx->ovf_list2.p;
    a.list_cap = list_cap;
    a.arena = (uint32_t*)ctx->arena.p;
    a.big_bitmap = (uint32_t*)ctx->big_bitmap.p;
    a.big_queue = (uint32_t*)ctx->big_queue.p;
    a.big_words = words;
    a.set_start = (uint64_t*)ctx->set_start.p;
    a.set_len = (uint32_t*)ctx->set_len.p;
    a.set_width = (uint64_t*)ctx->set_width.p;
    a.width_budget = ctx->width_budget;
    a.width_budget2 = ctx->width_budget2;
    a.chunk = std::max(1, ctx->chunk);
    // IC: room for the pass-1 state of up to count / 8 + 4096 handed-over sets (at most
    // 1 GiB); sets listed beyond it start over in pass 2
    a.hand = nullptr;
    a.hcap = 0;
    a.hw = 4u + (uint32_t)cap1;
    if (ctx->model == TIM_IC && count > 0) {
        const uint64_t maxslots = (1ull << 30) / ((uint64_t)a.hw * sizeof(uint32_t));
        const uint64_t hcap = std::min<uint64_t>(std::min<uint64_t>(count / 8 + 4096, maxslots),
                                                 list_cap);
        TIM_TRY(tim_ensure(ctx, ctx->hand, (size_t)hcap * a.hw * sizeof(uint32_t)));
        a.hand = (uint32_t*)ctx->hand.p;
        a.hcap = (uint32_t)hcap;
    }
    a.hand2 = nullptr;
    a.h2cap = 0;
    a.h2w = 4u + (uint32_t)Tier2::Q;
    if (ctx->model == TIM_IC && count > 0) {  // at most 1 GiB; later sets start over
        const uint64_t h2cap = std::min<uint64_t>((1ull << 30) / ((uint64_t)a.h2w * 4), list_cap);
        TIM_TRY(tim_ensure(ctx, ctx->hand2, (size_t)h2cap * a.h2w * sizeof(uint32_t)));
        a.hand2 = (uint32_t*)ctx->hand2.p;
        a.h2cap = (uint32_t)h2cap;
    }
    a.node_opt = (const uint64_t*)ctx->node_opt.p;
    a.opt_cum = (const uint32_t*)ctx->opt_cum.p;
    a.opt_off = (const uint64_t*)ctx->opt_off.p;
    a.opt_pos = (const uint32_t*)ctx->opt_pos.p;
    for (int attempt = 0; attempt < 4; attempt++) {
        a.pool = (uint32_t*)ctx->pool.p;
        a.pool_sid = (uint32_t*)ctx->pool_sid.p;
        a.pool_cap = emit ? ctx->pool.bytes / sizeof(uint32_t) : 0;
        TIM_TRY(tim_zero_scalars(ctx));
        uint64_t live3 = 0;
        if (count > 0) {
            cudaEventRecord(ctx->kev[0], ctx->stream);
            TIM_TRY(launch_tier1(ctx, a, grid1, smem1));
            cudaEventRecord(ctx->kev[1], ctx->stream);
            // team size of tier 2: intra-set parallelism when the listed sets are few
            int T = 1;
            if (ctx->model == TIM_IC) {
                TIM_TRY(tim_read_scalars(ctx));
                const uint64_t listed = ctx->h_scal->cnt1;
                const uint64_t slots1 = (uint64_t)grid2 * WARPS;
                T = ctx->team_size;
                if (T <= 0) {
                    T = 1;
                    while (T < 8 && listed * (uint64_t)ctx->team_factor < slots1 / T) T *= 2;
                }
                ctx->last_team = T;
            }
            TIM_TRY(launch_tier2(ctx, a, grid2, T));
            cudaEventRecord(ctx->kev[2], ctx->stream);
            if (ctx->model == TIM_IC) {
                TIM_TRY(tim_read_scalars(ctx));
                const unsigned n3 = std::min(ctx->h_scal->cnt2, list_cap);
                TIM_TRY(tim_bulk_ic(ctx, req, a.list2, n3, a.pool, a.pool_sid, a.pool_cap, a.ds,
                                    &live3, a.hand2, a.h2cap, a.h2w));
            } else if (ctx->model == TIM_TRIG) {
                rr_trig_big_kernel<<<slots, BIG_THREADS, 0, ctx->stream>>>(a);
                LAUNCH_CHECK(ctx, "rr_trig_big_kernel");
            } else {
                rr_lt_chain_kernel<<<slots, BIG_THREADS, 0, ctx->stream>>>(a);
                LAUNCH_CHECK(ctx, "rr_lt_chain_kernel");
            }
            cudaEventRecord(ctx->kev[3], ctx->stream);
        }
        TIM_TRY(tim_read_scalars(ctx));
        DevScalars& h = *ctx->h_scal;
        if (ctx->model == TIM_IC) h.live[2] = live3;
        if (h.err & TIM_DEV_ERR_POOL) {
            uint64_t need = h.pool_used + h.pool_used / 16 + 4096;
            tim_free(ctx->pool);
            tim_free(ctx->pool_sid);
            TIM_TRY(tim_ensure(ctx, ctx->pool, need * sizeof(uint32_t)));
            TIM_TRY(tim_ensure(ctx, ctx->pool_sid, need * sizeof(uint32_t)));
            continue;
        }
        if (h.err) {
            ctx->arena_clean = ctx->big_bitmap_clean = false;
            return tim_fail(ctx, TIM_ERR_CUDA, "device error flags set by the RR sampler");
        }
        if (count > 0) {
            float t[3] = {0.f, 0.f, 0.f};
            for (int i = 0; i < 3; i++) cudaEventElapsedTime(&t[i], ctx->kev[i], ctx->kev[i + 1]);
            const uint64_t sets[3] = {count - h.cnt1, (uint64_t)h.cnt1 - h.cnt2, h.cnt2};
            tim_profile& P = ctx->prof;
            uint64_t* L[3] = {&P.pass1_launches, &P.pass2_launches, &P.pass3_launches};
            double* T[3] = {&P.pass1_ms, &P.pass2_ms, &P.pass3_ms};
            uint64_t* S[3] = {&P.pass1_sets, &P.pass2_sets, &P.pass3_sets};
            uint64_t* W[3] = {&P.pass1_width, &P.pass2_width, &P.pass3_width};
            uint64_t* V[3] = {&P.pass1_live, &P.pass2_live, &P.pass3_live};
            uint64_t* M[3] = {&P.pass1_members, &P.pass2_members, &P.pass3_members};
            uint64_t* X[3] = {&P.pass1_examined, &P.pass2_examined, &P.pass3_examined};
            for (int i = 0; i < 3; i++) {
                *L[i] += 1;
                *T[i] += t[i];
                *S[i] += sets[i];
                *W[i] += h.width[i];
                *V[i] += h.live[i];
                *M[i] += h.memb[i];
                *X[i] += h.exam[i];
            }
        }
        if (res) {
            res->ksum = ((unsigned __int128)h.ksum_hi << 64) | h.ksum_lo;
            res->wsum = h.wsum;
            res->live = h.live[0] + h.live[1] + h.live[2];
            res->covered = h.covered;
            res->members = emit ? h.pool_used : 0;
            res->big_sets = h.cnt1;
        }
        if (emit) {
            ctx->n_sets = count;
            ctx->members = h.pool_used;
            ctx->select_open = false;
        }
        return TIM_OK;
    }
    return tim_fail(ctx, TIM_ERR_OOM, "RR-set store kept overflowing");
}

// ----------------------------------------------------- multi-query host driver

namespace {

// Tier-3 LT slots of one context: a visited bitmap of n bits and a queue of n entries
// each, at most ~2 GiB in total.
int ensure_lt_slots(tim_ctx* ctx, int* slots_out, uint64_t* words_out) {
    const uint64_t words = (uint64_t)(ctx->n + 31) / 32 + 1;
    const uint64_t per_slot = (words + (uint64_t)ctx->n) * sizeof(uint32_t);
    int slots = ctx->num_sms;
    const uint64_t budget = 2ull << 30;
    if ((uint64_t)slots * per_slot > budget) slots = (int)std::max<uint64_t>(1, budget / per_slot);
    void* prev_bm = ctx->big_bitmap.p;
    TIM_TRY(tim_ensure(ctx, ctx->big_bitmap, (size_t)slots * words * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->big_queue, (size_t)slots * (uint64_t)ctx->n * sizeof(uint32_t)));
    if (ctx->big_bitmap.p != prev_bm || !ctx->big_bitmap_clean) {
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->big_bitmap.p, 0, ctx->big_bitmap.bytes, ctx->stream));
        ctx->big_bitmap_clean = true;
    }
    *slots_out = slots;
    *words_out = words;
    return TIM_OK;
}

// Tier 3 for one query of a multi-query launch: the sets list_dev[0 .. n3) of ctx's
// graph, accumulating into ds. Runs on `stream`.
int run_tier3(tim_ctx* ctx, cudaStream_t stream, const SampleRequest& req, DevScalars* ds,
              uint32_t* pool, uint32_t* pool_sid, uint64_t pool_cap, const uint32_t* list_dev,
              unsigned n3, uint64_t* live3) {
    cudaStream_t saved = ctx->stream;
    ctx->stream = stream;
    int rc = TIM_OK;
    if (ctx->model == TIM_IC) {
        rc = tim_bulk_ic(ctx, req, list_dev, n3, pool, pool_sid, pool_cap, ds, live3);
    } else {
        int slots = 0;
        uint64_t words = 0;
        rc = ensure_lt_slots(ctx, &slots, &words);
        if (rc == TIM_OK) {
            SampleArgs a{};
            a.rowptr = (const uint64_t*)ctx->rowptr.p;
            a.src = (const uint32_t*)ctx->src.p;
            a.thr = (const uint32_t*)ctx->thr.p;
            a.n = (uint64_t)ctx->n;
            a.m = (uint64_t)ctx->m;
            a.K = tim_philox_keys(req.seed);
            a.sid0 = req.sid0;
            a.count = req.count;
            a.flags = req.flags;
            a.k = req.k;
            a.seed_mark = req.seed_mark;
            a.pool = pool;
            a.pool_sid = pool_sid;
            a.pool_cap = pool_cap;
            a.set_start = (uint64_t*)ctx->set_start.p;
            a.set_len = (uint32_t*)ctx->set_len.p;
            a.set_width = (uint64_t*)ctx->set_width.p;
            a.ds = ds;
            a.list2 = const_cast<uint32_t*>(list_dev);
            a.list_cap = n3 + 1;
            a.big_bitmap = (uint32_t*)ctx->big_bitmap.p;
            a.big_queue = (uint32_t*)ctx->big_queue.p;
            a.big_words = words;
            a.chunk = 1;
            rc = tim_cuda_check(ctx, cudaMemcpyAsync(&ds->cnt2, &n3, sizeof(unsigned),
                                                     cudaMemcpyHostToDevice, stream),
                                "tier-3 count");
            if (rc == TIM_OK) rc = tim_cuda_check(ctx, cudaMemsetAsync(&ds->next3, 0, 8, stream), "memset");
            if (rc == TIM_OK) rc = tim_cuda_check(ctx, cudaStreamSynchronize(stream), "sync");
            if (rc == TIM_OK) {
                rr_lt_chain_kernel<<<slots, BIG_THREADS, 0, stream>>>(a);
                ctx->launches++;
                rc = tim_cuda_check(ctx, cudaGetLastError(), "rr_lt_chain_kernel");
            }
        }
        *live3 = 0;
    }
    ctx->stream = saved;
    return rc;
}

}  // namespace

int tim_sample_multi(tim_ctx* owner, MultiQuery* qs, int nq, uint64_t seed) {
    if (nq <= 0) return TIM_OK;
    if (nq > MAXQ) return tim_fail(owner, TIM_ERR_ARG, "too many queries in one launch");
    // IC queries are sampled by rr_multi_kernel over their own set index space, LT
    // queries by rr_lt_lane_multi_kernel over theirs
    std::vector<unsigned long long> prefix(nq + 1, 0), prefix_lt(nq + 1, 0);
    uint64_t total = 0, total_ic = 0, total_lt = 0;
    for (int i = 0; i < nq; i++) {
        tim_ctx* c = qs[i].ctx;
        if (!c || !c->have_graph) return tim_fail(owner, TIM_ERR_STATE, "query without a graph");
        if (c->device != owner->device) return tim_fail(owner, TIM_ERR_ARG, "queries on several devices");
        if (c->model == TIM_TRIG)
            return tim_fail(owner, TIM_ERR_ARG,
                            "the multi-query sampler takes IC and LT graphs; a triggering-model "
                            "graph runs one query at a time");
        const uint64_t count = qs[i].req.count;
        if (count > 0xFFFFFFF0ull) return tim_fail(owner, TIM_ERR_ARG, "too many RR sets in one call");
        prefix[i] = total_ic;
        prefix_lt[i] = total_lt;
        if (c->model == TIM_LT)
            total_lt += count;
        else
            total_ic += count;
        total += count;
        if (qs[i].req.flags & SAMPLE_EMIT) {
            uint64_t cap_sets = 1024;
            while (cap_sets < count + 1) cap_sets <<= 1;
            TIM_TRY(tim_ensure(c, c->set_start, cap_sets * sizeof(uint64_t)));
            TIM_TRY(tim_ensure(c, c->set_len, cap_sets * sizeof(uint32_t)));
            TIM_TRY(tim_ensure(c, c->set_width, cap_sets * sizeof(uint64_t)));
            const uint64_t want = cap_sets * 8 + 4096;
            if (c->pool.bytes < want * sizeof(uint32_t)) {
                TIM_TRY(tim_ensure(c, c->pool, want * sizeof(uint32_t)));
                TIM_TRY(tim_ensure(c, c->pool_sid, want * sizeof(uint32_t)));
            }
        }
    }
    prefix[nq] = total_ic;
    prefix_lt[nq] = total_lt;
    if (total > 0xFFFFFFF0ull) return tim_fail(owner, TIM_ERR_ARG, "too many RR sets in one launch");
    // owner scratch: descriptors | IC prefix | per-query scalars | next[2] | cnt[2] | err |
    // LT work counter | LT prefix
    const size_t off_prefix = ((size_t)nq * sizeof(QueryDesc) + 255) & ~size_t(255);
    const size_t off_scal = (off_prefix + (size_t)(nq + 1) * 8 + 255) & ~size_t(255);
    const size_t off_ctr = (off_scal + (size_t)nq * sizeof(DevScalars) + 255) & ~size_t(255);
    const size_t off_prefix_lt = off_ctr + 64;
    const size_t batch_bytes = off_prefix_lt + (size_t)(nq + 1) * 8;
    TIM_TRY(tim_ensure(owner, owner->batch, batch_bytes));
    char* bb = (char*)owner->batch.p;
    QueryDesc* d_desc = (QueryDesc*)bb;
    unsigned long long* d_prefix = (unsigned long long*)(bb + off_prefix);
    DevScalars* d_scal = (DevScalars*)(bb + off_scal);
    unsigned long long* d_next = (unsigned long long*)(bb + off_ctr);
    unsigned* d_cnt = (unsigned*)(bb + off_ctr + 16);
    int* d_err = (int*)(bb + off_ctr + 24);
    unsigned long long* d_lt_next = (unsigned long long*)(bb + off_ctr + 32);
    unsigned long long* d_prefix_lt = (unsigned long long*)(bb + off_prefix_lt);
    unsigned grid_lt = 0;
    if (total_lt > 0) {
        int nb = 0;
        CUDA_TRY(owner, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &nb, rr_lt_lane_multi_kernel, LT_THREADS, LT_SMEM));
        grid_lt = (unsigned)(owner->num_sms * std::max(nb, 1));
        TIM_TRY(tim_ensure(owner, owner->lt_col,
                           (size_t)grid_lt * LT_THREADS * LT_CAP * sizeof(uint32_t)));
    }
    TIM_TRY(tim_ensure(owner, owner->ovf_list, (size_t)(total + 1) * sizeof(uint2)));
    TIM_TRY(tim_ensure(owner, owner->ovf_list2, (size_t)(total + 1) * sizeof(uint2)));
    // arena and occupancy as in the single-query path
    const int cap1 = owner->cap1;
    const size_t smem1 = (size_t)WARPS * sizeof(uint32_t) *
                         (cap1 == 128 ? Tier1S::WORDS : cap1 == 512 ? Tier1L::WORDS : Tier1::WORDS);
    const int nb1 = cap1 == 128   ? multi_occupancy<Tier1S, 1, 1>(smem1)
                    : cap1 == 512 ? multi_occupancy<Tier1L, 1, 1>(smem1)
                                  : multi_occupancy<Tier1, 1, 1>(smem1);
    const int nb2 = multi_occupancy<Tier2, 2, 1>(0);
    const unsigned grid1 = (unsigned)(owner->num_sms * nb1);
    const unsigned grid2 = (unsigned)(owner->num_sms * nb2);
    const size_t arena_bytes = (size_t)grid2 * WARPS * Tier2::WORDS * sizeof(uint32_t);
    void* prev_arena = owner->arena.p;
    TIM_TRY(tim_ensure(owner, owner->arena, arena_bytes));
    if (owner->arena.p != prev_arena || !owner->arena_clean) {
        CUDA_TRY(owner, cudaMemsetAsync(owner->arena.p, 0xFF, owner->arena.bytes, owner->stream));
        owner->arena_clean = true;
    }
    MultiArgs ma;
    ma.K = tim_philox_keys(seed);
    ma.q = d_desc;
    ma.prefix = d_prefix;
    ma.nq = nq;
    ma.chunk = std::max(1, owner->chunk);
    ma.next = d_next;
    ma.cnt = d_cnt;
    ma.err = d_err;
    ma.list1 = (uint2*)owner->ovf_list.p;
    ma.list2 = (uint2*)owner->ovf_list2.p;
    ma.list_cap = (uint32_t)(total + 1);
    ma.arena = (uint32_t*)owner->arena.p;
    // pass-1 state handed to pass 2 (IC queries), in the owner's scratch
    ma.hw = 4u + (uint32_t)cap1;
    {
        const uint64_t maxslots = (1ull << 30) / ((uint64_t)ma.hw * sizeof(uint32_t));
        const uint64_t hcap =
            std::min<uint64_t>(std::min<uint64_t>(total_ic / 8 + 4096, maxslots), total + 1);
        TIM_TRY(tim_ensure(owner, owner->hand, (size_t)hcap * ma.hw * sizeof(uint32_t)));
        ma.hand = (uint32_t*)owner->hand.p;
        ma.hcap = (uint32_t)hcap;
    }
    std::vector<QueryDesc> h_desc(nq);
    std::vector<DevScalars> h_scal(nq);
    for (int attempt = 0; attempt < 4; attempt++) {
        for (int i = 0; i < nq; i++) {
            tim_ctx* c = qs[i].ctx;
            const SampleRequest& r = qs[i].req;
            QueryDesc& d = h_desc[i];
            d.rowptr = (const uint64_t*)c->rowptr.p;
            d.src = (const uint32_t*)c->src.p;
            d.thr = (const uint32_t*)c->thr.p;
            d.node_thr = (const unsigned long long*)c->node_thr.p;
            d.qtab = (const unsigned long long*)c->qtab.p;
            d.n = (uint64_t)c->n;
            d.m = (uint64_t)c->m;
            d.sid0 = r.sid0;
            d.count = r.count;
            d.model = c->model;
            d.flags = r.flags;
            d.k = r.k;
            d.pad = 0;
            d.seed_mark = r.seed_mark;
            const bool emit = r.flags & SAMPLE_EMIT;
            d.pool = emit ? (uint32_t*)c->pool.p : nullptr;
            d.pool_sid = emit ? (uint32_t*)c->pool_sid.p : nullptr;
            d.pool_cap = emit ? c->pool.bytes / sizeof(uint32_t) : 0;
            d.set_start = (uint64_t*)c->set_start.p;
            d.set_len = (uint32_t*)c->set_len.p;
            d.set_width = (uint64_t*)c->set_width.p;
            d.ds = d_scal + i;
            d.width_budget = c->width_budget;
            d.width_budget2 = c->width_budget2;
        }
        CUDA_TRY(owner, cudaMemcpyAsync(d_desc, h_desc.data(), (size_t)nq * sizeof(QueryDesc),
                                        cudaMemcpyHostToDevice, owner->stream));
        CUDA_TRY(owner, cudaMemcpyAsync(d_prefix, prefix.data(), (size_t)(nq + 1) * 8,
                                        cudaMemcpyHostToDevice, owner->stream));
        CUDA_TRY(owner, cudaMemcpyAsync(d_prefix_lt, prefix_lt.data(), (size_t)(nq + 1) * 8,
                                        cudaMemcpyHostToDevice, owner->stream));
        CUDA_TRY(owner, cudaMemsetAsync(d_scal, 0, (size_t)nq * sizeof(DevScalars), owner->stream));
        CUDA_TRY(owner, cudaMemsetAsync(d_next, 0, 64, owner->stream));
        uint64_t live3_total = 0;
        std::vector<uint64_t> live3(nq, 0);
        if (total > 0) {
            if (total_ic > 0) TIM_TRY(launch_multi(owner, ma, 1, 1, grid1, smem1));
            if (total_lt > 0) {
                rr_lt_lane_multi_kernel<<<grid_lt, LT_THREADS, LT_SMEM, owner->stream>>>(
                    ma, d_prefix_lt, d_lt_next, (uint32_t*)owner->lt_col.p);
                LAUNCH_CHECK(owner, "rr_lt_lane_multi_kernel (tier 1)");
            }
            unsigned h_cnt[2] = {0, 0};
            CUDA_TRY(owner, cudaMemcpyAsync(h_cnt, d_cnt, sizeof h_cnt, cudaMemcpyDeviceToHost,
                                            owner->stream));
            TIM_TRY(tim_sync(owner));
            int T = owner->team_size;
            if (T <= 0) {
                T = 1;
                const uint64_t slots1 = (uint64_t)grid2 * WARPS;
                while (T < 8 && (uint64_t)h_cnt[0] * (uint64_t)owner->team_factor < slots1 / T)
                    T *= 2;
            }
            TIM_TRY(launch_multi(owner, ma, 2, T, grid2, 0));
            CUDA_TRY(owner, cudaMemcpyAsync(h_cnt, d_cnt, sizeof h_cnt, cudaMemcpyDeviceToHost,
                                            owner->stream));
            TIM_TRY(tim_sync(owner));
            const unsigned n3 = std::min<unsigned>(h_cnt[1], ma.list_cap);
            if (n3 > 0) {
                // the rare sets beyond tier 2: per query, with that query's context
                std::vector<uint2> l2(n3);
                CUDA_TRY(owner, cudaMemcpyAsync(l2.data(), ma.list2, (size_t)n3 * sizeof(uint2),
                                                cudaMemcpyDeviceToHost, owner->stream));
                TIM_TRY(tim_sync(owner));
                std::vector<std::vector<uint32_t>> per(nq);
                for (const uint2& e : l2) per[e.x].push_back(e.y);
                for (int i = 0; i < nq; i++) {
                    if (per[i].empty()) continue;
                    tim_ctx* c = qs[i].ctx;
                    TIM_TRY(tim_ensure(c, c->ovf_list2, per[i].size() * sizeof(uint32_t)));
                    CUDA_TRY(owner, cudaMemcpyAsync(c->ovf_list2.p, per[i].data(),
                                                    per[i].size() * sizeof(uint32_t),
                                                    cudaMemcpyHostToDevice, owner->stream));
                    SampleRequest r = qs[i].req;
                    TIM_TRY(run_tier3(c, owner->stream, r, d_scal + i, h_desc[i].pool,
                                      h_desc[i].pool_sid, h_desc[i].pool_cap,
                                      (const uint32_t*)c->ovf_list2.p, (unsigned)per[i].size(),
                                      &live3[i]));
                    live3_total += live3[i];
                }
            }
        }
        CUDA_TRY(owner, cudaMemcpyAsync(h_scal.data(), d_scal, (size_t)nq * sizeof(DevScalars),
                                        cudaMemcpyDeviceToHost, owner->stream));
        int h_err = 0;
        CUDA_TRY(owner, cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost,
                                        owner->stream));
        TIM_TRY(tim_sync(owner));
        bool regrow = false;
        for (int i = 0; i < nq; i++) {
            if (h_scal[i].err & TIM_DEV_ERR_POOL) {
                tim_ctx* c = qs[i].ctx;
                const uint64_t need = h_scal[i].pool_used + h_scal[i].pool_used / 16 + 4096;
                tim_free(c->pool);
                tim_free(c->pool_sid);
                TIM_TRY(tim_ensure(c, c->pool, need * sizeof(uint32_t)));
                TIM_TRY(tim_ensure(c, c->pool_sid, need * sizeof(uint32_t)));
                regrow = true;
            } else if (h_scal[i].err) {
                h_err |= h_scal[i].err;
            }
        }
        if (regrow) continue;
        if (h_err) {
            owner->arena_clean = false;
            return tim_fail(owner, TIM_ERR_CUDA, "device error flags set by the multi-query sampler");
        }
        for (int i = 0; i < nq; i++) {
            const DevScalars& h = h_scal[i];
            SampleResult& res = qs[i].res;
            res.ksum = ((unsigned __int128)h.ksum_hi << 64) | h.ksum_lo;
            res.wsum = h.wsum;
            res.live = h.live[0] + h.live[1] + live3[i];
            res.covered = h.covered;
            const bool emit = qs[i].req.flags & SAMPLE_EMIT;
            res.members = emit ? h.pool_used : 0;
            res.big_sets = 0;
            if (emit) {
                qs[i].ctx->n_sets = qs[i].req.count;
                qs[i].ctx->members = h.pool_used;
            }
        }
        (void)live3_total;
        return TIM_OK;
    }
    return tim_fail(owner, TIM_ERR_OOM, "RR-set stores kept overflowing");
}
