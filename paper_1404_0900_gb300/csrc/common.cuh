// common.cuh -- context state, error handling and device helpers shared by the
// translation units of libtim.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "tim.h"

// ------------------------------------------------------------------ host side

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Scalars the kernels update; one block of device memory per context, mirrored in
// pinned host memory for cheap read-back.
struct DevScalars {
    unsigned long long next_set;   // tier-1 work counter
    unsigned long long pool_used;  // RR-set store fill (members)
    unsigned long long ksum_lo;    // kappa fixed-point sum, low 64 bits
    unsigned long long ksum_hi;    // high 64 bits
    unsigned long long wsum;       // sum of widths, all tiers
    unsigned long long covered;    // covered-set counter
    unsigned long long next2;      // tier-2 work counter
    unsigned long long next3;      // tier-3 work counter
    unsigned int cnt1;             // sets tier 1 listed for tier 2
    unsigned int cnt2;             // sets tier 2 listed for tier 3
    int err;                       // device-side error bits (TIM_DEV_ERR_*)
    int pad0;
    unsigned long long width[3];   // sum of widths per tier
    unsigned long long live[3];    // live in-edges followed per tier
    unsigned long long memb[3];    // members per tier
    unsigned long long exam[3];    // in-edges whose own threshold was read, per tier
};

enum : int {
    TIM_DEV_ERR_POOL = 1,     // RR-set store too small (host grows it and re-runs)
    TIM_DEV_ERR_OVF_LIST = 2, // second-pass list too small
    TIM_DEV_ERR_GRAPH = 4,    // invalid graph (range, self-loop, duplicate)
    TIM_DEV_ERR_WEIGHT = 8,   // invalid weight
    TIM_DEV_ERR_BOUNDS = 16,  // an index check failed
    TIM_DEV_ERR_TIMEOUT = 32, // a bounded device wait gave up
};

struct tim_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    std::string last_err;
    unsigned long long launches = 0;

    // graph: G^T as in-CSR
    bool have_graph = false;
    int64_t n = 0, m = 0;
    int model = -1;
    DevBuf rowptr;  // uint64[n+1]
    DevBuf src;     // uint32[m + 4]
    DevBuf thr;     // uint32[m + 4] IC thresholds or LT inclusive cumulative thresholds
    DevBuf qtab;      // IC: per skip-rule node, Q_0..Q_31 of its geometric gaps (u64[32])
    // triggering model: options of node v at node_opt[v] .. node_opt[v+1] (u64[n+1]);
    // per option its inclusive cumulative threshold (u32) and its in-edges at opt_off[o]
    // .. opt_off[o+1] (u64) as in-CSR positions opt_pos (u32)
    DevBuf node_opt, opt_cum, opt_off, opt_pos, opt_node;
    DevBuf node_thr;  // IC: uint64[n], low word = threshold shared by all in-edges of v,
                      // bit 32 set when they do share one (empty in-lists included),
                      // bits 33..63 = 1 + index of the node's qtab entry (skip rule)

    // RR-set store
    uint64_t n_sets = 0;
    uint64_t members = 0;
    DevBuf pool;       // uint32 members, grouped by set (sets in any order)
    DevBuf pool_sid;   // uint32 set index of each member
    DevBuf set_start;  // uint64[n_sets]
    DevBuf set_len;    // uint32[n_sets]
    DevBuf set_width;  // uint64[n_sets]

    // greedy / index
    DevBuf counts;     // int32[n]
    DevBuf node_off;   // uint64[n+1]
    DevBuf cursor;     // uint32[n]
    DevBuf node_sets;  // uint32[members]
    DevBuf covered;    // uint8[n_sets]
    DevBuf chosen;     // uint8[n]
    DevBuf best;       // uint64[k]
    DevBuf seed_mark;  // uint32 bitmap[n/32 + 1]
    DevBuf seeds_dev;  // int32[n]
    DevBuf greedy_bar; // grid barrier of the cooperative greedy launch
    DevBuf greedy_chunks;  // cooperative greedy: member chunks of the round's large sets
    DevBuf greedy_nchunk;  // and their count per round

    // sets handed from tier 1 to tier 2 and from tier 2 to tier 3 of the sampler
    DevBuf ovf_list;    // uint32 set index
    DevBuf ovf_list2;   // uint32 set index
    DevBuf hand;        // IC: pass-1 state of the sets handed to pass 2
    DevBuf hand2;       // IC: pass-2 state of the sets handed to the heavy pass
    DevBuf arena;       // tier-2 per-warp hash + queue
    bool arena_clean = false;
    DevBuf lt_col;      // tier-1 LT: member columns, one per thread
    DevBuf big_bitmap;  // tier-3 LT: uint32[slots * words]
    DevBuf big_queue;   // tier-3 LT: uint32[slots * n]
    bool big_bitmap_clean = false;

    // batched second pass for heavy IC sets (sample_bulk.cu)
    DevBuf bulk_bitmap, bulk_slot, bulk_F, bulk_M, bulk_ng, bulk_gp, bulk_scal;
    DevBuf bulk_bsum, bulk_bar;  // persistent launch: per-block sums, grid barrier
    // run the heavy-set levels as host-stepped launches instead of one persistent launch
    bool bulk_stepped = false;
    bool bulk_bitmap_clean = false;
    uint64_t bulk_fcap = 0, bulk_mcap = 0;
    uint64_t bulk_budget = 0;  // bytes of visited bitmaps a heavy-pass batch may use
    // IC first pass: a warp gives a set to the second pass once its examined in-edges
    // would exceed this many
    unsigned long long width_budget = 16384;
    // IC second pass: a team gives a set to the heavy-set pass once its examined
    // in-edges would exceed this many
    unsigned long long width_budget2 = ~0ull;
    // IC tier 2: warps per RR set (1, 2, 4 or 8); 0 = chosen from the number of sets:
    // the smallest T with listed * team_factor >= resident warps / T (at most 8)
    int team_size = 0;
    int team_factor = 2;
    // IC tier 1: queue capacity of one warp's set (128, 256 or 512 members)
    int cap1 = 256;
    // sets claimed per work-counter increment in tiers 1 and 2
    int chunk = 2;
    // set-id tag of this context's runs: ids are (phase << 56) | (round << 48) |
    // (tag << 32) | j
    uint32_t query_tag = 0;
    // polls a block makes at a grid barrier of a persistent kernel before it gives up
    // (the call then fails with TIM_ERR_TIMEOUT)
    unsigned wait_limit = 1u << 24;
    // batch scratch (owner of a multi-query launch / batched greedy)
    DevBuf batch, greedy_batch;
    int last_team = 1;

    // graph-load temporaries (graph.cu), kept between loads
    DevBuf ld_keys, ld_vals, ld_lt_t, ld_lt_e, ld_nonuni, ld_srcof;
    DevBuf ld_posof;  // triggering model: in-CSR position of every out-CSR edge
    DevBuf ld_in_r, ld_in_d, ld_in_w;  // device copies of tim_load_graph's host arrays

    // forward cascades (spread.cu): G as out-records {in-CSR position, destination},
    // built from G^T on first use; per-block visited bitmaps (kept all-zero between
    // calls) and queues; cascade counts, seeds, counters
    DevBuf out_rowptr, out_rec, mc_bitmap, mc_queue, mc_counts, mc_seeds, mc_scal;
    bool have_out = false, mc_clean = false;

    // generic scratch for scans and sorts
    DevBuf scratch_a, scratch_b, scratch_c, scratch_d, scratch_e, scratch_f;

    DevBuf scal;
    DevScalars* h_scal = nullptr;  // pinned

    cudaEvent_t ev[8] = {};
    cudaEvent_t kev[4] = {};  // around the sampler's three tiers
    cudaEvent_t bev[2] = {};  // around each persistent launch of the heavy-set pass

    // a stepwise greedy is open on the store (tim_select_begin)
    bool select_open = false;
    // state of the last tim_kpt_estimate
    bool have_kpt = false;
    int kpt_round = 0, kpt_last_round = 0;
    uint64_t kpt_last_c = 0;
    double kpt_star = 1.0;
    int kpt_k = 0;
    double kpt_ell = 0.0;
    uint64_t kpt_seed = 0;
    uint64_t kpt_sets = 0, kpt_width = 0;

    // pooled graph features of the learned start round (learned.cu), cached per graph
    bool have_feat = false;
    float feat[TIM_GRAPH_FEATURES] = {};

    // kernel timing of the RR sampler (events around each launch)
    tim_profile prof = {};

    // state of the last tim_refine_kpt
    double ref_kpt_prime = 0.0, ref_kpt_plus = 0.0, ref_eps_prime = 0.0;
    uint64_t ref_theta_prime = 0, ref_covered = 0, ref_width = 0;
};

#define TIM_TRY(expr)                   \
    do {                                \
        int _rc = (expr);               \
        if (_rc != TIM_OK) return _rc;  \
    } while (0)

int tim_fail(tim_ctx* ctx, int code, const std::string& msg);
int tim_cuda_check(tim_ctx* ctx, cudaError_t e, const char* what);
#define CUDA_TRY(ctx, call) TIM_TRY(tim_cuda_check((ctx), (call), #call))
// After a kernel launch: count it and check the launch status.
#define LAUNCH_CHECK(ctx, name)                                  \
    do {                                                         \
        (ctx)->launches++;                                       \
        TIM_TRY(tim_cuda_check((ctx), cudaGetLastError(), name)); \
    } while (0)

int tim_ensure(tim_ctx* ctx, DevBuf& b, size_t bytes);
void tim_free(DevBuf& b);
int tim_sync(tim_ctx* ctx);
int tim_read_scalars(tim_ctx* ctx);  // copy DevScalars to h_scal and synchronise
int tim_zero_scalars(tim_ctx* ctx);
DevScalars* tim_dscal(tim_ctx* ctx);

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Set id of the j-th RR set of `round` in `phase` (the tag sits in bits 32..47 of j).
static inline uint64_t make_sid(uint64_t phase, uint64_t round, uint64_t j) {
    return (phase << 56) | (round << 48) | j;
}

// primitives (prims.cu)
// Exclusive scan of uint32 counts into uint64 offsets out[0..count] (out[count] = total).
int tim_scan_u32_to_u64(tim_ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t count);
// The same for uint64 counts (sums must stay below 2^64).
int tim_scan_u64(tim_ctx* ctx, const unsigned long long* in, uint64_t* out, uint64_t count);
// Stable LSD radix sort of (key, a, b) uint32 triples by the low `bits` bits of key,
// in place (alternate buffers are taken from scratch).
int tim_radix_sort_triples(tim_ctx* ctx, uint32_t* keys, uint32_t* va, uint32_t* vb,
                           uint64_t count, int bits);
// The same, the first pass reading (k0, a0, b0) (which may be the destination arrays);
// the sorted triples end in (keys, va, vb).
int tim_radix_sort_triples_from(tim_ctx* ctx, const uint32_t* k0, const uint32_t* a0,
                                const uint32_t* b0, uint32_t* keys, uint32_t* va, uint32_t* vb,
                                uint64_t count, int bits);

// graph.cu
int tim_graph_build(tim_ctx* ctx, int64_t n, int64_t m, const int64_t* d_rowptr,
                    const int32_t* d_dst, const float* d_w, int model);
// Triggering options on the graph just built (model TIM_TRIG): cumulative thresholds and
// in-CSR positions (ascending within each option) into the context (node_opt, opt_off,
// opt_pos already hold the offsets and room for the n_ent positions).
int tim_trig_build(tim_ctx* ctx, const int32_t* d_out_dst, const uint64_t* d_node_opt,
                   const float* d_opt_prob, uint64_t n_opts, const uint64_t* d_opt_off,
                   const int64_t* d_opt_edges, uint64_t n_ent);

// sample.cu
enum : int { SAMPLE_EMIT = 1, SAMPLE_KAPPA = 2, SAMPLE_COVER = 4 };
struct SampleRequest {
    uint64_t seed = 0;
    uint64_t sid0 = 0;
    uint64_t count = 0;
    int flags = 0;
    int k = 0;                         // kappa
    const uint32_t* seed_mark = nullptr;  // cover: bitmap of the seed set
};
struct SampleResult {
    unsigned __int128 ksum = 0;
    uint64_t wsum = 0;
    uint64_t live = 0;
    uint64_t covered = 0;
    uint64_t members = 0;
    uint64_t big_sets = 0;
};
int tim_sample(tim_ctx* ctx, const SampleRequest& req, SampleResult* res);
// Third tier for the heavy IC sets list[0 .. count) (sample_bulk.cu). With hand (may be
// null), the set at list position i < hcap starts from the state pass 2 left at
// hand + i hw: queue length, position of the batch to redo, then the queue.
int tim_bulk_ic(tim_ctx* ctx, const SampleRequest& req, const uint32_t* list, uint32_t count,
                uint32_t* pool, uint32_t* pool_sid, uint64_t pool_cap, DevScalars* ds,
                uint64_t* live_out, const uint32_t* hand = nullptr, uint32_t hcap = 0,
                uint32_t hw = 0);

// Several queries, each with its own context (graph, RR-set store), sampled by one
// launch per tier; all share the Philox key of `seed` and use the owner's stream and
// scratch. Per-query results in qs[i].res.
struct MultiQuery {
    tim_ctx* ctx = nullptr;
    SampleRequest req;
    SampleResult res;
};
int tim_sample_multi(tim_ctx* owner, MultiQuery* qs, int nq, uint64_t seed);

// select.cu
int tim_build_index(tim_ctx* ctx);
int tim_greedy(tim_ctx* ctx, int k, int32_t* host_seeds, uint64_t* covered);
int tim_mark_seeds(tim_ctx* ctx, const int32_t* d_seeds, int k);
// Stepwise greedy on the store: index and reset, then one caller-chosen node at a time.
int tim_greedy_begin(tim_ctx* ctx);
int tim_greedy_take(tim_ctx* ctx, int32_t v, uint64_t* newly_covered);
// Greedy of Algorithm 1 for several queries (each on its own context's store) with
// shared launches, optionally captured into one CUDA graph; seeds stay in each
// context's seeds_dev, host copies where host_seeds[i] is not NULL.
int tim_greedy_batch(tim_ctx* owner, tim_ctx* const* ctxs, const int* ks, int nq,
                     int32_t* const* host_seeds, uint64_t* covered, bool use_graph);

// learned.cu: start rounds i0 of Algorithm 2 predicted for ctxs[q] with k = ks[q]
int tim_learned_start_rounds(tim_mlp* mlp, tim_ctx* const* ctxs, const int* ks, int nq,
                             int* i0);

// scalar formulas (api.cu)
uint64_t tim_host_c_i(int64_t n, double ell, int i);
int tim_host_rounds(int64_t n);
double tim_host_lambda(int64_t n, int k, double eps, double ell);
double tim_host_eps_prime(double eps, int k, double ell);
double tim_host_lambda_prime(int64_t n, double eps_p, double ell);

// ---------------------------------------------------------------- device side

#define TIM_PHILOX_M0 0xD2511F53u
#define TIM_PHILOX_M1 0xCD9E8D57u
#define TIM_PHILOX_W0 0x9E3779B9u
#define TIM_PHILOX_W1 0xBB67AE85u

#define TIM_TAG_ROOT 0u
#define TIM_TAG_IC 1u
#define TIM_TAG_LT 2u
#define TIM_TAG_SKIP 0x100u  // + gap digit index b, 0..31
// shortest IC in-list sampled by geometric skipping (tim_skip_rule)
#define TIM_SKIP_MIN_INDEG 512u

// Philox round keys for one seed: key schedule k_r = k_0 + r * W, r = 0..9.
struct PhiloxKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

static inline PhiloxKeys tim_philox_keys(uint64_t seed) {
    PhiloxKeys K;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; r++) {
        K.k0[r] = a;
        K.k1[r] = b;
        a += TIM_PHILOX_W0;
        b += TIM_PHILOX_W1;
    }
    return K;
}

#ifdef __CUDACC__
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies and xors with the precomputed round keys.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                               uint32_t c3, const PhiloxKeys& K) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        unsigned long long p0 = (unsigned long long)c0 * TIM_PHILOX_M0;
        unsigned long long p1 = (unsigned long long)c2 * TIM_PHILOX_M1;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[r];
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Geometric-skip rule for IC in-lists. A list of d in-edges whose in-edges all carry
// one threshold t (per-node word nt: bit 32 set, low word t) takes the rule when
// d >= TIM_SKIP_MIN_INDEG, t > 0 and t (2 bitlength(d) + 2) < 2^32: a few geometric
// gaps then replace many coins. Each in-edge is still live with probability t / 2^32,
// independently, as with one coin per edge.
//   The gap G (dead in-edges before the next live one) has P(G >= g) = q^g, q = 1 - p.
// Since sum_g q^g = prod_b (1 + q^(2^b)), the binary digits of G are independent,
// digit b being 1 with probability q^(2^b) / (1 + q^(2^b)), and G >= 2^B has
// probability q^(2^B). With Q_b ~ q^(2^b) 2^64 (Q_0 = (2^32 - t) 2^32 exactly,
// Q_(b+1) = floor(Q_b^2 / 2^64)) a 64-bit uniform U decides digit b as
//   U (2^64 + Q_b) < Q_b 2^64  <=>  U < Q_b and floor(U Q_b / 2^64) < Q_b - U,
// and G >= 2^B (B = bit length of the R in-edges left, so 2^B > R) as U < Q_B.
// U for digit b of gap r = words (2(r&1), 2(r&1)+1) of Philox counter (sid lo,
// sid hi, beg + (r >> 1), TIM_TAG_SKIP + b); beg = in-CSR position of the list's first
// in-edge (r <= pos < d keeps beg + (r >> 1) inside the list). G >= R or G >= 2^B ends
// the list; otherwise position pos + G is live and the next gap starts after it.
__device__ __forceinline__ bool tim_skip_rule(unsigned long long nt, unsigned long long d) {
    const uint32_t t = (uint32_t)nt;
    if (!(nt >> 32) || t == 0u || d < TIM_SKIP_MIN_INDEG) return false;
    const int bl = 64 - __clzll((long long)d);
    return (unsigned long long)t * (unsigned long long)(2 * bl + 2) < 0x100000000ull;
}

__device__ __forceinline__ bool skip_digit(unsigned long long U, unsigned long long Q) {
    return U < Q && __umul64hi(U, Q) < Q - U;
}

// The gap table of a node under the rule: Q_b for b = 0..31, computed at load.
__device__ __forceinline__ const unsigned long long* skip_table(const unsigned long long* qtab,
                                                                unsigned long long nt) {
    return qtab + ((nt >> 33) - 1ull) * 32ull;
}

// Live in-edges of a list under the rule, warp-cooperatively: lane b decides digit b
// of each gap (Q_b from the node's table), one ballot gives G; a lane's draw for gap 2i
// also serves gap 2i + 1. visit(j) runs on every lane with the same in-CSR position j
// of each live in-edge, in increasing order, and returns true to stop early. All 32
// lanes must call it with the same arguments.
template <class Visit>
__device__ __forceinline__ void skip_live_warp(uint32_t s0, uint32_t s1, const PhiloxKeys& K,
                                               uint32_t beg, uint32_t d,
                                               const unsigned long long* qtab_node, int lane,
                                               Visit&& visit) {
    const int bmax = 32 - __clz((int)d);
    const unsigned long long Q = lane <= bmax && lane < 32 ? __ldg(qtab_node + lane) : 0ull;
    uint4 x = make_uint4(0u, 0u, 0u, 0u);
    uint32_t pos = 0;
    for (uint32_t r = 0; pos < d; r++) {
        const uint32_t rem = d - pos;
        const int B = 32 - __clz((int)rem);
        // B never grows along a list, so the lanes gap 2i + 1 needs drew for gap 2i
        if ((r & 1u) == 0u && lane <= B)
            x = philox4x32_10(s0, s1, beg + (r >> 1), TIM_TAG_SKIP + (uint32_t)lane, K);
        const unsigned long long U = (r & 1u) ? (((unsigned long long)x.w << 32) | x.z)
                                             : (((unsigned long long)x.y << 32) | x.x);
        const bool digit = lane < B && skip_digit(U, Q);
        const bool over = lane == B && U < Q;
        const uint32_t G = __ballot_sync(0xffffffffu, digit);
        if (__any_sync(0xffffffffu, over) || G >= rem) break;
        if (visit(beg + pos + G)) break;
        pos += G + 1u;
    }
}

// Uniform root: floor(x * n / 2^64) with x the first two words of the ROOT draw.
// LT triggering pick when all in-edges of v carry the same t = floor(b 2^32) (per-node
// word nt: bit 32 set, low word t): the cumulative thresholds are C_j = min((j + 1) t,
// 2^32 - 1), so the first j with x < C_j is floor(x / t) when that is below d and
// x < 2^32 - 1 (C never exceeds 2^32 - 1), and there is none otherwise -- the same
// in-edge as the search over C. Returns the in-CSR position, or end for none.
__device__ __forceinline__ uint64_t lt_uniform_pick(unsigned long long nt, uint64_t beg,
                                                    uint64_t end, uint32_t x) {
    const uint32_t t = (uint32_t)nt;
    if (t == 0u || x == 0xFFFFFFFFu) return end;
    const uint64_t q = x / t;
    return q < end - beg ? beg + q : end;
}

// First position j in [lo, hi) with thr[j] > x, by one thread.
__device__ __forceinline__ uint64_t lane_lt_search(const uint32_t* __restrict__ thr, uint64_t lo,
                                                   uint64_t hi, uint32_t x) {
    for (int it = 0; it < 40 && lo < hi; it++) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(thr + mid) > x)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ uint32_t rr_root(uint64_t sid, uint64_t n, const PhiloxKeys& K) {
    uint4 w = philox4x32_10((uint32_t)sid, (uint32_t)(sid >> 32), 0u, TIM_TAG_ROOT, K);
    unsigned long long x = ((unsigned long long)w.y << 32) | w.x;
    return (uint32_t)__umul64hi(x, (unsigned long long)n);
}

// kappa(R) of Eq. 6 as (w/m) * sum_{i<k} q^i, q = 1 - w/m, built over the bits of k
// (S_2j = S_j (1 + P_j), P_2j = P_j^2; set bit: S += P, P *= q). Every operation is
// an explicitly rounded FP64 intrinsic so that nothing is contracted into an FMA.
__device__ __forceinline__ double kappa_fp64(unsigned long long w, unsigned long long m, int k) {
    if (m == 0 || w == 0 || k <= 0) return 0.0;
    double x = __ddiv_rn((double)w, (double)m);
    double q = __dsub_rn(1.0, x);
    double S = 0.0, P = 1.0;
    int top = 31 - __clz(k);
    for (int b = top; b >= 0; b--) {
        S = __dmul_rn(S, __dadd_rn(1.0, P));
        P = __dmul_rn(P, P);
        if ((k >> b) & 1) {
            S = __dadd_rn(S, P);
            P = __dmul_rn(P, q);
        }
    }
    return __dmul_rn(x, S);
}

// kappa in 2^-63 fixed point, truncated toward zero.
__device__ __forceinline__ unsigned long long kappa_fixed(double kappa) {
    return __double2ull_rz(__dmul_rn(kappa, 9223372036854775808.0));
}

// Barrier over all blocks of a co-resident (cooperative) launch: sense reversal on a
// generation counter, which the host zeroes before each launch. The wait is bounded:
// after `limit` polls a block sets TIM_DEV_ERR_TIMEOUT in *err and the barrier returns
// false; it also returns false once any block has set that bit, so every block of the
// launch stops within one barrier of the first timeout.
struct GridBarrier {
    unsigned count;
    unsigned gen;
};

__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, int* err, unsigned limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned g = ((volatile unsigned*)&bar->gen)[0];
        if (atomicAdd(&bar->count, 1u) == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            unsigned it = 0;
            while (((volatile unsigned*)&bar->gen)[0] == g && it < limit) {
                __nanosleep(64);
                it++;
            }
            if (((volatile unsigned*)&bar->gen)[0] == g) {
                atomicOr(err, TIM_DEV_ERR_TIMEOUT);
                ok = 0;
            }
        }
        __threadfence();
        s_ok = ok && !(((volatile int*)err)[0] & TIM_DEV_ERR_TIMEOUT);
    }
    __syncthreads();
    return s_ok != 0;
}

// Add a 128-bit (hi, lo) into a global 128-bit accumulator.
__device__ __forceinline__ void atomic_add_u128(unsigned long long* lo_p,
                                                unsigned long long* hi_p,
                                                unsigned long long lo, unsigned long long hi) {
    unsigned long long old = atomicAdd(lo_p, lo);
    unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(hi_p, hi + carry);
}
#endif
