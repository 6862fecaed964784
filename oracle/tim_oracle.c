/*
 * tim_oracle.c -- plain CPU oracle for TIM / TIM+ (Tang, Xiao, Shi, "Influence
 * Maximization: Near-Optimal Time Complexity Meets Practical Efficiency", SIGMOD'14).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark load this file. The GPU library never includes, links or calls
 * it, and it never calls the GPU library: the two share no code.
 *
 * Every routine is a direct, slow restatement of the paper's definitions and
 * algorithms in the paper's order, written for readability:
 *   - IC model and RR sets: Section 2.1, Definitions 1-2 (Section 2.3).
 *   - RR-set generation by randomised BFS: Section 3.1 ("Implementation").
 *   - Width w(R): Eq. 1.  kappa(R): Eq. 6 (Lemma 5).
 *   - NodeSelection: Algorithm 1.  KptEstimation: Algorithm 2, c_i of Eq. 7.
 *   - lambda: Eq. 4.  theta = lambda / KPT: Section 3.3 and Eq. 5.
 *   - RefineKPT: Algorithm 3; eps' of Section 4.1; TIM+ of Section 4.1.
 *   - Triggering / LT RR sets: Section 4.2 and the LT setting of Section 6.
 *
 * Readings of points the paper leaves open (all shared with the GPU library by
 * specification only, never by code):
 *   - Randomness: Philox4x32-10 (Salmon et al., SC'11), key = 64-bit seed,
 *     counter = (set id lo, set id hi, element, tag). IC coin of in-CSR position j:
 *     word (j & 3) of counter (sid, j >> 2, TAG_IC). LT draw of node v: word 0 of
 *     counter (sid, v, TAG_LT). Root: words 0,1 of (sid, 0, TAG_ROOT) form a 64-bit
 *     x and root = floor(x * n / 2^64).
 *   - In-CSR order: in-edges of v ascending by source id (a stable counting sort of
 *     the out-CSR edges by destination).
 *   - IC coin: live iff x < thr, thr = floor(p * 2^32) for p < 1; p >= 1 is stored as
 *     0xFFFFFFFF and is always live.
 *   - IC in-lists of d >= SKIP_MIN_INDEG in-edges that all carry one threshold t with
 *     0 < t and t * (2 * bitlength(d) + 2) < 2^32 (weighted cascade gives every such
 *     node one): instead of one coin per in-edge, the live in-edges are found by
 *     drawing the geometric gaps between them (see skip_iter below). Each in-edge is
 *     still live with probability t / 2^32, independently (to within 2^-60 per gap
 *     digit). The bound on t keeps the rule to lists where a few gaps replace many
 *     coins. This rule and its random-number layout are frozen: the law of the
 *     sets it gives is checked against the per-edge mode (one coin per in-edge in
 *     every list, Section 3.1 as printed; or_sample_mode with per_edge = 1) by
 *     whole-graph statistics, and any change to either lands in an oracle-only change
 *     with its pins before a kernel follows it.
 *   - LT pick: t_j = floor(w_j * 2^32); C_j = inclusive prefix of t over v's
 *     in-edges in in-CSR order, saturated at 2^32 - 1; the first j with x < C_j is
 *     the triggering in-edge, none if x >= C_last.
 *   - kappa in FP64 as (w/m) * sum_{i<k} q^i with q = 1 - w/m (the geometric-series
 *     form of Eq. 6, free of cancellation), built by binary doubling over k;
 *     sum of kappa over a round in 2^-63 fixed point (each kappa truncated once,
 *     then an exact 128-bit integer sum); the stop test is done in integers.
 *   - Loop bound of Algorithm 2: i = 1 .. floor(log2 n) - 1; c_i rounded up.
 *   - theta, theta' rounded up.
 *   - Greedy ties: largest count, then smallest node id; chosen nodes excluded.
 *   - Set ids: sid = (phase << 56) | (round << 48) | (tag << 32) | j, with phase 1 =
 *     KptEstimation, 2 = RefineKPT's theta' sets, 3 = NodeSelection; the tag (0 by
 *     default) separates queries that share a seed.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC.
 * Floating point contraction must stay off so that every FP64 operation is a single
 * IEEE-rounded step, as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_OOM (-2)
#define OR_ERR_CAP (-3)

#define TAG_ROOT 0u
#define TAG_IC 1u
#define TAG_LT 2u
#define TAG_SKIP 0x100u /* + digit index b, 0..31 */
#define SKIP_MIN_INDEG 512

#define MODEL_IC 0
#define MODEL_LT 1
#define MODEL_TRIG 2

#define PHASE_KPT 1ull
#define PHASE_REFINE 2ull
#define PHASE_SELECT 3ull

/* ------------------------------------------------------------------ Philox */
/* Philox4x32-10 as published by Salmon, Moraes, Dror and Shaw (SC'11): ten rounds
 * of two 32x32->64 multiplications with a Weyl-sequence key schedule. */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k[0] += 0x9E3779B9u; /* golden ratio - 1, times 2^32 */
            k[1] += 0xBB67AE85u; /* sqrt(3) - 1, times 2^32 */
        }
        philox_round(c, k);
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

static void draw(uint64_t seed, uint64_t sid, uint32_t elem, uint32_t tag, uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)sid, (uint32_t)(sid >> 32), elem, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

uint64_t or_make_sid(uint64_t phase, uint64_t round, uint64_t j) {
    return (phase << 56) | (round << 48) | j;
}

/* Root of a random RR set: a node chosen uniformly at random (Definition 2). */
int64_t or_root(uint64_t seed, uint64_t sid, int64_t n) {
    uint32_t w[4];
    draw(seed, sid, 0u, TAG_ROOT, w);
    uint64_t x = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
    return (int64_t)(((u128)x * (u128)(uint64_t)n) >> 64);
}

/* IC coin word for in-CSR position j of RR set sid. */
uint32_t or_ic_word(uint64_t seed, uint64_t sid, int64_t j) {
    uint32_t w[4];
    draw(seed, sid, (uint32_t)((uint64_t)j >> 2), TAG_IC, w);
    return w[(uint64_t)j & 3u];
}

/* LT draw of node v for RR set sid. */
uint32_t or_lt_word(uint64_t seed, uint64_t sid, int64_t v) {
    uint32_t w[4];
    draw(seed, sid, (uint32_t)v, TAG_LT, w);
    return w[0];
}

/* ------------------------------------------------------------------ graph */
/* Transpose G^T (Table 1) as an in-CSR: for every node v its in-edges, ascending by
 * source. Validates the out-CSR: sorted offsets, ids in range, no self-loops, no
 * duplicate edges. The in-weights are permuted along with the edges. */
int or_transpose(int64_t n, int64_t m, const int64_t* out_rowptr, const int32_t* out_dst,
                 const float* out_w, int64_t* in_rowptr, int32_t* in_src, float* in_w) {
    if (n < 1 || m < 0 || out_rowptr[0] != 0 || out_rowptr[n] != m) return OR_ERR_ARG;
    for (int64_t u = 0; u < n; u++)
        if (out_rowptr[u + 1] < out_rowptr[u]) return OR_ERR_ARG;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return OR_ERR_OOM;
    for (int64_t u = 0; u < n; u++) {
        for (int64_t e = out_rowptr[u]; e < out_rowptr[u + 1]; e++) {
            int64_t v = out_dst[e];
            if (v < 0 || v >= n || v == u) {
                free(cnt);
                return OR_ERR_ARG;
            }
            cnt[v + 1]++;
        }
    }
    in_rowptr[0] = 0;
    for (int64_t v = 0; v < n; v++) in_rowptr[v + 1] = in_rowptr[v] + cnt[v + 1];
    for (int64_t v = 0; v < n; v++) cnt[v] = in_rowptr[v];
    /* Visiting edges in out-CSR order (ascending source) keeps each in-list sorted
     * by source. */
    for (int64_t u = 0; u < n; u++) {
        for (int64_t e = out_rowptr[u]; e < out_rowptr[u + 1]; e++) {
            int64_t v = out_dst[e];
            int64_t pos = cnt[v]++;
            in_src[pos] = (int32_t)u;
            in_w[pos] = out_w ? out_w[e] : 0.0f;
        }
    }
    free(cnt);
    /* duplicates: equal neighbouring sources inside one in-list */
    for (int64_t v = 0; v < n; v++)
        for (int64_t j = in_rowptr[v] + 1; j < in_rowptr[v + 1]; j++)
            if (in_src[j] == in_src[j - 1]) return OR_ERR_ARG;
    return OR_OK;
}

/* Triggering distribution on G^T from its description on G: node v has options
 * opt_rowptr[v] .. opt_rowptr[v+1]; option o has probability opt_prob[o] and the
 * out-CSR edge ids opt_edges[opt_edge_rowptr[o] .. opt_edge_rowptr[o+1]), each an edge
 * into v, distinct within the option. Writes the options' cumulative thresholds
 * (inclusive prefix of floor(pi * 2^32) over v's options, saturated at 2^32 - 1) and their
 * in-CSR positions. The in-CSR position of an out-edge is found by replaying the
 * transpose: in-lists are filled in out-CSR order. A node's probabilities must lie in
 * [0, 1] and sum to at most 1 + 1e-5. */
int or_trig_build(int64_t n, int64_t m, const int64_t* out_rowptr, const int32_t* out_dst,
                  const int64_t* in_rowptr, const int64_t* opt_rowptr, const float* opt_prob,
                  const int64_t* opt_edge_rowptr, const int64_t* opt_edges, uint32_t* opt_cum,
                  int64_t* opt_pos) {
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!pos || !cur) {
        free(pos);
        free(cur);
        return OR_ERR_OOM;
    }
    for (int64_t v = 0; v <= n; v++) cur[v] = v < n ? in_rowptr[v] : 0;
    for (int64_t u = 0; u < n; u++)
        for (int64_t e = out_rowptr[u]; e < out_rowptr[u + 1]; e++) pos[e] = cur[out_dst[e]]++;
    free(cur);
    int rc = OR_OK;
    if (opt_rowptr[0] != 0) rc = OR_ERR_ARG;
    for (int64_t v = 0; v < n && rc == OR_OK; v++) {
        if (opt_rowptr[v + 1] < opt_rowptr[v]) {
            rc = OR_ERR_ARG;
            break;
        }
        double tot = 0.0;
        uint64_t acc = 0;
        for (int64_t o = opt_rowptr[v]; o < opt_rowptr[v + 1] && rc == OR_OK; o++) {
            double p = (double)opt_prob[o];
            if (!(p >= 0.0 && p <= 1.0) || opt_edge_rowptr[o + 1] < opt_edge_rowptr[o]) {
                rc = OR_ERR_ARG;
                break;
            }
            tot += p;
            acc += (uint64_t)floor(p * 4294967296.0);
            opt_cum[o] = acc > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)acc;
            for (int64_t i = opt_edge_rowptr[o]; i < opt_edge_rowptr[o + 1]; i++) {
                int64_t e = opt_edges[i];
                if (e < 0 || e >= m || out_dst[e] != v) {
                    rc = OR_ERR_ARG;
                    break;
                }
                opt_pos[i] = pos[e];
                for (int64_t i2 = opt_edge_rowptr[o]; i2 < i; i2++)
                    if (opt_edges[i2] == e) rc = OR_ERR_ARG;  /* repeated edge */
            }
        }
        if (tot > 1.0 + 1e-5) rc = OR_ERR_ARG;
    }
    free(pos);
    return rc;
}

/* IC live-edge threshold of each in-edge: live iff word < thr (p >= 1: always). */
int or_ic_thresholds(int64_t m, const float* in_w, uint32_t* thr) {
    for (int64_t j = 0; j < m; j++) {
        double p = (double)in_w[j];
        if (!(p >= 0.0 && p <= 1.0)) return OR_ERR_ARG;
        if (p >= 1.0)
            thr[j] = 0xFFFFFFFFu;
        else
            thr[j] = (uint32_t)floor(p * 4294967296.0);
    }
    return OR_OK;
}

/* LT cumulative thresholds (inclusive, saturated at 2^32 - 1) per in-list. */
int or_lt_thresholds(int64_t n, const int64_t* in_rowptr, const float* in_w, uint32_t* cum) {
    for (int64_t v = 0; v < n; v++) {
        double tot = 0.0;
        uint64_t acc = 0;
        for (int64_t j = in_rowptr[v]; j < in_rowptr[v + 1]; j++) {
            double w = (double)in_w[j];
            if (!(w >= 0.0 && w <= 1.0)) return OR_ERR_ARG;
            tot += w;
            acc += (uint64_t)floor(w * 4294967296.0);
            cum[j] = acc > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)acc;
        }
        if (tot > 1.0 + 1e-5) return OR_ERR_ARG;
    }
    return OR_OK;
}

/* A triggering model (Section 4.2) on G^T: node v picks option o in node_opt[v] ..
 * node_opt[v+1] with probability pi_o (none with the rest); option o activates v through
 * the in-edges at in-CSR positions opt_pos[opt_off[o] .. opt_off[o+1]). opt_cum holds the
 * inclusive prefix of floor(pi * 2^32) over v's options, saturated at 2^32 - 1. */
typedef struct {
    const int64_t* node_opt;
    const uint32_t* opt_cum;
    const int64_t* opt_off;
    const int64_t* opt_pos;
} or_trig;

typedef struct {
    int64_t n, m;
    const int64_t* rowptr; /* in-CSR offsets, n+1 */
    const int32_t* src;    /* in-CSR sources, m */
    const uint32_t* thr;   /* IC thresholds or LT cumulative thresholds, m */
    int model;
    int per_edge; /* 1: one coin per in-edge in every IC list (no geometric skipping) */
    const or_trig* trig; /* MODEL_TRIG only */
} or_graph;

static int64_t indeg(const or_graph* g, int64_t v) { return g->rowptr[v + 1] - g->rowptr[v]; }

static int ic_live(uint32_t x, uint32_t thr) { return thr == 0xFFFFFFFFu || x < thr; }

/* ------------------------------------------------ geometric skipping (IC)
 * For an in-list of d in-edges that are each live with probability p = t / 2^32,
 * independently, the number G of dead in-edges before the next live one is
 * geometric: P(G >= g) = q^g with q = 1 - p. Since sum_g q^g = prod_b (1 + q^(2^b)),
 *   P(G = g) = (1 - q) q^g = prod_b q^(2^b g_b) / (1 + q^(2^b))
 * for the binary digits g_b of g: the digits are independent, digit b being 1 with
 * probability rho_b = q^(2^b) / (1 + q^(2^b)), and "some digit >= B is 1", i.e.
 * G >= 2^B, has probability q^(2^B).
 *
 * Fixed point: Q_b approximates q^(2^b) 2^64; Q_0 = (2^32 - t) 2^32 is exact and
 * Q_(b+1) = floor(Q_b^2 / 2^64). A 64-bit uniform U decides digit b as
 *   U / 2^64 < Q_b / (2^64 + Q_b)  <=>  U < Q_b  and  floor(U Q_b / 2^64) < Q_b - U,
 * and "G >= 2^B" as U < Q_B.
 *
 * Gap r of a list starts at relative position pos (< d); R = d - pos remaining,
 * B = bit length of R (so 2^B > R). Uniform U_b (b = 0 .. B) = words (2(r&1),
 * 2(r&1)+1) (low, high) of Philox counter (sid lo, sid hi, beg + (r >> 1), TAG_SKIP +
 * b), beg = in-CSR position of the list's first in-edge: one draw per digit serves two
 * consecutive gaps. If G >= 2^B or G >= R the list has no further live in-edge; else
 * position pos + G is live and the next gap starts at pos + G + 1. (r <= pos < d keeps
 * beg + (r >> 1) inside the list, so no two lists share a counter.) */
uint64_t or_skip_q(uint32_t t, int b) {
    uint64_t q = (uint64_t)(0x100000000ull - (uint64_t)t) << 32;
    for (int i = 0; i < b; i++) q = (uint64_t)(((u128)q * q) >> 64);
    return q;
}

int or_skip_bit(uint64_t u, uint64_t q) {
    return u < q && (uint64_t)(((u128)u * q) >> 64) < q - u;
}

typedef struct {
    uint64_t seed, sid;
    int64_t beg, d, pos, r;
    uint64_t q[33];
} skip_iter;

static void skip_begin(skip_iter* it, uint64_t seed, uint64_t sid, int64_t beg, int64_t d,
                       uint32_t t) {
    it->seed = seed;
    it->sid = sid;
    it->beg = beg;
    it->d = d;
    it->pos = 0;
    it->r = 0;
    it->q[0] = (uint64_t)(0x100000000ull - (uint64_t)t) << 32;
    for (int b = 1; b < 33; b++) it->q[b] = (uint64_t)(((u128)it->q[b - 1] * it->q[b - 1]) >> 64);
}

static uint64_t skip_uniform(const skip_iter* it, int b) {
    uint32_t w[4];
    draw(it->seed, it->sid, (uint32_t)(it->beg + (it->r >> 1)), TAG_SKIP + (uint32_t)b, w);
    return (it->r & 1) ? ((uint64_t)w[3] << 32 | w[2]) : ((uint64_t)w[1] << 32 | w[0]);
}

/* Next live relative position into *j; 0 when the list has no more. */
static int skip_next(skip_iter* it, int64_t* j) {
    if (it->pos >= it->d) return 0;
    int64_t rem = it->d - it->pos;
    int B = 0;
    while (B < 63 && ((int64_t)1 << B) <= rem) B++;
    if (skip_uniform(it, B) < it->q[B]) return 0;
    int64_t gap = 0;
    for (int b = 0; b < B; b++)
        if (or_skip_bit(skip_uniform(it, b), it->q[b])) gap |= (int64_t)1 << b;
    if (gap >= rem) return 0;
    *j = it->pos + gap;
    it->pos += gap + 1;
    it->r++;
    return 1;
}

/* Live relative positions of one skip list (tests); returns their number. */
int64_t or_skip_live(uint64_t seed, uint64_t sid, int64_t beg, int64_t d, uint32_t t,
                     int64_t* out) {
    if (d < 1 || d > 0x7FFFFFFF || t == 0u || t == 0xFFFFFFFFu) return OR_ERR_ARG;
    skip_iter it;
    skip_begin(&it, seed, sid, beg, d, t);
    int64_t n = 0, j;
    while (skip_next(&it, &j)) out[n++] = j;
    return n;
}

/* Does v's in-list take the skip rule? Then *t is its shared threshold. In the
 * per-edge mode no list does: every in-edge draws its own coin, as Section 3.1 states
 * the procedure. That mode exists only to check, by statistics over whole graphs, that
 * the skip rule gives RR sets of the same law; it is never compared with the GPU. */
static int skip_list(const or_graph* g, int64_t v, uint32_t* t) {
    if (g->model != MODEL_IC || g->per_edge) return 0;
    int64_t a = g->rowptr[v], b = g->rowptr[v + 1], d = b - a;
    if (d < SKIP_MIN_INDEG) return 0;
    uint32_t t0 = g->thr[a];
    int bl = 0;
    while (bl < 63 && ((int64_t)1 << bl) <= d) bl++;
    if (t0 == 0u || (uint64_t)t0 * (uint64_t)(2 * bl + 2) >= 0x100000000ull) return 0;
    for (int64_t j = a + 1; j < b; j++)
        if (g->thr[j] != t0) return 0;
    *t = t0;
    return 1;
}

/* LT triggering in-edge of v for RR set sid: an in-CSR position, or -1 for none. */
static int64_t lt_pick(const or_graph* g, uint64_t seed, uint64_t sid, int64_t v) {
    uint32_t x = or_lt_word(seed, sid, v);
    for (int64_t j = g->rowptr[v]; j < g->rowptr[v + 1]; j++)
        if (x < g->thr[j]) return j;
    return -1;
}

/* Triggering option of v for RR set sid (Section 4.2): the same draw as the LT pick,
 * the first option whose cumulative threshold exceeds it; -1 for none. */
static int64_t trig_pick(const or_graph* g, uint64_t seed, uint64_t sid, int64_t v) {
    uint32_t x = or_lt_word(seed, sid, v);
    for (int64_t o = g->trig->node_opt[v]; o < g->trig->node_opt[v + 1]; o++)
        if (x < g->trig->opt_cum[o]) return o;
    return -1;
}

/* One random RR set by randomised BFS from a uniform root (Section 3.1,
 * "Implementation"; triggering form of Section 4.2). members[] doubles as the BFS
 * queue; mark[] is an n-byte scratch array that is all-zero on entry and on exit.
 * Returns |R| and stores w(R) (Eq. 1). */
static int64_t rr_bfs(const or_graph* g, uint64_t seed, uint64_t sid, int32_t* members,
                      uint8_t* mark, int64_t* width) {
    int64_t root = or_root(seed, sid, g->n);
    int64_t head = 0, tail = 0, w = 0;
    members[tail++] = (int32_t)root;
    mark[root] = 1;
    while (head < tail) {
        int64_t v = members[head++];
        w += indeg(g, v);
        uint32_t t;
        if (g->model == MODEL_IC && skip_list(g, v, &t)) {
            skip_iter it;
            int64_t rel;
            skip_begin(&it, seed, sid, g->rowptr[v], indeg(g, v), t);
            while (skip_next(&it, &rel)) {
                int32_t u = g->src[g->rowptr[v] + rel];
                if (!mark[u]) {
                    mark[u] = 1;
                    members[tail++] = u;
                }
            }
        } else if (g->model == MODEL_IC) {
            for (int64_t j = g->rowptr[v]; j < g->rowptr[v + 1]; j++) {
                int32_t u = g->src[j];
                if (mark[u]) continue;
                if (ic_live(or_ic_word(seed, sid, j), g->thr[j])) {
                    mark[u] = 1;
                    members[tail++] = u;
                }
            }
        } else if (g->model == MODEL_TRIG) {
            int64_t o = trig_pick(g, seed, sid, v);
            if (o >= 0)
                for (int64_t e = g->trig->opt_off[o]; e < g->trig->opt_off[o + 1]; e++) {
                    int32_t u = g->src[g->trig->opt_pos[e]];
                    if (!mark[u]) {
                        mark[u] = 1;
                        members[tail++] = u;
                    }
                }
        } else {
            int64_t j = lt_pick(g, seed, sid, v);
            if (j >= 0) {
                int32_t u = g->src[j];
                if (!mark[u]) {
                    mark[u] = 1;
                    members[tail++] = u;
                }
            }
        }
    }
    for (int64_t i = 0; i < tail; i++) mark[members[i]] = 0;
    *width = w;
    return tail;
}

/* The same RR set straight from Definitions 1-2: draw the whole random graph g
 * first (every IC coin, or every node's LT triggering choice), keep its live edges
 * as a plain edge list, then take the closure "u can reach the root in g" by
 * repeated passes over that list until nothing changes. Independent of any search
 * order. Returns |R|; members are written in ascending id order. */
int64_t or_rr_by_definition_mode(const int64_t* rowptr, const int32_t* src,
                                 const uint32_t* thr, int64_t n, int64_t m, int model, const or_trig* trig,
                                 int per_edge, uint64_t seed, uint64_t sid, int32_t* members,
                                 int64_t* width) {
    or_graph g = {n, m, rowptr, src, thr, model, per_edge, trig};
    int64_t* lu = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t* lv = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    uint8_t* in_r = (uint8_t*)calloc((size_t)n, 1);
    if (!lu || !lv || !in_r) {
        free(lu);
        free(lv);
        free(in_r);
        return OR_ERR_OOM;
    }
    int64_t nl = 0;
    for (int64_t v = 0; v < n; v++) {
        uint32_t t;
        if (skip_list(&g, v, &t)) {
            skip_iter it;
            int64_t rel;
            skip_begin(&it, seed, sid, rowptr[v], rowptr[v + 1] - rowptr[v], t);
            while (skip_next(&it, &rel)) {
                lu[nl] = src[rowptr[v] + rel];
                lv[nl] = v;
                nl++;
            }
        } else if (model == MODEL_IC) {
            for (int64_t j = rowptr[v]; j < rowptr[v + 1]; j++)
                if (ic_live(or_ic_word(seed, sid, j), thr[j])) {
                    lu[nl] = src[j];
                    lv[nl] = v;
                    nl++;
                }
        } else if (model == MODEL_TRIG) {
            int64_t o = trig_pick(&g, seed, sid, v);
            if (o >= 0)
                for (int64_t e = trig->opt_off[o]; e < trig->opt_off[o + 1]; e++) {
                    lu[nl] = src[trig->opt_pos[e]];
                    lv[nl] = v;
                    nl++;
                }
        } else {
            int64_t j = lt_pick(&g, seed, sid, v);
            if (j >= 0) {
                lu[nl] = src[j];
                lv[nl] = v;
                nl++;
            }
        }
    }
    in_r[or_root(seed, sid, n)] = 1;
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int64_t e = 0; e < nl; e++)
            if (in_r[lv[e]] && !in_r[lu[e]]) {
                in_r[lu[e]] = 1;
                changed = 1;
            }
    }
    int64_t cnt = 0, w = 0;
    for (int64_t v = 0; v < n; v++)
        if (in_r[v]) {
            members[cnt++] = (int32_t)v;
            w += rowptr[v + 1] - rowptr[v];
        }
    *width = w;
    free(lu);
    free(lv);
    free(in_r);
    return cnt;
}

int64_t or_rr_by_definition(const int64_t* rowptr, const int32_t* src, const uint32_t* thr,
                            int64_t n, int64_t m, int model, const or_trig* trig, uint64_t seed, uint64_t sid,
                            int32_t* members, int64_t* width) {
    return or_rr_by_definition_mode(rowptr, src, thr, n, m, model, trig, 0, seed, sid, members,
                                    width);
}

/* One RR set by BFS, exported for single-set checks (per_edge: see skip_list). */
int64_t or_rr_one_mode(const int64_t* rowptr, const int32_t* src, const uint32_t* thr,
                       int64_t n, int64_t m, int model, const or_trig* trig, int per_edge, uint64_t seed,
                       uint64_t sid, int32_t* members, int64_t* width) {
    or_graph g = {n, m, rowptr, src, thr, model, per_edge, trig};
    uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
    if (!mark) return OR_ERR_OOM;
    int64_t r = rr_bfs(&g, seed, sid, members, mark, width);
    free(mark);
    return r;
}

int64_t or_rr_one(const int64_t* rowptr, const int32_t* src, const uint32_t* thr, int64_t n,
                  int64_t m, int model, const or_trig* trig, uint64_t seed, uint64_t sid, int32_t* members,
                  int64_t* width) {
    return or_rr_one_mode(rowptr, src, thr, n, m, model, trig, 0, seed, sid, members, width);
}

/* ---------------------------------------------------------- kappa, Eq. 6 */
/* kappa(R) = 1 - (1 - w/m)^k, evaluated through the geometric series
 *   1 - q^k = (1 - q) * (1 + q + ... + q^(k-1)),  q = 1 - w/m,
 * so that a width far below m does not cancel to nothing in FP64. The series sum
 * S_k and power P_k = q^k are built over the bits of k from the most significant:
 * doubling j -> 2j gives S_2j = S_j * (1 + P_j), P_2j = P_j^2; a set bit j -> j+1
 * gives S_(j+1) = S_j + P_j, P_(j+1) = P_j * q. All terms are non-negative. */
double or_kappa(int64_t w, int64_t m, int k) {
    if (m <= 0 || w <= 0 || k <= 0) return 0.0;
    double x = (double)w / (double)m; /* 1 - q */
    double q = 1.0 - x;
    double S = 0.0, P = 1.0;
    int top = 31;
    while (top > 0 && !(((unsigned)k >> top) & 1u)) top--;
    for (int b = top; b >= 0; b--) {
        S = S * (1.0 + P);
        P = P * P;
        if (((unsigned)k >> b) & 1u) {
            S = S + P;
            P = P * q;
        }
    }
    return x * S;
}

/* kappa in 2^-63 fixed point, truncated (kappa lies in [0, 1]). */
uint64_t or_kappa_fixed(double kappa) { return (uint64_t)ldexp(kappa, 63); }

/* --------------------------------------------------- sampling many RR sets */
typedef struct {
    int64_t n_sets;
    int64_t* len;
    int64_t* width;
    int32_t* mem;
    int64_t used, cap;
    int err;
} chunk_buf;

static void chunk_push(chunk_buf* b, const int32_t* m, int64_t cnt) {
    if (b->err) return;
    if (b->used + cnt > b->cap) {
        int64_t nc = b->cap ? b->cap : 1024;
        while (nc < b->used + cnt) nc *= 2;
        int32_t* nm = (int32_t*)realloc(b->mem, sizeof(int32_t) * (size_t)nc);
        if (!nm) {
            b->err = 1;
            return;
        }
        b->mem = nm;
        b->cap = nc;
    }
    memcpy(b->mem + b->used, m, sizeof(int32_t) * (size_t)cnt);
    b->used += cnt;
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    return nthreads;
#else
    (void)nthreads;
    return 1;
#endif
}

/* Generate RR sets with ids sids(j) = sid0 + j, j in [0, count) (Algorithm 1,
 * its sampling step). Writes a CSR-of-sets (off[count+1], mem) and optional widths.
 * Returns the total member count; if it exceeds mem_cap nothing is copied into mem
 * and the caller retries with a bigger buffer. Sets are independent, so chunks of
 * set ids may run on several host threads; the result does not depend on it. */
int64_t or_sample_mode(const int64_t* rowptr, const int32_t* src, const uint32_t* thr,
                       int64_t n, int64_t m, int model, const or_trig* trig, int per_edge, uint64_t seed,
                       uint64_t sid0, int64_t count, int64_t* off, int32_t* mem,
                       int64_t mem_cap, int64_t* widths, int nthreads) {
    or_graph g = {n, m, rowptr, src, thr, model, per_edge, trig};
    if (count < 0) return OR_ERR_ARG;
    off[0] = 0;
    if (count == 0) return 0;
    nthreads = set_threads(nthreads);
    const int64_t CH = 4096;
    int64_t nch = (count + CH - 1) / CH;
    chunk_buf* bufs = (chunk_buf*)calloc((size_t)nch, sizeof(chunk_buf));
    if (!bufs) return OR_ERR_OOM;
    int fail = 0;
#pragma omp parallel num_threads(nthreads)
    {
        uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!mark || !tmp) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < nch; c++) {
            if (!mark || !tmp) continue;
            chunk_buf* b = &bufs[c];
            int64_t lo = c * CH, hi = lo + CH < count ? lo + CH : count;
            b->n_sets = hi - lo;
            b->len = (int64_t*)malloc(sizeof(int64_t) * (size_t)b->n_sets);
            b->width = (int64_t*)malloc(sizeof(int64_t) * (size_t)b->n_sets);
            if (!b->len || !b->width) {
                b->err = 1;
                continue;
            }
            for (int64_t j = lo; j < hi; j++) {
                int64_t w;
                int64_t cnt = rr_bfs(&g, seed, sid0 + (uint64_t)j, tmp, mark, &w);
                b->len[j - lo] = cnt;
                b->width[j - lo] = w;
                chunk_push(b, tmp, cnt);
            }
        }
        free(mark);
        free(tmp);
    }
    int64_t total = 0;
    for (int64_t c = 0; c < nch; c++)
        if (bufs[c].err) fail = 1;
    if (!fail) {
        int64_t j = 0;
        for (int64_t c = 0; c < nch; c++)
            for (int64_t t = 0; t < bufs[c].n_sets; t++, j++) {
                total += bufs[c].len[t];
                off[j + 1] = total;
                if (widths) widths[j] = bufs[c].width[t];
            }
        if (total <= mem_cap) {
            int64_t pos = 0;
            for (int64_t c = 0; c < nch; c++) {
                memcpy(mem + pos, bufs[c].mem, sizeof(int32_t) * (size_t)bufs[c].used);
                pos += bufs[c].used;
            }
        }
    }
    for (int64_t c = 0; c < nch; c++) {
        free(bufs[c].len);
        free(bufs[c].width);
        free(bufs[c].mem);
    }
    free(bufs);
    return fail ? OR_ERR_OOM : total;
}

int64_t or_sample(const int64_t* rowptr, const int32_t* src, const uint32_t* thr, int64_t n,
                  int64_t m, int model, const or_trig* trig, uint64_t seed, uint64_t sid0, int64_t count,
                  int64_t* off, int32_t* mem, int64_t mem_cap, int64_t* widths, int nthreads) {
    return or_sample_mode(rowptr, src, thr, n, m, model, trig, 0, seed, sid0, count, off, mem,
                          mem_cap, widths, nthreads);
}

/* Sum of kappa over RR sets sid0 .. sid0+count-1 in 2^-63 fixed point, as a
 * 128-bit integer split into (hi, lo). Optionally returns sum of widths. */
int or_kappa_sum(const int64_t* rowptr, const int32_t* src, const uint32_t* thr, int64_t n,
                 int64_t m, int model, const or_trig* trig, int k, uint64_t seed, uint64_t sid0, int64_t count,
                 uint64_t* sum_hi, uint64_t* sum_lo, int64_t* width_sum, int nthreads) {
    or_graph g = {n, m, rowptr, src, thr, model, 0, trig};
    nthreads = set_threads(nthreads);
    u128 total = 0;
    int64_t wtot = 0;
    int fail = 0;
#pragma omp parallel num_threads(nthreads)
    {
        uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        u128 part = 0;
        int64_t wpart = 0;
        if (!mark || !tmp) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 256)
        for (int64_t j = 0; j < count; j++) {
            if (!mark || !tmp) continue;
            int64_t w;
            rr_bfs(&g, seed, sid0 + (uint64_t)j, tmp, mark, &w);
            part += (u128)or_kappa_fixed(or_kappa(w, m, k));
            wpart += w;
        }
#pragma omp critical
        {
            total += part;
            wtot += wpart;
        }
        free(mark);
        free(tmp);
    }
    *sum_hi = (uint64_t)(total >> 64);
    *sum_lo = (uint64_t)total;
    if (width_sum) *width_sum = wtot;
    return fail ? OR_ERR_OOM : OR_OK;
}

/* --------------------------------------------------------- scalar formulas */
/* ln C(n, k) as a sum of k logarithms. */
double or_log_binom(int64_t n, int64_t k) {
    double s = 0.0;
    for (int64_t i = 0; i < k; i++) s += log((double)(n - i) / (double)(k - i));
    return s;
}

/* Eq. 4. */
double or_lambda(int64_t n, int k, double eps, double ell) {
    double ln_n = log((double)n);
    return (8.0 + 2.0 * eps) * (double)n * (ell * ln_n + or_log_binom(n, k) + log(2.0)) /
           (eps * eps);
}

/* eps' of TIM+ (Section 4.1). */
double or_eps_prime(double eps, int k, double ell) {
    return 5.0 * cbrt(ell * eps * eps / ((double)k + ell));
}

/* lambda' of Algorithm 3. */
double or_lambda_prime(int64_t n, double eps_p, double ell) {
    return (2.0 + eps_p) * ell * (double)n * log((double)n) / (eps_p * eps_p);
}

/* c_i of Eq. 7, rounded up. */
int64_t or_c_i(int64_t n, double ell, int i) {
    double ln_n = log((double)n);
    double c = (6.0 * ell * ln_n + 6.0 * log(log2((double)n))) * ldexp(1.0, i);
    return (int64_t)ceil(c);
}

/* Number of rounds of Algorithm 2: floor(log2 n) - 1 (0 when n < 4). */
int or_kpt_rounds(int64_t n) {
    int fl = 0;
    while (((int64_t)1 << (fl + 1)) <= n) fl++;
    return fl - 1 > 0 ? fl - 1 : 0;
}

/* ----------------------------------------------------------- Algorithm 2 */
/* KptEstimation. Returns the round i that stopped (0 if none did: KPT* = 1) and
 * KPT*. Also returns the last executed round (the R' of Algorithm 3) and that
 * round's exact fixed-point kappa sum and set count. */
int or_kpt_estimate(const int64_t* rowptr, const int32_t* src, const uint32_t* thr, int64_t n,
                    int64_t m, int model, const or_trig* trig, int k, double ell, uint64_t seed, uint64_t tag,
                    int nthreads,
                    double* kpt_star, int* stop_round, int* last_round, int64_t* last_c,
                    uint64_t* last_sum_hi, uint64_t* last_sum_lo) {
    int rounds = or_kpt_rounds(n);
    *kpt_star = 1.0;
    *stop_round = 0;
    *last_round = 0;
    *last_c = 0;
    *last_sum_hi = *last_sum_lo = 0;
    for (int i = 1; i <= rounds; i++) {
        int64_t c = or_c_i(n, ell, i);
        uint64_t hi, lo;
        int rc = or_kappa_sum(rowptr, src, thr, n, m, model, trig, k, seed,
                              or_make_sid(PHASE_KPT, i, tag << 32), c, &hi, &lo, NULL, nthreads);
        if (rc) return rc;
        *last_round = i;
        *last_c = c;
        *last_sum_hi = hi;
        *last_sum_lo = lo;
        u128 s = ((u128)hi << 64) | lo;
        /* sum / c_i > 2^-i  <=>  S * 2^-63 > c_i * 2^-i  <=>  S > c_i * 2^(63 - i) */
        u128 bound = (u128)(uint64_t)c << (63 - i);
        if (s > bound) {
            double sum = ldexp((double)s, -63);
            *kpt_star = (double)n * sum / (2.0 * (double)c);
            *stop_round = i;
            return OR_OK;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------ greedy maximum coverage */
/* The greedy of Algorithm 1 over a CSR-of-sets, written naively: every
 * round recounts, for every node, the sets not yet covered that contain it, picks
 * the node with the largest count (ties: smallest id; chosen nodes excluded) and
 * marks the sets it covers. Returns the number of covered sets. */
int64_t or_greedy(int64_t n, int64_t n_sets, const int64_t* off, const int32_t* mem, int k,
                  int32_t* seeds, int64_t* counts_first_round) {
    if (k < 0 || k > n) return OR_ERR_ARG;
    uint8_t* covered = (uint8_t*)calloc((size_t)(n_sets > 0 ? n_sets : 1), 1);
    uint8_t* chosen = (uint8_t*)calloc((size_t)n, 1);
    int64_t* count = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!covered || !chosen || !count) {
        free(covered);
        free(chosen);
        free(count);
        return OR_ERR_OOM;
    }
    for (int r = 0; r < k; r++) {
        memset(count, 0, sizeof(int64_t) * (size_t)n);
        for (int64_t s = 0; s < n_sets; s++)
            if (!covered[s])
                for (int64_t t = off[s]; t < off[s + 1]; t++) count[mem[t]]++;
        if (r == 0 && counts_first_round) memcpy(counts_first_round, count, sizeof(int64_t) * (size_t)n);
        int64_t best = -1;
        for (int64_t v = 0; v < n; v++)
            if (!chosen[v] && (best < 0 || count[v] > count[best])) best = v;
        chosen[best] = 1;
        seeds[r] = (int32_t)best;
        for (int64_t s = 0; s < n_sets; s++)
            if (!covered[s])
                for (int64_t t = off[s]; t < off[s + 1]; t++)
                    if (mem[t] == best) {
                        covered[s] = 1;
                        break;
                    }
    }
    int64_t cov = 0;
    for (int64_t s = 0; s < n_sets; s++) cov += covered[s];
    free(covered);
    free(chosen);
    free(count);
    return cov;
}

/* Number of RR sets sid0 .. sid0+count-1 that intersect the node set `in_s`
 * (n bytes, 1 = member): the covered count of Algorithm 3. */
int64_t or_covered_count(const int64_t* rowptr, const int32_t* src, const uint32_t* thr,
                         int64_t n, int64_t m, int model, const or_trig* trig, uint64_t seed, uint64_t sid0,
                         int64_t count, const uint8_t* in_s, int nthreads) {
    or_graph g = {n, m, rowptr, src, thr, model, 0, trig};
    nthreads = set_threads(nthreads);
    int64_t cov = 0;
    int fail = 0;
#pragma omp parallel num_threads(nthreads) reduction(+ : cov)
    {
        uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!mark || !tmp) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 256)
        for (int64_t j = 0; j < count; j++) {
            if (!mark || !tmp) continue;
            int64_t w;
            int64_t len = rr_bfs(&g, seed, sid0 + (uint64_t)j, tmp, mark, &w);
            for (int64_t t = 0; t < len; t++)
                if (in_s[tmp[t]]) {
                    cov++;
                    break;
                }
        }
        free(mark);
        free(tmp);
    }
    return fail ? OR_ERR_OOM : cov;
}

/* ------------------------------------------------ forward Monte-Carlo spread
 * Section 2.1 (the Monte Carlo estimate of E[I(S)] of Kempe et al.): draw a random
 * graph g -- every edge kept with its propagation probability -- and count the nodes
 * of g reachable from S; the average over independent draws estimates E[I(S)]
 * (Section 7 averages 10^5 of them). Triggering form (Section 4.2): every node keeps
 * the in-edges of its sampled triggering set, and the nodes reachable from S over
 * kept edges are the activated ones.
 *
 * Cascade c draws the world of set id sid = sid0 + c with the keys of the RR sets:
 * the IC in-edge at in-CSR position j is kept iff ic_live(or_ic_word(sid, j), thr_j)
 * -- one coin per in-edge, also in the lists that RR sampling treats by geometric
 * skipping -- and under LT node v keeps the in-edge lt_pick(sid, v). So where no list
 * is skipped, the RR set of sid is exactly the set of nodes that reach its root in
 * the world of the cascade with the same sid.
 *
 * The walk needs G itself: or_out_positions lists, for every node u, the in-CSR
 * positions of its out-edges (ascending), and the destination of every position. */
int or_out_positions(int64_t n, int64_t m, const int64_t* rowptr, const int32_t* src,
                     int64_t* out_rowptr, int64_t* out_pos, int32_t* pos_dst) {
    int64_t* cur = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cur) return OR_ERR_OOM;
    for (int64_t v = 0; v <= n; v++) out_rowptr[v] = 0;
    for (int64_t j = 0; j < m; j++) out_rowptr[src[j] + 1]++;
    for (int64_t v = 0; v < n; v++) out_rowptr[v + 1] += out_rowptr[v];
    for (int64_t v = 0; v < n; v++)
        for (int64_t j = rowptr[v]; j < rowptr[v + 1]; j++) {
            pos_dst[j] = (int32_t)v;
            int64_t u = src[j];
            out_pos[out_rowptr[u] + cur[u]++] = j;
        }
    free(cur);
    return OR_OK;
}

/* One cascade: the nodes reachable from the distinct seeds in the world of sid, in
 * queue[] (BFS order); mark[] is all-zero on entry and on exit. Returns their count. */
static int64_t cascade(const or_graph* g, const int64_t* out_rowptr, const int64_t* out_pos,
                       const int32_t* pos_dst, uint64_t seed, uint64_t sid, const int32_t* seeds,
                       int k, int32_t* queue, uint8_t* mark) {
    int64_t tail = 0;
    for (int i = 0; i < k; i++)
        if (!mark[seeds[i]]) {
            mark[seeds[i]] = 1;
            queue[tail++] = seeds[i];
        }
    for (int64_t head = 0; head < tail; head++) {
        int64_t u = queue[head];
        for (int64_t e = out_rowptr[u]; e < out_rowptr[u + 1]; e++) {
            int64_t j = out_pos[e];
            int32_t v = pos_dst[j];
            if (mark[v]) continue;
            int kept;
            if (g->model == MODEL_IC) {
                kept = ic_live(or_ic_word(seed, sid, j), g->thr[j]);
            } else if (g->model == MODEL_TRIG) {
                int64_t o = trig_pick(g, seed, sid, v);
                kept = 0;
                if (o >= 0)
                    for (int64_t e = g->trig->opt_off[o]; e < g->trig->opt_off[o + 1]; e++)
                        if (g->trig->opt_pos[e] == j) kept = 1;
            } else {
                kept = lt_pick(g, seed, sid, v) == j;
            }
            if (kept) {
                mark[v] = 1;
                queue[tail++] = v;
            }
        }
    }
    for (int64_t i = 0; i < tail; i++) mark[queue[i]] = 0;
    return tail;
}

/* The activated nodes of one cascade (sid) into members[] (capacity n); returns their
 * count. */
int64_t or_cascade_one(const int64_t* rowptr, const int32_t* src, const uint32_t* thr, int64_t n,
                       int64_t m, int model, const or_trig* trig, const int64_t* out_rowptr, const int64_t* out_pos,
                       const int32_t* pos_dst, uint64_t seed, uint64_t sid, const int32_t* seeds,
                       int k, int32_t* members) {
    or_graph g = {n, m, rowptr, src, thr, model, 0, trig};
    for (int i = 0; i < k; i++)
        if (seeds[i] < 0 || seeds[i] >= n) return OR_ERR_ARG;
    uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
    if (!mark) return OR_ERR_OOM;
    int64_t cnt = cascade(&g, out_rowptr, out_pos, pos_dst, seed, sid, seeds, k, members, mark);
    free(mark);
    return cnt;
}

/* Cascades sid0 .. sid0+count-1: counts[c] = activated nodes of cascade c. Returns
 * the total over all cascades (an exact integer; the estimate of E[I(S)] is
 * total / count) or an error code. */
int64_t or_spread_mc(const int64_t* rowptr, const int32_t* src, const uint32_t* thr, int64_t n,
                     int64_t m, int model, const or_trig* trig, const int64_t* out_rowptr, const int64_t* out_pos,
                     const int32_t* pos_dst, uint64_t seed, uint64_t sid0, int64_t count,
                     const int32_t* seeds, int k, int64_t* counts, int nthreads) {
    or_graph g = {n, m, rowptr, src, thr, model, 0, trig};
    for (int i = 0; i < k; i++)
        if (seeds[i] < 0 || seeds[i] >= n) return OR_ERR_ARG;
    nthreads = set_threads(nthreads);
    int64_t total = 0;
    int fail = 0;
#pragma omp parallel num_threads(nthreads) reduction(+ : total)
    {
        uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
        int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
        if (!mark || !queue) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t c = 0; c < count; c++) {
            if (!mark || !queue) continue;
            int64_t a = cascade(&g, out_rowptr, out_pos, pos_dst, seed, sid0 + (uint64_t)c, seeds,
                                k, queue, mark);
            counts[c] = a;
            total += a;
        }
        free(mark);
        free(queue);
    }
    return fail ? OR_ERR_OOM : total;
}
