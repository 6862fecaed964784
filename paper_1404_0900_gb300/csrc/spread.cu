// spread.cu -- forward Monte-Carlo spread of a seed set (Section 2.1: E[I(S)] estimated
// as the average number of nodes reachable from S in random graphs g, every edge kept
// with its propagation probability; Section 4.2: under a triggering model every node
// keeps the in-edges of its sampled triggering set; Section 7 averages 10^5 cascades).
//
// Cascade c walks the world of set id sid = first_set_id + c with the keys of the RR
// sets: the IC in-edge at in-CSR position j is kept iff word (j & 3) of Philox(seed;
// sid, j >> 2, TAG_IC) is below its threshold (one coin per in-edge, also in lists that
// RR sampling treats by geometric skipping), under LT node v keeps the in-edge that
// word 0 of Philox(seed; sid, v, TAG_LT) picks, and under a general triggering model the
// in-edges of the option that the same word picks. Where no list is skipped, the RR set
// of sid is then exactly the set of nodes that reach its root in this cascade's world.
//
// The walk needs G itself: out-records {in-CSR position, destination} grouped by
// source, built from G^T on first use. One block per cascade: its visited bitmap (n
// bits) and queue (the activated nodes, n slots) live in global memory, one pair per
// resident block; the block expands the queue round by round (warps claim queued nodes
// and stride over their out-records) until a round adds nothing.
#include <algorithm>

#include "common.cuh"

namespace {

constexpr int MC_THREADS = 256;

__global__ void out_count_kernel(const uint32_t* __restrict__ src, uint64_t m,
                                 uint32_t* __restrict__ cnt) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < m;
         j += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[__ldg(src + j)], 1u);
}

// One warp per destination v: each in-edge j = (u -> v) becomes out-record {j, v} of u.
__global__ void out_scatter_kernel(const uint64_t* __restrict__ rowptr,
                                   const uint32_t* __restrict__ src, uint64_t n,
                                   const uint64_t* __restrict__ out_rowptr,
                                   uint32_t* __restrict__ cursor, uint2* __restrict__ out_rec) {
    const int lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        const uint64_t b = rowptr[v], e = rowptr[v + 1];
        for (uint64_t j = b + lane; j < e; j += 32) {
            const uint32_t u = __ldg(src + j);
            const uint32_t slot = atomicAdd(&cursor[u], 1u);
            out_rec[out_rowptr[u] + slot] = make_uint2((uint32_t)j, (uint32_t)v);
        }
    }
}

struct McArgs {
    const uint64_t* rowptr;
    const uint32_t* thr;
    const unsigned long long* node_thr;
    const uint64_t* out_rowptr;
    const uint2* out_rec;
    int model;
    uint64_t n;
    PhiloxKeys K;
    uint64_t sid0, count;
    const int32_t* seeds;
    int k;
    uint32_t* bitmap;  // slots * words
    uint32_t* queue;   // slots * n
    uint64_t words;
    uint32_t* counts;              // per cascade
    unsigned long long* scal;      // [0] next cascade, [1] total activated
    // triggering model: options per node, cumulative thresholds, sorted in-CSR positions
    const uint64_t* node_opt;
    const uint32_t* opt_cum;
    const uint64_t* opt_off;
    const uint32_t* opt_pos;
};

// Does v keep in-edge j in the world of sid (LT)?
__device__ __forceinline__ bool lt_kept(const McArgs& a, uint32_t s0, uint32_t s1, uint32_t v,
                                        uint32_t j) {
    const uint64_t beg = __ldg(a.rowptr + v), end = __ldg(a.rowptr + v + 1);
    const uint32_t x = philox4x32_10(s0, s1, v, TIM_TAG_LT, a.K).x;
    const unsigned long long nt = __ldg(a.node_thr + v);
    const uint64_t p = (nt >> 32) ? lt_uniform_pick(nt, beg, end, x)
                                  : lane_lt_search(a.thr, beg, end, x);
    return p == (uint64_t)j;
}

// Does v keep in-edge j in the world of sid (triggering model)? v picks its option with
// the RR walk's draw; j is kept iff it is among the option's positions (ascending).
__device__ __forceinline__ bool trig_kept(const McArgs& a, uint32_t s0, uint32_t s1, uint32_t v,
                                          uint32_t j) {
    const uint64_t o0 = __ldg(a.node_opt + v), o1 = __ldg(a.node_opt + v + 1);
    if (o1 == o0) return false;
    const uint32_t x = philox4x32_10(s0, s1, v, TIM_TAG_LT, a.K).x;
    const uint64_t o = lane_lt_search(a.opt_cum, o0, o1, x);
    if (o >= o1) return false;
    uint64_t lo = __ldg(a.opt_off + o), hi = __ldg(a.opt_off + o + 1);
    for (int it = 0; it < 40 && lo < hi; it++) {  // first position >= j
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(a.opt_pos + mid) < j)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo < __ldg(a.opt_off + o + 1) && __ldg(a.opt_pos + lo) == j;
}

__global__ void __launch_bounds__(MC_THREADS) mc_cascade_kernel(McArgs a) {
    __shared__ unsigned long long s_c;
    __shared__ uint32_t s_tail, s_next;
    const int lane = threadIdx.x & 31;
    uint32_t* bm = a.bitmap + (uint64_t)blockIdx.x * a.words;
    uint32_t* q = a.queue + (uint64_t)blockIdx.x * a.n;
    for (;;) {
        if (threadIdx.x == 0) {
            s_c = atomicAdd(&a.scal[0], 1ull);
            s_tail = 0;
        }
        __syncthreads();
        const unsigned long long c = s_c;
        if (c >= a.count) break;
        const uint64_t sid = a.sid0 + c;
        const uint32_t s0 = (uint32_t)sid, s1 = (uint32_t)(sid >> 32);
        for (int i = threadIdx.x; i < a.k; i += blockDim.x) {
            const uint32_t v = (uint32_t)a.seeds[i];
            const uint32_t b = 1u << (v & 31);
            if (!(atomicOr(&bm[v >> 5], b) & b)) q[atomicAdd(&s_tail, 1u)] = v;
        }
        __syncthreads();
        uint32_t head = 0;
        // every round either adds a node or ends the cascade: at most n + 1 rounds
        for (uint64_t round = 0; round <= a.n; round++) {
            const uint32_t tail = s_tail;
            if (head >= tail) break;
            if (threadIdx.x == 0) s_next = head;
            __syncthreads();
            for (;;) {
                uint32_t i = 0;
                if (lane == 0) i = atomicAdd(&s_next, 1u);
                i = __shfl_sync(0xffffffffu, i, 0);
                if (i >= tail) break;
                const uint32_t u = __ldcg(q + i);
                const uint64_t e0 = __ldg(a.out_rowptr + u), e1 = __ldg(a.out_rowptr + u + 1);
                for (uint64_t e = e0 + lane; e < e1; e += 32) {
                    const uint2 r = __ldg(a.out_rec + e);
                    const uint32_t j = r.x, v = r.y;
                    const uint32_t b = 1u << (v & 31);
                    // a plain (L2) read first: a stale zero only costs a draw
                    if (__ldcg(bm + (v >> 5)) & b) continue;
                    bool kept;
                    if (a.model == TIM_IC) {
                        const uint4 x = philox4x32_10(s0, s1, j >> 2, TIM_TAG_IC, a.K);
                        const uint32_t w = (j & 3) == 0 ? x.x : (j & 3) == 1 ? x.y
                                         : (j & 3) == 2 ? x.z : x.w;
                        const uint32_t t = __ldg(a.thr + j);
                        kept = t == 0xFFFFFFFFu || w < t;
                    } else if (a.model == TIM_TRIG) {
                        kept = trig_kept(a, s0, s1, v, j);
                    } else {
                        kept = lt_kept(a, s0, s1, v, j);
                    }
                    if (kept && !(atomicOr(&bm[v >> 5], b) & b)) q[atomicAdd(&s_tail, 1u)] = v;
                }
            }
            __syncthreads();
            head = tail;
        }
        const uint32_t act = s_tail;
        if (threadIdx.x == 0) {
            a.counts[c] = act;
            atomicAdd(&a.scal[1], (unsigned long long)act);
        }
        // leave the bitmap all-zero: every set bit belongs to a queued node
        for (uint32_t i = threadIdx.x; i < act; i += blockDim.x) bm[__ldcg(q + i) >> 5] = 0u;
        __syncthreads();
    }
}

int build_out_records(tim_ctx* ctx) {
    if (ctx->have_out) return TIM_OK;
    const uint64_t n = (uint64_t)ctx->n, m = (uint64_t)ctx->m;
    TIM_TRY(tim_ensure(ctx, ctx->out_rowptr, (n + 1) * sizeof(uint64_t)));
    TIM_TRY(tim_ensure(ctx, ctx->out_rec, std::max<uint64_t>(m, 1) * sizeof(uint2)));
    TIM_TRY(tim_ensure(ctx, ctx->scratch_a, (n + 1) * sizeof(uint32_t)));
    auto* cnt = (uint32_t*)ctx->scratch_a.p;
    CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, (n + 1) * sizeof(uint32_t), ctx->stream));
    const unsigned G = (unsigned)(ctx->num_sms * 8);
    if (m) {
        out_count_kernel<<<G, 256, 0, ctx->stream>>>((const uint32_t*)ctx->src.p, m, cnt);
        LAUNCH_CHECK(ctx, "out_count_kernel");
    }
    TIM_TRY(tim_scan_u32_to_u64(ctx, cnt, (uint64_t*)ctx->out_rowptr.p, n));
    CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, (n + 1) * sizeof(uint32_t), ctx->stream));
    if (m) {
        out_scatter_kernel<<<G, 256, 0, ctx->stream>>>(
            (const uint64_t*)ctx->rowptr.p, (const uint32_t*)ctx->src.p, n,
            (const uint64_t*)ctx->out_rowptr.p, cnt, (uint2*)ctx->out_rec.p);
        LAUNCH_CHECK(ctx, "out_scatter_kernel");
    }
    ctx->have_out = true;
    return TIM_OK;
}

}  // namespace

extern "C" int tim_spread_mc(tim_ctx* ctx, const int32_t* seeds, int k, uint64_t count,
                             uint64_t seed, uint64_t first_set_id, uint64_t* total, double* mean,
                             uint32_t* counts_out) {
    if (!ctx) return TIM_ERR_ARG;
    if (!ctx->have_graph) return tim_fail(ctx, TIM_ERR_STATE, "no graph loaded");
    if (k < 0 || (k > 0 && !seeds)) return tim_fail(ctx, TIM_ERR_ARG, "bad seed list");
    const uint64_t n = (uint64_t)ctx->n;
    for (int i = 0; i < k; i++)
        if (seeds[i] < 0 || (uint64_t)seeds[i] >= n)
            return tim_fail(ctx, TIM_ERR_ARG, "seed out of range");
    if (count > 0xFFFFFFFFull) return tim_fail(ctx, TIM_ERR_ARG, "count must be below 2^32");
    DeviceGuard g(ctx->device);
    if (total) *total = 0;
    if (mean) *mean = 0.0;
    if (count == 0) return TIM_OK;
    TIM_TRY(build_out_records(ctx));
    // one bitmap + queue per resident block, within ~4 GiB
    const uint64_t words = n / 32 + 1;
    const uint64_t per_slot = words * 4 + n * 4;
    uint64_t slots = std::max<uint64_t>(1, (4ull << 30) / per_slot);
    slots = std::min<uint64_t>(slots, (uint64_t)ctx->num_sms * 4);
    slots = std::min<uint64_t>(slots, count);
    void* prev = ctx->mc_bitmap.p;
    TIM_TRY(tim_ensure(ctx, ctx->mc_bitmap, slots * words * 4));
    if (ctx->mc_bitmap.p != prev || !ctx->mc_clean) {
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->mc_bitmap.p, 0, ctx->mc_bitmap.bytes, ctx->stream));
        ctx->mc_clean = true;
    }
    TIM_TRY(tim_ensure(ctx, ctx->mc_queue, slots * n * 4));
    TIM_TRY(tim_ensure(ctx, ctx->mc_counts, count * 4));
    TIM_TRY(tim_ensure(ctx, ctx->mc_seeds, std::max(k, 1) * sizeof(int32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->mc_scal, 2 * sizeof(unsigned long long)));
    if (k > 0)
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->mc_seeds.p, seeds, (size_t)k * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->mc_scal.p, 0, 2 * sizeof(unsigned long long), ctx->stream));
    McArgs a;
    a.rowptr = (const uint64_t*)ctx->rowptr.p;
    a.thr = (const uint32_t*)ctx->thr.p;
    a.node_thr = (const unsigned long long*)ctx->node_thr.p;
    a.out_rowptr = (const uint64_t*)ctx->out_rowptr.p;
    a.out_rec = (const uint2*)ctx->out_rec.p;
    a.model = ctx->model;
    a.n = n;
    a.K = tim_philox_keys(seed);
    a.sid0 = first_set_id;
    a.count = count;
    a.seeds = (const int32_t*)ctx->mc_seeds.p;
    a.k = k;
    a.bitmap = (uint32_t*)ctx->mc_bitmap.p;
    a.queue = (uint32_t*)ctx->mc_queue.p;
    a.words = words;
    a.counts = (uint32_t*)ctx->mc_counts.p;
    a.scal = (unsigned long long*)ctx->mc_scal.p;
    a.node_opt = (const uint64_t*)ctx->node_opt.p;
    a.opt_cum = (const uint32_t*)ctx->opt_cum.p;
    a.opt_off = (const uint64_t*)ctx->opt_off.p;
    a.opt_pos = (const uint32_t*)ctx->opt_pos.p;
    ctx->mc_clean = false;
    mc_cascade_kernel<<<(unsigned)slots, MC_THREADS, 0, ctx->stream>>>(a);
    LAUNCH_CHECK(ctx, "mc_cascade_kernel");
    unsigned long long h[2] = {0, 0};
    CUDA_TRY(ctx, cudaMemcpyAsync(h, ctx->mc_scal.p, sizeof h, cudaMemcpyDeviceToHost,
                                  ctx->stream));
    if (counts_out)
        CUDA_TRY(ctx, cudaMemcpyAsync(counts_out, ctx->mc_counts.p, count * 4,
                                      cudaMemcpyDeviceToHost, ctx->stream));
    TIM_TRY(tim_sync(ctx));
    ctx->mc_clean = true;
    if (total) *total = h[1];
    if (mean) *mean = (double)h[1] / (double)count;
    return TIM_OK;
}
