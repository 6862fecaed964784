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
#include <algorithm>

#include "common.cuh"

namespace {

struct BulkScalars {
    unsigned long long f_count;  // frontier items appended (all levels)
    unsigned long long m_count;  // members appended
    unsigned long long live;     // live in-edges followed
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
    uint32_t* bitmap;
    uint64_t words;
    unsigned long long* slot_width;
    uint32_t* slot_cnt;
    uint32_t* slot_flag;
    unsigned long long* slot_start;
    uint32_t* slot_cursor;
    uint2* F;
    uint64_t fcap;
    uint2* M;
    uint64_t mcap;
    BulkScalars* bs;
    uint64_t lvl_lo, lvl_n;  // current level: F[lvl_lo .. lvl_lo + lvl_n)
    const uint32_t* ng;
    const uint64_t* gp;  // exclusive group prefix of the level, gp[lvl_n] = total
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

__device__ __forceinline__ uint32_t pick4(uint4 v, int c) {
    return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}

__global__ void bulk_init_kernel(BulkArgs a) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < a.S; s += gridDim.x * blockDim.x) {
        const uint32_t j = a.list[a.base + s];
        const uint64_t sid = a.sid0 + j;
        const uint32_t root = rr_root(sid, a.n, a.K);
        atomicOr(&a.bitmap[(uint64_t)s * a.words + (root >> 5)], 1u << (root & 31));
        const uint64_t beg = a.rowptr[root], end = a.rowptr[root + 1];
        a.slot_width[s] = end - beg;
        a.slot_cnt[s] = 1;
        a.slot_cursor[s] = 0;
        const bool cov = (a.flags & SAMPLE_COVER) && marked(a.seed_mark, root);
        a.slot_flag[s] = cov ? 1u : 0u;
        unsigned long long pm = atomicAdd(&a.bs->m_count, 1ull);
        if (pm < a.mcap)
            a.M[pm] = make_uint2(s, root);
        else
            atomicOr(&a.bs->err, 2);
        if (end > beg && !cov) {
            unsigned long long pf = atomicAdd(&a.bs->f_count, 1ull);
            if (pf < a.fcap)
                a.F[pf] = make_uint2(s, root);
            else
                atomicOr(&a.bs->err, 1);
        }
    }
}

// Does in-list [beg, end) with per-node threshold word nt take the skip rule?
__device__ __forceinline__ bool skip_rule(unsigned long long nt, uint64_t beg, uint64_t end) {
    return tim_skip_rule(nt, end - beg);
}

__global__ void bulk_ng_kernel(BulkArgs a, uint32_t* ng) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.lvl_n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = a.F[a.lvl_lo + i].y;
        const uint64_t beg = a.rowptr[v], end = a.rowptr[v + 1];
        ng[i] = skip_rule(a.node_thr[v], beg, end)
                    ? 1u  // placeholder, ignored by bulk_expand_kernel
                    : (uint32_t)(((end - 1) >> 2) - (beg >> 2) + 1);  // end > beg here
    }
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

// Appends of one block staged in shared memory: a warp reserves buffer space with a
// shared atomic, and the block reserves the global range once, at its end (a list's
// global counter is one address for the whole GPU: one atomic per warp and step there
// serialises). Appends that do not fit go to the global list directly.
constexpr unsigned STAGE = 1024;
struct Stage {
    uint2 f[STAGE];
    uint2 m[STAGE];
    unsigned nf, nm;
    unsigned long long gf, gm;
};

__device__ __forceinline__ void staged_append(bool pred, uint32_t s, uint32_t u, uint2* buf,
                                              unsigned* used, unsigned long long* counter,
                                              uint2* list, uint64_t cap, int* err, int errbit,
                                              int lane) {
    const uint32_t bal = __ballot_sync(0xffffffffu, pred);
    if (!bal) return;
    const int leader = __ffs(bal) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(used, (unsigned)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, leader);
    const unsigned r = __popc(bal & ((1u << lane) - 1u));
    const bool staged = pred && base + r < STAGE;
    if (staged) buf[base + r] = make_uint2(s, u);
    warp_append(pred && !staged, s, u, counter, list, cap, err, errbit, lane);
}

// Copy a block's staged appends to one reserved range of each global list.
__device__ __forceinline__ void stage_flush(Stage& st, const BulkArgs& a) {
    __syncthreads();
    const unsigned nf = min(st.nf, STAGE), nm = min(st.nm, STAGE);
    if (threadIdx.x == 0) {
        st.gf = nf ? atomicAdd(&a.bs->f_count, (unsigned long long)nf) : 0ull;
        st.gm = nm ? atomicAdd(&a.bs->m_count, (unsigned long long)nm) : 0ull;
    }
    __syncthreads();
    for (unsigned i = threadIdx.x; i < nf; i += blockDim.x) {
        if (st.gf + i < a.fcap)
            a.F[st.gf + i] = st.f[i];
        else
            atomicOr(&a.bs->err, 1);
    }
    for (unsigned i = threadIdx.x; i < nm; i += blockDim.x) {
        if (st.gm + i < a.mcap)
            a.M[st.gm + i] = st.m[i];
        else
            atomicOr(&a.bs->err, 2);
    }
}

// Add a fresh member's in-degree and count to its set, one atomic per set and warp.
__device__ __forceinline__ void slot_add(bool fresh, uint32_t s, uint64_t deg, const BulkArgs& a,
                                         int lane) {
    const uint32_t fm = __ballot_sync(0xffffffffu, fresh);
    if (!fresh) return;
    const uint32_t grp = __match_any_sync(fm, s);
    // the group's members are distinct nodes of one set: their in-degrees sum below m
    const unsigned dsum = __reduce_add_sync(grp, (unsigned)deg);
    if (lane == __ffs(grp) - 1) {
        atomicAdd(&a.slot_width[s], (unsigned long long)dsum);
        atomicAdd(&a.slot_cnt[s], (unsigned)__popc(grp));
    }
}

__global__ void __launch_bounds__(256) bulk_expand_kernel(BulkArgs a) {
    __shared__ Stage st;
    if (threadIdx.x == 0) st.nf = st.nm = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t G = a.gp[a.lvl_n];
    const uint64_t nchunks = (G + 31) >> 5;
    const uint64_t wid = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t per = (nchunks + nw - 1) / nw;
    const uint64_t c0 = min(wid * per, nchunks);
    const uint64_t c1 = min(c0 + per, nchunks);
    const bool cover = a.flags & SAMPLE_COVER;
    // item holding group 32 * c0: the last i with gp[i] <= 32 * c0
    uint64_t i0 = 0;
    if (c0 < c1) {
        uint64_t lo = 0, hi = a.lvl_n;  // gp[lo] <= x < gp[hi]
        const uint64_t x = c0 << 5;
        while (hi - lo > 1) {
            uint64_t mid = (lo + hi) >> 1;
            if (a.gp[mid] <= x)
                lo = mid;
            else
                hi = mid;
        }
        i0 = lo;
    }
    uint32_t live_acc = 0;
    for (uint64_t c = c0; c < c1; c++) {
        const uint64_t base = c << 5;
        for (int guard = 0; guard < 64 && i0 + 1 < a.lvl_n && a.gp[i0 + 1] <= base; guard++) i0++;
        // boundaries of the next 32 items relative to this chunk
        const uint64_t bi = i0 + 1 + lane;
        const uint64_t bj = bi <= a.lvl_n ? a.gp[bi] : ~0ull;
        const uint32_t bit = (bj > base && bj < base + 32) ? (1u << (uint32_t)(bj - base)) : 0u;
        const uint32_t mask = __reduce_or_sync(0xffffffffu, bit);
        const int q = __popc(mask & ((2u << lane) - 1u));
        const uint64_t gstart_q = __shfl_sync(0xffffffffu, bj, max(q - 1, 0));
        const uint64_t i = i0 + q;
        const uint64_t t = base + lane;
        const bool active = t < G;
        uint32_t s = 0, v = 0;
        uint64_t beg = 0, end = 0, g = 0;
        bool work = false;
        if (active) {
            const uint64_t gstart = q ? gstart_q : a.gp[i0];
            const uint2 it = a.F[a.lvl_lo + i];
            s = it.x;
            v = it.y;
            work = !(cover && *(volatile uint32_t*)&a.slot_flag[s]);
            if (work) {
                beg = __ldg(a.rowptr + v);
                end = __ldg(a.rowptr + v + 1);
                g = (beg >> 2) + (t - gstart);
                work = !skip_rule(__ldg(a.node_thr + v), beg, end);
            }
        }
        uint4 x = make_uint4(0, 0, 0, 0), tv = make_uint4(0, 0, 0, 0);
        uint32_t nlive = 0;
        uint32_t j = 0;
        if (work) {
            j = __ldg(a.list + a.base + s);
            const uint64_t sid = a.sid0 + j;
            x = philox4x32_10((uint32_t)sid, (uint32_t)(sid >> 32), (uint32_t)g, TIM_TAG_IC, a.K);
            tv = __ldg(reinterpret_cast<const uint4*>(a.thr) + g);
        }
#pragma unroll
        for (int cc = 0; cc < 4; cc++) {
            const uint64_t p = (g << 2) + cc;
            bool fresh = false;
            uint32_t u = 0;
            uint64_t ub = 0, ue = 0;
            if (work && p >= beg && p < end) {
                const uint32_t th = pick4(tv, cc);
                if (th == 0xFFFFFFFFu || pick4(x, cc) < th) {
                    nlive++;
                    u = __ldg(a.src + p);
                    const uint32_t b = 1u << (u & 31);
                    const uint32_t old = atomicOr(&a.bitmap[(uint64_t)s * a.words + (u >> 5)], b);
                    fresh = !(old & b);
                    if (fresh) {
                        ub = __ldg(a.rowptr + u);
                        ue = __ldg(a.rowptr + u + 1);
                        if (cover && marked(a.seed_mark, u)) a.slot_flag[s] = 1u;
                    }
                }
            }
            slot_add(fresh, s, ue - ub, a, lane);
            staged_append(fresh, s, u, st.m, &st.nm, &a.bs->m_count, a.M, a.mcap, &a.bs->err, 2,
                          lane);
            const bool push = fresh && ue > ub && !(cover && a.slot_flag[s]);
            staged_append(push, s, u, st.f, &st.nf, &a.bs->f_count, a.F, a.fcap, &a.bs->err, 1,
                          lane);
        }
        i0 = __shfl_sync(0xffffffffu, i, 31);
        live_acc += nlive;
    }
    live_acc = __reduce_add_sync(0xffffffffu, live_acc);
    if (lane == 0 && live_acc) atomicAdd(&a.bs->live, (unsigned long long)live_acc);
    stage_flush(st, a);
}

// The level's items under the skip rule: one warp per item draws the live in-edges
// by geometric skipping and handles each like bulk_expand_kernel does.
__global__ void __launch_bounds__(256) bulk_skip_kernel(BulkArgs a) {
    const int lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const bool cover = a.flags & SAMPLE_COVER;
    uint32_t live_acc = 0;
    for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; i < a.lvl_n;
         i += nw) {
        const uint2 it = a.F[a.lvl_lo + i];
        const uint32_t s = it.x, v = it.y;
        const uint64_t beg = __ldg(a.rowptr + v), end = __ldg(a.rowptr + v + 1);
        const unsigned long long nt = __ldg(a.node_thr + v);
        if (!skip_rule(nt, beg, end)) continue;
        if (cover && *(volatile uint32_t*)&a.slot_flag[s]) continue;
        const uint64_t sid = a.sid0 + __ldg(a.list + a.base + s);
        skip_live_warp((uint32_t)sid, (uint32_t)(sid >> 32), a.K, (uint32_t)beg,
                       (uint32_t)(end - beg), skip_table(a.qtab, nt), lane, [&](uint32_t p) {
                           bool fresh = false;
                           uint32_t u = 0;
                           uint64_t ub = 0, ue = 0;
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
                                   atomicAdd(&a.slot_width[s], ue - ub);
                                   atomicAdd(&a.slot_cnt[s], 1u);
                                   if (cover && marked(a.seed_mark, u)) a.slot_flag[s] = 1u;
                               }
                           }
                           warp_append(fresh, s, u, &a.bs->m_count, a.M, a.mcap, &a.bs->err, 2,
                                       lane);
                           const bool push = fresh && ue > ub && !(cover && a.slot_flag[s]);
                           warp_append(push, s, u, &a.bs->f_count, a.F, a.fcap, &a.bs->err, 1,
                                       lane);
                           return false;
                       });
    }
    live_acc = __reduce_add_sync(0xffffffffu, live_acc);
    if (lane == 0 && live_acc) atomicAdd(&a.bs->live, (unsigned long long)live_acc);
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
                uint64_t* live_out) {
    if (count == 0) return TIM_OK;
    const uint64_t n = (uint64_t)ctx->n;
    const uint64_t words = (n + 31) / 32 + 1;
    // slots: visited bitmaps of at most ~2 GiB
    uint64_t smax = std::max<uint64_t>(32, (2ull << 30) / (words * 4));
    smax = std::min<uint64_t>(smax, 65536);
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
    TIM_TRY(tim_ensure(ctx, ctx->bulk_F, ctx->bulk_fcap * sizeof(uint2)));
    TIM_TRY(tim_ensure(ctx, ctx->bulk_M, ctx->bulk_mcap * sizeof(uint2)));
    TIM_TRY(tim_ensure(ctx, ctx->bulk_ng, ctx->bulk_fcap * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->bulk_gp, (ctx->bulk_fcap + 1) * sizeof(uint64_t)));
    TIM_TRY(tim_ensure(ctx, ctx->bulk_scal, sizeof(BulkScalars)));

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
    BulkScalars hb;
    const unsigned GX = (unsigned)(ctx->num_sms * 4);
    uint32_t done = 0;
    uint64_t live = 0;
    while (done < count) {
        const uint32_t bs = std::min<uint32_t>(S, count - done);
        a.base = done;
        a.S = bs;
        a.F = (uint2*)ctx->bulk_F.p;
        a.M = (uint2*)ctx->bulk_M.p;
        a.fcap = ctx->bulk_fcap;
        a.mcap = ctx->bulk_mcap;
        CUDA_TRY(ctx, cudaMemsetAsync(a.bs, 0, sizeof(BulkScalars), ctx->stream));
        bulk_init_kernel<<<(bs + 255) / 256, 256, 0, ctx->stream>>>(a);
        LAUNCH_CHECK(ctx, "bulk_init_kernel");
        CUDA_TRY(ctx, cudaMemcpyAsync(&hb, a.bs, sizeof hb, cudaMemcpyDeviceToHost, ctx->stream));
        TIM_TRY(tim_sync(ctx));
        uint64_t lo = 0, hi = hb.f_count;
        bool overflow = hb.err != 0;
        for (int level = 0; !overflow && hi > lo && level < (1 << 26); level++) {
            a.lvl_lo = lo;
            a.lvl_n = hi - lo;
            if (a.lvl_n > ctx->bulk_fcap) {
                overflow = true;
                break;
            }
            a.ng = (const uint32_t*)ctx->bulk_ng.p;
            a.gp = (const uint64_t*)ctx->bulk_gp.p;
            bulk_ng_kernel<<<GX * 2, 256, 0, ctx->stream>>>(a, (uint32_t*)ctx->bulk_ng.p);
            LAUNCH_CHECK(ctx, "bulk_ng_kernel");
            TIM_TRY(tim_scan_u32_to_u64(ctx, (const uint32_t*)ctx->bulk_ng.p,
                                        (uint64_t*)ctx->bulk_gp.p, a.lvl_n));
            bulk_expand_kernel<<<GX * 4, 256, 0, ctx->stream>>>(a);
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
            TIM_TRY(tim_ensure(ctx, ctx->bulk_F, ctx->bulk_fcap * sizeof(uint2)));
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
    }
    if (live_out) *live_out = live;
    return TIM_OK;
}
