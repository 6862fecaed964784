// select.cu -- greedy maximum coverage over the RR-set store (the selection of
// Algorithm 1; also the greedy on R' of Algorithm 3).
//
// Index: coverage counts (how many stored sets contain each node) by a histogram over
// the store, an exclusive scan into node offsets, and a scatter of set ids into
// per-node lists (node -> sets).
// Greedy round r: an argmax over the counts with a warp-shuffle reduction of the key
// (count << 32 | ~node) so ties go to the smallest id and chosen nodes are skipped
// (counts read four at a time, several loads in flight per thread: the scan runs at
// DRAM speed when the counts outgrow L2); then every not-yet-covered set in the chosen
// node's list is marked covered and each of its members loses one from its count (in
// the cooperative launch, sets of more than COVER_CHUNK members are cut into chunks
// that all warps share). The chosen node is read on the device, so the k rounds run
// without host round trips.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

// Both index kernels take four members per thread and step (16-byte loads of the pool,
// which is 16-byte aligned): four independent atomics per thread are in flight at once.
__global__ void count_members_kernel(const uint32_t* __restrict__ pool, uint64_t members,
                                     uint32_t* __restrict__ cnt) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t quads = members >> 2;
    const uint4* pool4 = reinterpret_cast<const uint4*>(pool);
    for (uint64_t q = tid; q < quads; q += stride) {
        const uint4 u = __ldg(pool4 + q);
        atomicAdd(&cnt[u.x], 1u);
        atomicAdd(&cnt[u.y], 1u);
        atomicAdd(&cnt[u.z], 1u);
        atomicAdd(&cnt[u.w], 1u);
    }
    for (uint64_t p = (quads << 2) + tid; p < members; p += stride) atomicAdd(&cnt[pool[p]], 1u);
}

// Node v's sets: node_sets[start(v) .. start(v + 1)). next[v] holds start(v) on entry
// (next = node_off + 1, the exclusive scan written one place to the right); each member
// takes its position with one atomic on it, so that afterwards next[v] = start(v + 1):
// node_off[0 .. n] are the node offsets with no cursor array and no offset load.
__global__ void scatter_sets_kernel(const uint32_t* __restrict__ pool,
                                    const uint32_t* __restrict__ pool_sid, uint64_t members,
                                    unsigned long long* __restrict__ next,
                                    uint32_t* __restrict__ node_sets) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t quads = members >> 2;
    const uint4* pool4 = reinterpret_cast<const uint4*>(pool);
    const uint4* sid4 = reinterpret_cast<const uint4*>(pool_sid);
    for (uint64_t q = tid; q < quads; q += stride) {
        const uint4 u = __ldg(pool4 + q);
        const uint4 j = __ldg(sid4 + q);
        const unsigned long long p0 = atomicAdd(&next[u.x], 1ull), p1 = atomicAdd(&next[u.y], 1ull);
        const unsigned long long p2 = atomicAdd(&next[u.z], 1ull), p3 = atomicAdd(&next[u.w], 1ull);
        node_sets[p0] = j.x;
        node_sets[p1] = j.y;
        node_sets[p2] = j.z;
        node_sets[p3] = j.w;
    }
    for (uint64_t p = (quads << 2) + tid; p < members; p += stride)
        node_sets[atomicAdd(&next[pool[p]], 1ull)] = pool_sid[p];
}

__device__ __forceinline__ unsigned long long greedy_key(int cnt, uint32_t v) {
    return ((unsigned long long)(uint32_t)max(cnt, 0) << 32) | (unsigned long long)(~v);
}

// Best key of nodes 4q .. 4q+3 (0 for chosen nodes): counts as one 16-byte load, the
// chosen flags as one 32-bit word.
__device__ __forceinline__ unsigned long long quad_key(int4 c, uint32_t ch, uint64_t q) {
    const uint32_t v = (uint32_t)(q << 2);
    unsigned long long b = (ch & 0xFFu) ? 0ull : greedy_key(c.x, v);
    b = max(b, (ch & 0xFF00u) ? 0ull : greedy_key(c.y, v + 1));
    b = max(b, (ch & 0xFF0000u) ? 0ull : greedy_key(c.z, v + 2));
    b = max(b, (ch & 0xFF000000u) ? 0ull : greedy_key(c.w, v + 3));
    return b;
}

// Best key over the thread's share of the nodes (thread t of `stride` takes quads t,
// t + stride, ...; four quads in flight; the last n mod 4 nodes one by one). Counts
// and flags are read from L2 (__ldcg): other blocks change them between rounds. Both
// arrays start 16-byte aligned (cudaMalloc).
__device__ __forceinline__ unsigned long long slice_argmax(const int* counts,
                                                           const uint8_t* chosen, uint64_t n,
                                                           uint64_t t, uint64_t stride) {
    const int4* c4 = reinterpret_cast<const int4*>(counts);
    const uint32_t* h4 = reinterpret_cast<const uint32_t*>(chosen);
    const uint64_t nq = n >> 2;
    unsigned long long b = 0;
    uint64_t q = t;
    for (; q + 3 * stride < nq; q += 4 * stride) {
        int4 c[4];
        uint32_t h[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            c[i] = __ldcg(c4 + q + i * stride);
            h[i] = __ldcg(h4 + q + i * stride);
        }
#pragma unroll
        for (int i = 0; i < 4; i++) b = max(b, quad_key(c[i], h[i], q + i * stride));
    }
    for (; q < nq; q += stride) b = max(b, quad_key(__ldcg(c4 + q), __ldcg(h4 + q), q));
    for (uint64_t v = (nq << 2) + t; v < n; v += stride)
        if (!__ldcg(chosen + v)) b = max(b, greedy_key(__ldcg(counts + v), (uint32_t)v));
    return b;
}

__global__ void argmax_kernel(const int* __restrict__ counts, const uint8_t* __restrict__ chosen,
                              uint64_t n, unsigned long long* __restrict__ best) {
    unsigned long long b = slice_argmax(counts, chosen, n,
                                        blockIdx.x * (uint64_t)blockDim.x + threadIdx.x,
                                        (uint64_t)gridDim.x * blockDim.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
        b = y > b ? y : b;
    }
    __shared__ unsigned long long wb[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wb[wid] = b;
    __syncthreads();
    if (wid == 0) {
        b = lane < (int)(blockDim.x >> 5) ? wb[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
            b = y > b ? y : b;
        }
        if (lane == 0 && b) atomicMax(best, b);
    }
}

__global__ void set_key_kernel(unsigned long long* key, unsigned long long value) { *key = value; }

__global__ void cover_kernel(const unsigned long long* __restrict__ best,
                             const uint64_t* __restrict__ node_off,
                             const uint32_t* __restrict__ node_sets,
                             const uint64_t* __restrict__ set_start,
                             const uint32_t* __restrict__ set_len,
                             const uint32_t* __restrict__ pool, uint8_t* __restrict__ covered,
                             int* __restrict__ counts, uint8_t* __restrict__ chosen,
                             int32_t* __restrict__ seed_out, unsigned long long* __restrict__ ncov) {
    const unsigned long long key = *best;
    if (key == 0) return;  // no candidate (cannot happen for k <= n)
    const uint32_t v = ~(uint32_t)(key & 0xFFFFFFFFull);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        chosen[v] = 1;
        *seed_out = (int32_t)v;
    }
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t a = node_off[v], b = node_off[v + 1];
    unsigned long long fresh = 0;
    for (uint64_t i = a + warp; i < b; i += nwarps) {
        uint32_t s = node_sets[i];
        if (covered[s]) continue;  // uniform across the warp
        __syncwarp();
        if (lane == 0) {
            covered[s] = 1;
            fresh++;
        }
        const uint64_t st = set_start[s];
        const uint32_t len = set_len[s];
        for (uint32_t t = lane; t < len; t += 32) atomicSub(&counts[pool[st + t]], 1);
    }
    if (lane == 0 && fresh) atomicAdd(ncov, fresh);
}

// Members per chunk of a large set in the cooperative greedy: a newly covered set with
// more members is split into chunks that all warps share after the cover step (one warp
// walking a set of 10^4 - 10^6 members would hold up the round).
constexpr uint32_t COVER_CHUNK = 4096;

// All k greedy rounds in one cooperative launch: per round an argmax over the counts
// (every block reduces a slice, atomicMax into best[r]), a grid barrier, the cover step
// of the chosen node (warps over its set list; a set of more than COVER_CHUNK members is
// only marked, and its member chunks listed), a second barrier, and when chunks were
// listed, the chunks over all warps and a third barrier. chunks holds at most
// chunk_cap entries (set id | chunk << 32); nchunk[r] counts round r's.
__global__ void __launch_bounds__(256)
greedy_rounds_kernel(int* __restrict__ counts, uint8_t* __restrict__ chosen, uint64_t n,
                     const uint64_t* __restrict__ node_off, const uint32_t* __restrict__ node_sets,
                     const uint64_t* __restrict__ set_start, const uint32_t* __restrict__ set_len,
                     const uint32_t* __restrict__ pool, uint8_t* __restrict__ covered, int k,
                     unsigned long long* __restrict__ best, int32_t* __restrict__ seeds,
                     unsigned long long* __restrict__ ncov, GridBarrier* bar, int* err,
                     unsigned limit, unsigned long long* __restrict__ chunks,
                     unsigned long long* __restrict__ nchunk, unsigned long long chunk_cap) {
    __shared__ unsigned long long wb[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long fresh = 0;
    for (int r = 0; r < k; r++) {
        unsigned long long b = slice_argmax(counts, chosen, n,
                                            blockIdx.x * (uint64_t)blockDim.x + threadIdx.x,
                                            (uint64_t)gridDim.x * blockDim.x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
            b = y > b ? y : b;
        }
        if (lane == 0) wb[wid] = b;
        __syncthreads();
        if (wid == 0) {
            b = lane < (int)(blockDim.x >> 5) ? wb[lane] : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
                b = y > b ? y : b;
            }
            if (lane == 0 && b) atomicMax(best + r, b);
        }
        if (!grid_barrier(bar, err, limit)) return;
        const unsigned long long key = ((volatile unsigned long long*)best)[r];
        if (key != 0) {
            const uint32_t v = ~(uint32_t)(key & 0xFFFFFFFFull);
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                chosen[v] = 1;
                seeds[r] = (int32_t)v;
            }
            const uint64_t a = node_off[v], e = node_off[v + 1];
            for (uint64_t i = a + warp; i < e; i += nwarps) {
                const uint32_t s = node_sets[i];
                if (((volatile uint8_t*)covered)[s]) continue;  // uniform across the warp
                __syncwarp();
                if (lane == 0) {
                    covered[s] = 1;
                    fresh++;
                }
                const uint64_t st = set_start[s];
                const uint32_t len = set_len[s];
                if (len <= COVER_CHUNK) {
                    for (uint32_t t = lane; t < len; t += 32) atomicSub(&counts[pool[st + t]], 1);
                } else {
                    const uint32_t nc = (len + COVER_CHUNK - 1) / COVER_CHUNK;
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(nchunk + r, (unsigned long long)nc);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    for (uint32_t c = lane; c < nc; c += 32) {
                        if (base + c < chunk_cap)
                            chunks[base + c] = (unsigned long long)s | ((unsigned long long)c << 32);
                        else
                            atomicOr(err, TIM_DEV_ERR_BOUNDS);
                    }
                }
            }
        }
        if (!grid_barrier(bar, err, limit)) return;
        // the large sets' member chunks, over all warps, eight loads in flight per lane
        const unsigned long long nc = min(((volatile unsigned long long*)nchunk)[r], chunk_cap);
        if (nc) {
            for (uint64_t w = warp; w < nc; w += nwarps) {
                const unsigned long long e = chunks[w];
                const uint32_t s = (uint32_t)e, c = (uint32_t)(e >> 32);
                const uint64_t st = set_start[s] + (uint64_t)c * COVER_CHUNK;
                const uint32_t len = min(COVER_CHUNK, set_len[s] - c * COVER_CHUNK);
                for (uint32_t t = lane; t < len; t += 256) {
                    uint32_t u[8];
#pragma unroll
                    for (int q = 0; q < 8; q++)
                        u[q] = t + 32u * q < len ? __ldg(pool + st + t + 32u * q) : 0u;
#pragma unroll
                    for (int q = 0; q < 8; q++)
                        if (t + 32u * q < len) atomicSub(&counts[u[q]], 1);
                }
            }
            if (!grid_barrier(bar, err, limit)) return;
        }
    }
    if (lane == 0 && fresh) atomicAdd(ncov, fresh);
}

}  // namespace

int tim_build_index(tim_ctx* ctx) {
    const uint64_t n = (uint64_t)ctx->n, members = ctx->members;
    TIM_TRY(tim_ensure(ctx, ctx->counts, (n + 1) * sizeof(int)));
    TIM_TRY(tim_ensure(ctx, ctx->node_off, (n + 2) * sizeof(uint64_t)));
    TIM_TRY(tim_ensure(ctx, ctx->node_sets, (members + 1) * sizeof(uint32_t)));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->counts.p, 0, (n + 1) * sizeof(int), ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->node_off.p, 0, sizeof(uint64_t), ctx->stream));
    const unsigned G = (unsigned)(ctx->num_sms * 8);
    if (members) {
        count_members_kernel<<<G, 256, 0, ctx->stream>>>((const uint32_t*)ctx->pool.p, members,
                                                         (uint32_t*)ctx->counts.p);
        LAUNCH_CHECK(ctx, "count_members_kernel");
    }
    // node_off[v + 1] = start of node v's sets (node_off[0] = 0); the scatter turns it
    // into start(v + 1)
    TIM_TRY(tim_scan_u32_to_u64(ctx, (const uint32_t*)ctx->counts.p,
                                (uint64_t*)ctx->node_off.p + 1, n));
    if (members) {
        scatter_sets_kernel<<<G, 256, 0, ctx->stream>>>(
            (const uint32_t*)ctx->pool.p, (const uint32_t*)ctx->pool_sid.p, members,
            (unsigned long long*)ctx->node_off.p + 1, (uint32_t*)ctx->node_sets.p);
        LAUNCH_CHECK(ctx, "scatter_sets_kernel");
    }
    return TIM_OK;
}

int tim_greedy(tim_ctx* ctx, int k, int32_t* host_seeds, uint64_t* covered) {
    const uint64_t n = (uint64_t)ctx->n;
    if (k < 1 || (uint64_t)k > n) return tim_fail(ctx, TIM_ERR_ARG, "k must be in [1, n]");
    TIM_TRY(tim_ensure(ctx, ctx->covered, ctx->n_sets + 1));
    TIM_TRY(tim_ensure(ctx, ctx->chosen, n + 1));
    TIM_TRY(tim_ensure(ctx, ctx->best, (size_t)k * sizeof(unsigned long long)));
    TIM_TRY(tim_ensure(ctx, ctx->seeds_dev, (size_t)k * sizeof(int32_t)));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->covered.p, 0, ctx->n_sets + 1, ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->chosen.p, 0, n + 1, ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->best.p, 0, (size_t)k * sizeof(unsigned long long),
                                  ctx->stream));
    TIM_TRY(tim_zero_scalars(ctx));
    DevScalars* ds = tim_dscal(ctx);
    auto* best = (unsigned long long*)ctx->best.p;
    // all rounds in one cooperative launch when the device supports it
    int coop = 0, nb = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (coop &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, greedy_rounds_kernel, 256, 0) ==
            cudaSuccess &&
        nb > 0) {
        TIM_TRY(tim_ensure(ctx, ctx->greedy_bar, sizeof(GridBarrier)));
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->greedy_bar.p, 0, sizeof(GridBarrier), ctx->stream));
        // every covered set is listed at most once, in ceil(len / COVER_CHUNK) chunks
        unsigned long long chunk_cap = ctx->n_sets + ctx->members / COVER_CHUNK + 1;
        TIM_TRY(tim_ensure(ctx, ctx->greedy_chunks, chunk_cap * sizeof(unsigned long long)));
        TIM_TRY(tim_ensure(ctx, ctx->greedy_nchunk, (size_t)k * sizeof(unsigned long long)));
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->greedy_nchunk.p, 0, (size_t)k * sizeof(unsigned long long),
                                      ctx->stream));
        auto* d_chunks = (unsigned long long*)ctx->greedy_chunks.p;
        auto* d_nchunk = (unsigned long long*)ctx->greedy_nchunk.p;
        const unsigned grid = (unsigned)(ctx->num_sms * std::min(nb, 4));
        int* d_counts = (int*)ctx->counts.p;
        uint8_t* d_chosen = (uint8_t*)ctx->chosen.p;
        uint64_t nn = n;
        const uint64_t* d_off = (const uint64_t*)ctx->node_off.p;
        const uint32_t* d_ns = (const uint32_t*)ctx->node_sets.p;
        const uint64_t* d_ss = (const uint64_t*)ctx->set_start.p;
        const uint32_t* d_sl = (const uint32_t*)ctx->set_len.p;
        const uint32_t* d_pool = (const uint32_t*)ctx->pool.p;
        uint8_t* d_cov = (uint8_t*)ctx->covered.p;
        int kk = k;
        int32_t* d_seeds = (int32_t*)ctx->seeds_dev.p;
        unsigned long long* d_ncov = &ds->covered;
        GridBarrier* d_bar = (GridBarrier*)ctx->greedy_bar.p;
        int* d_err = &ds->err;
        unsigned limit = ctx->wait_limit;
        void* args[] = {&d_counts, &d_chosen, &nn, &d_off, &d_ns, &d_ss, &d_sl, &d_pool,
                        &d_cov, &kk, &best, &d_seeds, &d_ncov, &d_bar, &d_err, &limit,
                        &d_chunks, &d_nchunk, &chunk_cap};
        CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)greedy_rounds_kernel, dim3(grid),
                                                  dim3(256), args, 0, ctx->stream));
        LAUNCH_CHECK(ctx, "greedy_rounds_kernel");
        if (host_seeds)
            CUDA_TRY(ctx, cudaMemcpyAsync(host_seeds, ctx->seeds_dev.p, (size_t)k * sizeof(int32_t),
                                          cudaMemcpyDeviceToHost, ctx->stream));
        TIM_TRY(tim_read_scalars(ctx));
        if (ctx->h_scal->err & TIM_DEV_ERR_TIMEOUT)
            return tim_fail(ctx, TIM_ERR_TIMEOUT, "greedy grid barrier timed out");
        if (ctx->h_scal->err)
            return tim_fail(ctx, TIM_ERR_CUDA, "device error flags set by the greedy");
        if (covered) *covered = ctx->h_scal->covered;
        return TIM_OK;
    }
    const unsigned GA = (unsigned)(ctx->num_sms * 4);
    const unsigned GC = (unsigned)(ctx->num_sms * 2);
    for (int r = 0; r < k; r++) {
        argmax_kernel<<<GA, 512, 0, ctx->stream>>>((const int*)ctx->counts.p,
                                                   (const uint8_t*)ctx->chosen.p, n, best + r);
        LAUNCH_CHECK(ctx, "argmax_kernel");
        cover_kernel<<<GC, 256, 0, ctx->stream>>>(
            best + r, (const uint64_t*)ctx->node_off.p, (const uint32_t*)ctx->node_sets.p,
            (const uint64_t*)ctx->set_start.p, (const uint32_t*)ctx->set_len.p,
            (const uint32_t*)ctx->pool.p, (uint8_t*)ctx->covered.p, (int*)ctx->counts.p,
            (uint8_t*)ctx->chosen.p, (int32_t*)ctx->seeds_dev.p + r, &ds->covered);
        LAUNCH_CHECK(ctx, "cover_kernel");
    }
    if (host_seeds)
        CUDA_TRY(ctx, cudaMemcpyAsync(host_seeds, ctx->seeds_dev.p, (size_t)k * sizeof(int32_t),
                                      cudaMemcpyDeviceToHost, ctx->stream));
    TIM_TRY(tim_read_scalars(ctx));
    if (covered) *covered = ctx->h_scal->covered;
    return TIM_OK;
}

// Bitmap of a seed set held in device memory (for Algorithm 3's coverage test).
__global__ void mark_seeds_kernel(const int32_t* __restrict__ seeds, int k,
                                  uint32_t* __restrict__ mark) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        uint32_t u = (uint32_t)seeds[i];
        atomicOr(&mark[u >> 5], 1u << (u & 31));
    }
}

// Stepwise greedy: the caller chooses each node (for example from coverage counts summed
// over several contexts), the context covers that node's sets of its own store.
int tim_greedy_begin(tim_ctx* ctx) {
    TIM_TRY(tim_build_index(ctx));
    TIM_TRY(tim_ensure(ctx, ctx->covered, ctx->n_sets + 1));
    TIM_TRY(tim_ensure(ctx, ctx->chosen, (uint64_t)ctx->n + 1));
    TIM_TRY(tim_ensure(ctx, ctx->best, sizeof(unsigned long long)));
    TIM_TRY(tim_ensure(ctx, ctx->seeds_dev, sizeof(int32_t)));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->covered.p, 0, ctx->n_sets + 1, ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->chosen.p, 0, (uint64_t)ctx->n + 1, ctx->stream));
    return TIM_OK;
}

int tim_greedy_take(tim_ctx* ctx, int32_t v, uint64_t* newly_covered) {
    // the key cover_kernel decodes: any count, node v
    const unsigned long long key = (1ull << 32) | (unsigned long long)(~(uint32_t)v);
    TIM_TRY(tim_zero_scalars(ctx));
    DevScalars* ds = tim_dscal(ctx);
    set_key_kernel<<<1, 1, 0, ctx->stream>>>((unsigned long long*)ctx->best.p, key);
    LAUNCH_CHECK(ctx, "set_key_kernel");
    cover_kernel<<<(unsigned)(ctx->num_sms * 2), 256, 0, ctx->stream>>>(
        (const unsigned long long*)ctx->best.p, (const uint64_t*)ctx->node_off.p,
        (const uint32_t*)ctx->node_sets.p, (const uint64_t*)ctx->set_start.p,
        (const uint32_t*)ctx->set_len.p, (const uint32_t*)ctx->pool.p, (uint8_t*)ctx->covered.p,
        (int*)ctx->counts.p, (uint8_t*)ctx->chosen.p, (int32_t*)ctx->seeds_dev.p, &ds->covered);
    LAUNCH_CHECK(ctx, "cover_kernel");
    TIM_TRY(tim_read_scalars(ctx));
    if (newly_covered) *newly_covered = ctx->h_scal->covered;
    return TIM_OK;
}

int tim_mark_seeds(tim_ctx* ctx, const int32_t* d_seeds, int k) {
    const uint64_t words = (uint64_t)(ctx->n + 31) / 32 + 1;
    TIM_TRY(tim_ensure(ctx, ctx->seed_mark, words * sizeof(uint32_t)));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->seed_mark.p, 0, words * sizeof(uint32_t), ctx->stream));
    if (k > 0) {
        mark_seeds_kernel<<<(k + 255) / 256, 256, 0, ctx->stream>>>(d_seeds, k,
                                                                    (uint32_t*)ctx->seed_mark.p);
        LAUNCH_CHECK(ctx, "mark_seeds_kernel");
    }
    return TIM_OK;
}

// ------------------------------------------------------ several queries at once
//
// The greedy of Algorithm 1 for a batch of queries, each over its own context's
// RR-set store: every kernel covers all queries (each query owns a range of blocks in
// proportion to its work), so one round of the batch is two launches whatever the
// number of queries, and the whole sequence
// (index build and the k rounds) is captured once into a CUDA graph and launched as
// one unit.

namespace {

struct GreedyDesc {
    const uint32_t* pool;
    const uint32_t* pool_sid;
    uint64_t members;
    const uint64_t* set_start;
    const uint32_t* set_len;
    int* counts;
    uint64_t* node_off;
    uint32_t* cursor;
    uint32_t* node_sets;
    uint8_t* covered;
    uint8_t* chosen;
    unsigned long long* best;
    int32_t* seeds;
    unsigned long long* ncov;
    uint64_t n;
    int k;
    int pad;
};

// Blocks are shared out among the queries in proportion to their work; block b belongs
// to the query q with bstart[q] <= b < bstart[q + 1] and is its (b - bstart[q])-th.
__device__ __forceinline__ int block_query(const unsigned* __restrict__ bstart, int nq,
                                           unsigned* local, unsigned* count) {
    int lo = 0, hi = nq;  // bstart[lo] <= b < bstart[hi]
    const unsigned b = blockIdx.x;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bstart[mid] <= b)
            lo = mid;
        else
            hi = mid;
    }
    *local = b - bstart[lo];
    *count = bstart[lo + 1] - bstart[lo];
    return lo;
}

__global__ void mcount_kernel(const GreedyDesc* __restrict__ gd, const unsigned* __restrict__ bstart,
                              int nq) {
    unsigned lb, nb;
    const GreedyDesc& d = gd[block_query(bstart, nq, &lb, &nb)];
    for (uint64_t p = lb * (uint64_t)blockDim.x + threadIdx.x; p < d.members;
         p += (uint64_t)nb * blockDim.x)
        atomicAdd((unsigned*)&d.counts[d.pool[p]], 1u);
}

__global__ void mscatter_kernel(const GreedyDesc* __restrict__ gd,
                                const unsigned* __restrict__ bstart, int nq) {
    unsigned lb, nb;
    const GreedyDesc& d = gd[block_query(bstart, nq, &lb, &nb)];
    for (uint64_t p = lb * (uint64_t)blockDim.x + threadIdx.x; p < d.members;
         p += (uint64_t)nb * blockDim.x) {
        const uint32_t u = d.pool[p];
        const uint32_t slot = atomicAdd(&d.cursor[u], 1u);
        d.node_sets[d.node_off[u] + slot] = d.pool_sid[p];
    }
}

__global__ void margmax_kernel(const GreedyDesc* __restrict__ gd, const unsigned* __restrict__ bstart,
                               int nq, int r) {
    unsigned lb, nb;
    const GreedyDesc& d = gd[block_query(bstart, nq, &lb, &nb)];
    if (r >= d.k) return;
    unsigned long long b = slice_argmax(d.counts, d.chosen, d.n,
                                        lb * (uint64_t)blockDim.x + threadIdx.x,
                                        (uint64_t)nb * blockDim.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
        b = y > b ? y : b;
    }
    if ((threadIdx.x & 31) == 0 && b) atomicMax(&d.best[r], b);
}

__global__ void mcover_kernel(const GreedyDesc* __restrict__ gd, const unsigned* __restrict__ bstart,
                              int nq, int r) {
    unsigned lb, nb;
    const GreedyDesc& d = gd[block_query(bstart, nq, &lb, &nb)];
    if (r >= d.k) return;
    const unsigned long long key = d.best[r];
    if (key == 0) return;
    const uint32_t v = ~(uint32_t)(key & 0xFFFFFFFFull);
    if (lb == 0 && threadIdx.x == 0) {
        d.chosen[v] = 1;
        d.seeds[r] = (int32_t)v;
    }
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (lb * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)nb * blockDim.x) >> 5;
    const uint64_t a = d.node_off[v], b = d.node_off[v + 1];
    unsigned long long fresh = 0;
    for (uint64_t i = a + warp; i < b; i += nwarps) {
        const uint32_t s = d.node_sets[i];
        if (d.covered[s]) continue;
        __syncwarp();
        if (lane == 0) {
            d.covered[s] = 1;
            fresh++;
        }
        const uint64_t st = d.set_start[s];
        const uint32_t len = d.set_len[s];
        for (uint32_t t = lane; t < len; t += 32) atomicSub(&d.counts[d.pool[st + t]], 1);
    }
    if (lane == 0 && fresh) atomicAdd(d.ncov, fresh);
}

}  // namespace

int tim_greedy_batch(tim_ctx* owner, tim_ctx* const* ctxs, const int* ks, int nq,
                     int32_t* const* host_seeds, uint64_t* covered, bool use_graph) {
    if (nq <= 0) return TIM_OK;
    int kmax = 0;
    std::vector<GreedyDesc> gd(nq);
    for (int i = 0; i < nq; i++) {
        tim_ctx* c = ctxs[i];
        const uint64_t n = (uint64_t)c->n;
        const int k = ks[i];
        if (k < 1 || (uint64_t)k > n) return tim_fail(owner, TIM_ERR_ARG, "k must be in [1, n]");
        kmax = std::max(kmax, k);
        TIM_TRY(tim_ensure(c, c->counts, (n + 1) * sizeof(int)));
        TIM_TRY(tim_ensure(c, c->node_off, (n + 1) * sizeof(uint64_t)));
        TIM_TRY(tim_ensure(c, c->cursor, (n + 1) * sizeof(uint32_t)));
        TIM_TRY(tim_ensure(c, c->node_sets, (c->members + 1) * sizeof(uint32_t)));
        TIM_TRY(tim_ensure(c, c->covered, c->n_sets + 1));
        TIM_TRY(tim_ensure(c, c->chosen, n + 1));
        TIM_TRY(tim_ensure(c, c->best, (size_t)k * sizeof(unsigned long long) + 8));
        TIM_TRY(tim_ensure(c, c->seeds_dev, (size_t)k * sizeof(int32_t)));
        // the scan's block sums, so that nothing is allocated inside the capture
        TIM_TRY(tim_ensure(c, c->scratch_e, ((n + 4095) / 4096 + 1) * sizeof(unsigned long long)));
        if (!c->pool.p) TIM_TRY(tim_ensure(c, c->pool, 16));
        if (!c->pool_sid.p) TIM_TRY(tim_ensure(c, c->pool_sid, 16));
        if (!c->set_start.p) TIM_TRY(tim_ensure(c, c->set_start, 16));
        if (!c->set_len.p) TIM_TRY(tim_ensure(c, c->set_len, 16));
        GreedyDesc& d = gd[i];
        d.pool = (const uint32_t*)c->pool.p;
        d.pool_sid = (const uint32_t*)c->pool_sid.p;
        d.members = c->members;
        d.set_start = (const uint64_t*)c->set_start.p;
        d.set_len = (const uint32_t*)c->set_len.p;
        d.counts = (int*)c->counts.p;
        d.node_off = (uint64_t*)c->node_off.p;
        d.cursor = (uint32_t*)c->cursor.p;
        d.node_sets = (uint32_t*)c->node_sets.p;
        d.covered = (uint8_t*)c->covered.p;
        d.chosen = (uint8_t*)c->chosen.p;
        d.best = (unsigned long long*)c->best.p;
        d.seeds = (int32_t*)c->seeds_dev.p;
        d.n = n;
        d.k = k;
        d.pad = 0;
    }
    // blocks per query in proportion to its work: nodes (argmax) and members (index,
    // cover); every query gets at least one block
    const unsigned total_blocks = (unsigned)std::max(nq, owner->num_sms * 8);
    std::vector<unsigned> bs_nodes(nq + 1, 0), bs_memb(nq + 1, 0);
    {
        double wn = 0, wm = 0;
        for (int i = 0; i < nq; i++) {
            wn += (double)gd[i].n;
            wm += (double)gd[i].members + 1.0;
        }
        for (int i = 0; i < nq; i++) {
            bs_nodes[i + 1] = bs_nodes[i] +
                              std::max(1u, (unsigned)(total_blocks * ((double)gd[i].n / wn)));
            bs_memb[i + 1] = bs_memb[i] + std::max(1u, (unsigned)(total_blocks *
                                                                  (((double)gd[i].members + 1.0) / wm)));
        }
    }
    // descriptors | covered counters | block starts (nodes) | block starts (members)
    const size_t off_cov = ((size_t)nq * sizeof(GreedyDesc) + 255) & ~size_t(255);
    const size_t off_bn = (off_cov + (size_t)nq * 8 + 255) & ~size_t(255);
    const size_t off_bm = (off_bn + (size_t)(nq + 1) * 4 + 255) & ~size_t(255);
    TIM_TRY(tim_ensure(owner, owner->greedy_batch, off_bm + (size_t)(nq + 1) * 4));
    GreedyDesc* d_gd = (GreedyDesc*)owner->greedy_batch.p;
    unsigned long long* d_cov = (unsigned long long*)((char*)owner->greedy_batch.p + off_cov);
    unsigned* d_bn = (unsigned*)((char*)owner->greedy_batch.p + off_bn);
    unsigned* d_bm = (unsigned*)((char*)owner->greedy_batch.p + off_bm);
    for (int i = 0; i < nq; i++) gd[i].ncov = d_cov + i;
    cudaStream_t st = owner->stream;
    CUDA_TRY(owner, cudaMemcpyAsync(d_gd, gd.data(), (size_t)nq * sizeof(GreedyDesc),
                                    cudaMemcpyHostToDevice, st));
    CUDA_TRY(owner, cudaMemcpyAsync(d_bn, bs_nodes.data(), (size_t)(nq + 1) * 4,
                                    cudaMemcpyHostToDevice, st));
    CUDA_TRY(owner, cudaMemcpyAsync(d_bm, bs_memb.data(), (size_t)(nq + 1) * 4,
                                    cudaMemcpyHostToDevice, st));
    CUDA_TRY(owner, cudaStreamSynchronize(st));
    std::vector<cudaStream_t> saved(nq);
    for (int i = 0; i < nq; i++) {
        saved[i] = ctxs[i]->stream;
        ctxs[i]->stream = st;
    }
    cudaGraph_t graph = nullptr;
    int rc = TIM_OK;
    if (use_graph &&
        cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        use_graph = false;
    }
    do {
        if ((rc = tim_cuda_check(owner, cudaMemsetAsync(d_cov, 0, (size_t)nq * 8, st), "memset")))
            break;
        for (int i = 0; i < nq && rc == TIM_OK; i++) {
            const GreedyDesc& d = gd[i];
            if ((rc = tim_cuda_check(owner, cudaMemsetAsync(d.counts, 0, (d.n + 1) * 4, st), "memset")))
                break;
            if ((rc = tim_cuda_check(owner, cudaMemsetAsync(d.cursor, 0, (d.n + 1) * 4, st), "memset")))
                break;
            if ((rc = tim_cuda_check(owner, cudaMemsetAsync(d.covered, 0, ctxs[i]->n_sets + 1, st),
                                     "memset")))
                break;
            if ((rc = tim_cuda_check(owner, cudaMemsetAsync(d.chosen, 0, d.n + 1, st), "memset")))
                break;
            if ((rc = tim_cuda_check(owner, cudaMemsetAsync(d.best, 0, (size_t)d.k * 8, st), "memset")))
                break;
        }
        if (rc) break;
        mcount_kernel<<<bs_memb[nq], 256, 0, st>>>(d_gd, d_bm, nq);
        owner->launches++;
        for (int i = 0; i < nq && rc == TIM_OK; i++)
            rc = tim_scan_u32_to_u64(ctxs[i], (const uint32_t*)gd[i].counts, gd[i].node_off, gd[i].n);
        if (rc) break;
        mscatter_kernel<<<bs_memb[nq], 256, 0, st>>>(d_gd, d_bm, nq);
        owner->launches++;
        for (int r = 0; r < kmax; r++) {
            margmax_kernel<<<bs_nodes[nq], 512, 0, st>>>(d_gd, d_bn, nq, r);
            mcover_kernel<<<bs_memb[nq], 256, 0, st>>>(d_gd, d_bm, nq, r);
            owner->launches += 2;
        }
        rc = tim_cuda_check(owner, cudaGetLastError(), "batched greedy kernels");
    } while (0);
    if (use_graph) {
        cudaError_t e = cudaStreamEndCapture(st, &graph);
        if (rc == TIM_OK && e != cudaSuccess) rc = tim_cuda_check(owner, e, "cudaStreamEndCapture");
        if (rc == TIM_OK) {
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            if (e == cudaSuccess) {
                e = cudaGraphLaunch(exec, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                cudaGraphExecDestroy(exec);
            }
            rc = tim_cuda_check(owner, e, "batched greedy graph");
        }
        if (graph) cudaGraphDestroy(graph);
    }
    for (int i = 0; i < nq; i++) ctxs[i]->stream = saved[i];
    if (rc) return rc;
    std::vector<unsigned long long> hc(nq);
    CUDA_TRY(owner, cudaMemcpyAsync(hc.data(), d_cov, (size_t)nq * 8, cudaMemcpyDeviceToHost, st));
    for (int i = 0; i < nq; i++)
        if (host_seeds && host_seeds[i])
            CUDA_TRY(owner, cudaMemcpyAsync(host_seeds[i], gd[i].seeds, (size_t)gd[i].k * 4,
                                            cudaMemcpyDeviceToHost, st));
    CUDA_TRY(owner, cudaStreamSynchronize(st));
    for (int i = 0; i < nq; i++)
        if (covered) covered[i] = hc[i];
    return TIM_OK;
}
