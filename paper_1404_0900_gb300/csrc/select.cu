// select.cu -- greedy maximum coverage over the RR-set store (Algorithm 1, lines 3-7;
// also lines 2-6 of Algorithm 3).
//
// Index: coverage counts (how many stored sets contain each node) by a histogram over
// the store, an exclusive scan into node offsets, and a scatter of set ids into
// per-node lists (node -> sets).
// Greedy round r: an argmax over the counts with a warp-shuffle reduction of the key
// (count << 32 | ~node) so ties go to the smallest id and chosen nodes are skipped;
// then every not-yet-covered set in the chosen node's list is marked covered and each
// of its members loses one from its count. The chosen node is read on the device, so
// the k rounds run without host round trips.
#include "common.cuh"

namespace {

__global__ void count_members_kernel(const uint32_t* __restrict__ pool, uint64_t members,
                                     uint32_t* __restrict__ cnt) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < members;
         p += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[pool[p]], 1u);
}

__global__ void scatter_sets_kernel(const uint32_t* __restrict__ pool,
                                    const uint32_t* __restrict__ pool_sid, uint64_t members,
                                    const uint64_t* __restrict__ node_off,
                                    uint32_t* __restrict__ cursor,
                                    uint32_t* __restrict__ node_sets) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < members;
         p += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = pool[p];
        uint32_t slot = atomicAdd(&cursor[u], 1u);
        node_sets[node_off[u] + slot] = pool_sid[p];
    }
}

__device__ __forceinline__ unsigned long long greedy_key(int cnt, uint32_t v) {
    return ((unsigned long long)(uint32_t)max(cnt, 0) << 32) | (unsigned long long)(~v);
}

__global__ void argmax_kernel(const int* __restrict__ counts, const uint8_t* __restrict__ chosen,
                              uint64_t n, unsigned long long* __restrict__ best) {
    unsigned long long b = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        if (!chosen[v]) {
            unsigned long long key = greedy_key(counts[v], (uint32_t)v);
            b = key > b ? key : b;
        }
    }
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

}  // namespace

int tim_build_index(tim_ctx* ctx) {
    const uint64_t n = (uint64_t)ctx->n, members = ctx->members;
    TIM_TRY(tim_ensure(ctx, ctx->counts, (n + 1) * sizeof(int)));
    TIM_TRY(tim_ensure(ctx, ctx->node_off, (n + 1) * sizeof(uint64_t)));
    TIM_TRY(tim_ensure(ctx, ctx->cursor, (n + 1) * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->node_sets, (members + 1) * sizeof(uint32_t)));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->counts.p, 0, (n + 1) * sizeof(int), ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->cursor.p, 0, (n + 1) * sizeof(uint32_t), ctx->stream));
    const unsigned G = (unsigned)(ctx->num_sms * 8);
    if (members) {
        count_members_kernel<<<G, 256, 0, ctx->stream>>>((const uint32_t*)ctx->pool.p, members,
                                                         (uint32_t*)ctx->counts.p);
        LAUNCH_CHECK(ctx, "count_members_kernel");
    }
    TIM_TRY(tim_scan_u32_to_u64(ctx, (const uint32_t*)ctx->counts.p, (uint64_t*)ctx->node_off.p, n));
    if (members) {
        scatter_sets_kernel<<<G, 256, 0, ctx->stream>>>(
            (const uint32_t*)ctx->pool.p, (const uint32_t*)ctx->pool_sid.p, members,
            (const uint64_t*)ctx->node_off.p, (uint32_t*)ctx->cursor.p,
            (uint32_t*)ctx->node_sets.p);
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
    const unsigned GA = (unsigned)(ctx->num_sms * 4);
    const unsigned GC = (unsigned)(ctx->num_sms * 2);
    auto* best = (unsigned long long*)ctx->best.p;
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
