// prims.cu -- device primitives: exclusive scan and a stable LSD radix sort of
// (key, value) pairs. Used to build G^T and the node -> RR-set index.
#include "common.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 4096

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the exclusive prefix and
// the block total via *total.
__device__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* total) {
    __shared__ unsigned long long warp_tot[33];  // [32] holds the block total
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    unsigned long long inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        unsigned long long t = lane < nw ? warp_tot[lane] : 0ull;
        unsigned long long ti = warp_incl_scan(t);
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == nw - 1) warp_tot[32] = ti;
    }
    __syncthreads();
    unsigned long long res = warp_tot[wid] + inc - v;
    *total = warp_tot[32];
    __syncthreads();
    return res;
}

template <class TIn>
__global__ void scan_reduce_kernel(const TIn* __restrict__ in, uint64_t count,
                                   unsigned long long* __restrict__ block_sums) {
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        uint64_t idx = base + (uint64_t)i * SCAN_THREADS + threadIdx.x;
        if (idx < count) s += in[idx];
    }
    unsigned long long tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// One block scans the per-tile sums sequentially in chunks; writes the grand total to
// out_total.
__global__ void scan_block_sums_kernel(unsigned long long* __restrict__ sums, uint64_t nblocks,
                                       uint64_t* __restrict__ out_total) {
    unsigned long long carry = 0;
    for (uint64_t base = 0; base < nblocks; base += blockDim.x) {
        uint64_t idx = base + threadIdx.x;
        unsigned long long v = idx < nblocks ? sums[idx] : 0ull;
        unsigned long long tot;
        unsigned long long ex = block_excl_scan(v, &tot);
        if (idx < nblocks) sums[idx] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *out_total = carry;
}

template <class TIn>
__global__ void scan_apply_kernel(const TIn* __restrict__ in, uint64_t count,
                                  const unsigned long long* __restrict__ block_off,
                                  uint64_t* __restrict__ out) {
    // blocked layout: thread t owns SCAN_ITEMS consecutive elements
    // padded index: one extra word per 32 keeps the blocked read free of bank conflicts
    __shared__ TIn tile[SCAN_TILE + SCAN_TILE / 32];
    uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int x = i * SCAN_THREADS + threadIdx.x;
        uint64_t idx = base + (uint64_t)x;
        tile[x + (x >> 5)] = idx < count ? in[idx] : (TIn)0;
    }
    __syncthreads();
    TIn loc[SCAN_ITEMS];
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        int x = threadIdx.x * SCAN_ITEMS + i;
        loc[i] = tile[x + (x >> 5)];
        s += loc[i];
    }
    unsigned long long tot;
    unsigned long long ex = block_excl_scan(s, &tot) + block_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        uint64_t idx = base + (uint64_t)threadIdx.x * SCAN_ITEMS + i;
        if (idx < count) out[idx] = ex;
        ex += loc[i];
    }
}

// ---------------------------------------------------------------- radix sort

constexpr int RS_WARPS = 8;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_WARPS * RS_ROUNDS * 32;  // 2048 keys per block
constexpr int RS_BINS = 256;

__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, uint64_t count, int shift,
                                  uint64_t ntiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[RS_BINS];
    for (int i = threadIdx.x; i < RS_BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += blockDim.x) {
        uint64_t idx = base + i;
        if (idx < count) atomicAdd(&h[(keys[idx] >> shift) & (RS_BINS - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += blockDim.x)
        hist[(uint64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter of one tile: warp w owns keys [w*256, (w+1)*256) of the tile, taken
// 32 at a time in order; equal digits are ranked by __match_any_sync, so the order of
// equal digits is the input order.
__global__ void __launch_bounds__(RS_WARPS * 32)
radix_scatter_kernel(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                     uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                     uint64_t count, int shift, uint64_t ntiles,
                     const uint64_t* __restrict__ offsets) {
    __shared__ uint32_t run[RS_WARPS][RS_BINS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += blockDim.x) (&run[0][0])[i] = 0;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t kk[RS_ROUNDS], vv[RS_ROUNDS], rank[RS_ROUNDS];
    uint64_t base = (uint64_t)blockIdx.x * RS_TILE + (uint64_t)w * (RS_ROUNDS * 32);
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        uint64_t idx = base + (uint64_t)r * 32 + lane;
        bool valid = idx < count;
        kk[r] = valid ? keys_in[idx] : 0u;
        vv[r] = valid ? vals_in[idx] : 0u;
        uint32_t d = (kk[r] >> shift) & (RS_BINS - 1);
        uint32_t tag = valid ? d : (RS_BINS + lane);
        uint32_t peers = __match_any_sync(0xffffffffu, tag);
        uint32_t before = (valid ? run[w][d] : 0u);
        rank[r] = before + __popc(peers & lt_mask);
        __syncwarp();
        if (valid && (peers & lt_mask) == 0) run[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += blockDim.x) {
        uint32_t acc = 0;
        for (int ww = 0; ww < RS_WARPS; ww++) {
            uint32_t t = run[ww][d];
            run[ww][d] = acc;
            acc += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        uint64_t idx = base + (uint64_t)r * 32 + lane;
        if (idx < count) {
            uint32_t d = (kk[r] >> shift) & (RS_BINS - 1);
            uint64_t pos = offsets[(uint64_t)d * ntiles + blockIdx.x] + run[w][d] + rank[r];
            keys_out[pos] = kk[r];
            vals_out[pos] = vv[r];
        }
    }
}

}  // namespace

template <class TIn>
static int scan_to_u64(tim_ctx* ctx, const TIn* in, uint64_t* out, uint64_t count) {
    uint64_t nblocks = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (nblocks == 0) {
        CUDA_TRY(ctx, cudaMemsetAsync(out, 0, sizeof(uint64_t), ctx->stream));
        return TIM_OK;
    }
    TIM_TRY(tim_ensure(ctx, ctx->scratch_e, nblocks * sizeof(unsigned long long)));
    auto* sums = (unsigned long long*)ctx->scratch_e.p;
    scan_reduce_kernel<TIn><<<(unsigned)nblocks, SCAN_THREADS, 0, ctx->stream>>>(in, count, sums);
    LAUNCH_CHECK(ctx, "scan_reduce_kernel");
    scan_block_sums_kernel<<<1, 1024, 0, ctx->stream>>>(sums, nblocks, out + count);
    LAUNCH_CHECK(ctx, "scan_block_sums_kernel");
    scan_apply_kernel<TIn><<<(unsigned)nblocks, SCAN_THREADS, 0, ctx->stream>>>(in, count, sums,
                                                                               out);
    LAUNCH_CHECK(ctx, "scan_apply_kernel");
    return TIM_OK;
}

int tim_scan_u32_to_u64(tim_ctx* ctx, const uint32_t* in, uint64_t* out, uint64_t count) {
    return scan_to_u64<uint32_t>(ctx, in, out, count);
}

int tim_scan_u64(tim_ctx* ctx, const unsigned long long* in, uint64_t* out, uint64_t count) {
    return scan_to_u64<unsigned long long>(ctx, in, out, count);
}

int tim_radix_sort_pairs(tim_ctx* ctx, uint32_t* keys, uint32_t* vals, uint64_t count, int bits) {
    if (count <= 1 || bits <= 0) return TIM_OK;
    uint64_t ntiles = (count + RS_TILE - 1) / RS_TILE;
    uint64_t nh = ntiles * RS_BINS;
    TIM_TRY(tim_ensure(ctx, ctx->scratch_a, count * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->scratch_b, count * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->scratch_c, nh * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->scratch_d, (nh + 1) * sizeof(uint64_t)));
    uint32_t* k_alt = (uint32_t*)ctx->scratch_a.p;
    uint32_t* v_alt = (uint32_t*)ctx->scratch_b.p;
    uint32_t* hist = (uint32_t*)ctx->scratch_c.p;
    uint64_t* offs = (uint64_t*)ctx->scratch_d.p;
    uint32_t *kin = keys, *vin = vals, *kout = k_alt, *vout = v_alt;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; p++) {
        int shift = 8 * p;
        radix_hist_kernel<<<(unsigned)ntiles, 256, 0, ctx->stream>>>(kin, count, shift, ntiles,
                                                                     hist);
        LAUNCH_CHECK(ctx, "radix_hist_kernel");
        TIM_TRY(tim_scan_u32_to_u64(ctx, hist, offs, nh));
        radix_scatter_kernel<<<(unsigned)ntiles, RS_WARPS * 32, 0, ctx->stream>>>(
            kin, vin, kout, vout, count, shift, ntiles, offs);
        LAUNCH_CHECK(ctx, "radix_scatter_kernel");
        uint32_t* t;
        t = kin; kin = kout; kout = t;
        t = vin; vin = vout; vout = t;
    }
    if (kin != keys) {
        CUDA_TRY(ctx, cudaMemcpyAsync(keys, kin, count * sizeof(uint32_t),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(vals, vin, count * sizeof(uint32_t),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return TIM_OK;
}
