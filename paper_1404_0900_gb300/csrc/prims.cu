// prims.cu -- device primitives: exclusive scan and a stable LSD radix sort of
// (key, value, value) triples. Used to build G^T.
#include <utility>

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

// 8 warps x 6 rounds of 32 keys: tiles of 1536 keep the kernel at 64 registers, four
// blocks per SM (4096-key tiles needed 127, two blocks); timed on the largest graph
constexpr int RS_WARPS = 8;
constexpr int RS_ROUNDS = 6;
constexpr int RS_TILE = RS_WARPS * RS_ROUNDS * 32;  // 1536 keys per block
constexpr int RS_MAXBINS = 256;
// dynamic shared memory of the scatter: the tile's keys and two value arrays in digit
// order, per-warp digit counts, the tile's digit starts
constexpr size_t RS_SMEM = (size_t)RS_TILE * 3 * sizeof(uint32_t) +
                           (size_t)RS_WARPS * RS_MAXBINS * sizeof(uint32_t) +
                           RS_MAXBINS * sizeof(uint32_t);

__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, uint64_t count, int shift,
                                  uint32_t mask, uint64_t ntiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[RS_MAXBINS];
    for (int i = threadIdx.x; i <= (int)mask; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += blockDim.x) {
        const uint64_t idx = base + i;
        if (idx < count) atomicAdd(&h[(keys[idx] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d <= (int)mask; d += blockDim.x)
        hist[(uint64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter of one tile of (key, a, b): warp w owns elements [w*192, (w+1)*192) of
// the tile, taken 32 at a time in order, ranked among equal digits by __match_any_sync
// (so equal digits keep the input order). The tile is first rearranged in shared memory
// into digit order, then written out so that consecutive threads write consecutive
// positions of each digit's run (coalesced stores).
__global__ void __launch_bounds__(RS_WARPS * 32)
radix_scatter3_kernel(const uint32_t* __restrict__ k_in, const uint32_t* __restrict__ a_in,
                      const uint32_t* __restrict__ b_in, uint32_t* __restrict__ k_out,
                      uint32_t* __restrict__ a_out, uint32_t* __restrict__ b_out,
                      uint64_t count, int shift, uint32_t mask, uint64_t ntiles,
                      const uint64_t* __restrict__ offsets, int* __restrict__ err) {
    extern __shared__ uint32_t rs_smem[];
    __shared__ unsigned long long goff[RS_MAXBINS];  // the tile's output start per digit
    uint32_t* sk = rs_smem;
    uint32_t* sa = sk + RS_TILE;
    uint32_t* sb = sa + RS_TILE;
    uint32_t* run = sb + RS_TILE;              // [RS_WARPS][RS_MAXBINS]
    uint32_t* dstart = run + RS_WARPS * RS_MAXBINS;  // [RS_MAXBINS]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t nbins = mask + 1;
    // loaded now, read after the ranking: the write-out needs no global load per element
    for (uint32_t d = threadIdx.x; d < nbins; d += blockDim.x)
        goff[d] = offsets[(uint64_t)d * ntiles + blockIdx.x];
    for (int i = threadIdx.x; i < RS_WARPS * RS_MAXBINS; i += blockDim.x) run[i] = 0;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint64_t tile0 = (uint64_t)blockIdx.x * RS_TILE;
    const uint64_t base = tile0 + (uint64_t)w * (RS_ROUNDS * 32);
    uint32_t kk[RS_ROUNDS], aa[RS_ROUNDS], bb[RS_ROUNDS], rank[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        const uint64_t idx = base + (uint64_t)r * 32 + lane;
        const bool valid = idx < count;
        kk[r] = valid ? k_in[idx] : 0u;
        aa[r] = valid ? a_in[idx] : 0u;
        bb[r] = valid ? b_in[idx] : 0u;
    }
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        const uint64_t idx = base + (uint64_t)r * 32 + lane;
        const bool valid = idx < count;
        const uint32_t d = (kk[r] >> shift) & mask;
        const uint32_t tag = valid ? d : (RS_MAXBINS + lane);
        const uint32_t peers = __match_any_sync(0xffffffffu, tag);
        const uint32_t before = valid ? run[w * RS_MAXBINS + d] : 0u;
        rank[r] = before + __popc(peers & lt_mask);
        __syncwarp();
        if (valid && (peers & lt_mask) == 0) run[w * RS_MAXBINS + d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: prefix over the warps, and the digit's count in the tile
    uint32_t dcount = 0;
    if (threadIdx.x < nbins) {
        uint32_t acc = 0;
        for (int ww = 0; ww < RS_WARPS; ww++) {
            const uint32_t t = run[ww * RS_MAXBINS + threadIdx.x];
            run[ww * RS_MAXBINS + threadIdx.x] = acc;
            acc += t;
        }
        dcount = acc;
    }
    unsigned long long tot;
    const unsigned long long ds = block_excl_scan(dcount, &tot);  // nbins <= blockDim.x
    if (threadIdx.x < nbins) dstart[threadIdx.x] = (uint32_t)ds;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; r++) {
        const uint64_t idx = base + (uint64_t)r * 32 + lane;
        if (idx < count) {
            const uint32_t d = (kk[r] >> shift) & mask;
            const uint32_t lp = dstart[d] + run[w * RS_MAXBINS + d] + rank[r];
            if (lp < RS_TILE) {
                sk[lp] = kk[r];
                sa[lp] = aa[r];
                sb[lp] = bb[r];
            } else {
                atomicOr(err, TIM_DEV_ERR_BOUNDS);
            }
        }
    }
    __syncthreads();
    const uint32_t n_tile = (uint32_t)min((uint64_t)RS_TILE, count - tile0);
    for (uint32_t i = threadIdx.x; i < n_tile; i += blockDim.x) {
        const uint32_t k = sk[i];
        const uint32_t d = (k >> shift) & mask;
        const uint64_t pos = goff[d] + (i - dstart[d]);
        if (i < dstart[d] || pos >= count) {  // cannot happen for a consistent tile
            atomicOr(err, TIM_DEV_ERR_BOUNDS);
            continue;
        }
        k_out[pos] = k;
        a_out[pos] = sa[i];
        b_out[pos] = sb[i];
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

int tim_radix_sort_triples_from(tim_ctx* ctx, const uint32_t* k0, const uint32_t* a0,
                                const uint32_t* b0, uint32_t* keys, uint32_t* va, uint32_t* vb,
                                uint64_t count, int bits) {
    auto copy_to = [&](const uint32_t* k, const uint32_t* a, const uint32_t* b) -> int {
        if (k != keys)
            CUDA_TRY(ctx, cudaMemcpyAsync(keys, k, count * sizeof(uint32_t),
                                          cudaMemcpyDeviceToDevice, ctx->stream));
        if (a != va)
            CUDA_TRY(ctx, cudaMemcpyAsync(va, a, count * sizeof(uint32_t),
                                          cudaMemcpyDeviceToDevice, ctx->stream));
        if (b != vb)
            CUDA_TRY(ctx, cudaMemcpyAsync(vb, b, count * sizeof(uint32_t),
                                          cudaMemcpyDeviceToDevice, ctx->stream));
        return TIM_OK;
    };
    if (count <= 1 || bits <= 0) return count ? copy_to(k0, a0, b0) : TIM_OK;
    // passes of at most 8 bits, the digit width spread evenly over them (26 bits: four
    // passes of 7 bits; fewer bins make longer runs per tile)
    const int passes = (bits + 7) / 8;
    const int width = (bits + passes - 1) / passes;
    const uint32_t mask = (1u << width) - 1u;
    const uint64_t ntiles = (count + RS_TILE - 1) / RS_TILE;
    const uint64_t nh = ntiles * (mask + 1);
    TIM_TRY(tim_ensure(ctx, ctx->scratch_a, count * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->scratch_b, count * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->scratch_f, count * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->scratch_c, nh * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->scratch_d, (nh + 1) * sizeof(uint64_t)));
    CUDA_TRY(ctx, cudaFuncSetAttribute(radix_scatter3_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_SMEM));
    uint32_t* hist = (uint32_t*)ctx->scratch_c.p;
    uint64_t* offs = (uint64_t*)ctx->scratch_d.p;
    // pass p writes the scratch arrays when p is even and the destination when p is odd,
    // so that the first pass may read the caller's arrays (which may be the destination's)
    uint32_t* const S[3] = {(uint32_t*)ctx->scratch_a.p, (uint32_t*)ctx->scratch_b.p,
                            (uint32_t*)ctx->scratch_f.p};
    uint32_t* const D[3] = {keys, va, vb};
    const uint32_t *kin = k0, *ain = a0, *bin = b0;
    for (int p = 0; p < passes; p++) {
        const int shift = width * p;
        uint32_t* const* out = (p % 2 == 0) ? S : D;
        radix_hist_kernel<<<(unsigned)ntiles, 256, 0, ctx->stream>>>(kin, count, shift, mask,
                                                                     ntiles, hist);
        LAUNCH_CHECK(ctx, "radix_hist_kernel");
        TIM_TRY(tim_scan_u32_to_u64(ctx, hist, offs, nh));
        radix_scatter3_kernel<<<(unsigned)ntiles, RS_WARPS * 32, RS_SMEM, ctx->stream>>>(
            kin, ain, bin, out[0], out[1], out[2], count, shift, mask, ntiles, offs,
            &tim_dscal(ctx)->err);
        LAUNCH_CHECK(ctx, "radix_scatter3_kernel");
        kin = out[0];
        ain = out[1];
        bin = out[2];
    }
    return copy_to(kin, ain, bin);
}

int tim_radix_sort_triples(tim_ctx* ctx, uint32_t* keys, uint32_t* va, uint32_t* vb,
                           uint64_t count, int bits) {
    return tim_radix_sort_triples_from(ctx, keys, va, vb, keys, va, vb, count, bits);
}
