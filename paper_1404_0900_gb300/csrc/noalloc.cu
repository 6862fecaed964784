// noalloc.cu -- tim_node_select_noalloc: the greedy node selection of tim_node_select
// (node -> set index, exclusive scan, k rounds of argmax and cover) over a CSR of RR
// sets that the caller owns, for callers that cannot let the library allocate device
// memory: code whose device memory is owned by another allocator or a fixed budget,
// and code that must not trigger the device-wide synchronisation that cudaMalloc and
// cudaFree imply. Nothing here calls cudaMalloc, cudaFree or an allocating library.
//
// All scratch lives in one file-scope __device__ array of NA_SCRATCH_BYTES (about
// 13.3 MiB), which every GPU that loads the library holds until the process exits. Host code
// cannot use the array's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device current) and keeps
// it; make that first call before any stream capture. Every call also reads two
// offsets back to the host and waits for its stream. Every call shares the array and
// leaves its contents behind: each call clears what must start at zero, and calls
// whose work overlaps on the GPU (other streams, other host threads) race. Members
// must be distinct within a set; a repeated member is not detected.
#include <mutex>

#include "common.cuh"

namespace {

// Limits of the caller's problem, fixed by the size of the scratch array.
constexpr int64_t NA_MAX_NODES = 1 << 18;        // n
constexpr uint64_t NA_MAX_SETS = 1 << 20;        // number of RR sets
constexpr uint64_t NA_MAX_MEMBERS = 1 << 21;     // sum of |R|
constexpr int NA_MAX_K = 1024;                   // seeds
constexpr int NA_SCAN_TILE = 4096;
constexpr uint64_t NA_SCAN_BLOCKS = (NA_MAX_NODES + NA_SCAN_TILE - 1) / NA_SCAN_TILE + 1;

// Layout of the scratch array (byte offsets, each a multiple of 256).
constexpr uint64_t al(uint64_t x) { return (x + 255) & ~uint64_t(255); }
constexpr uint64_t OFF_COUNTS = 0;                                           // int32[n]
constexpr uint64_t OFF_NODE_OFF = al(OFF_COUNTS + 4 * NA_MAX_NODES);         // u64[n+1]
constexpr uint64_t OFF_CURSOR = al(OFF_NODE_OFF + 8 * (NA_MAX_NODES + 1));   // u32[n]
constexpr uint64_t OFF_NODE_SETS = al(OFF_CURSOR + 4 * NA_MAX_NODES);        // u32[members]
constexpr uint64_t OFF_COVERED = al(OFF_NODE_SETS + 4 * NA_MAX_MEMBERS);     // u8[sets]
constexpr uint64_t OFF_CHOSEN = al(OFF_COVERED + NA_MAX_SETS);               // u8[n]
constexpr uint64_t OFF_BEST = al(OFF_CHOSEN + NA_MAX_NODES);                 // u64[k]
constexpr uint64_t OFF_SUMS = al(OFF_BEST + 8 * NA_MAX_K);                   // u64[blocks]
constexpr uint64_t OFF_FLAGS = al(OFF_SUMS + 8 * NA_SCAN_BLOCKS);            // u64[4]
constexpr uint64_t NA_SCRATCH_BYTES = al(OFF_FLAGS + 32);

static __device__ __align__(256) unsigned char na_scratch[NA_SCRATCH_BYTES];

struct NaView {
    int* counts;
    uint64_t* node_off;
    uint32_t* cursor;
    uint32_t* node_sets;
    uint8_t* covered;
    uint8_t* chosen;
    unsigned long long* best;
    unsigned long long* sums;
    unsigned long long* flags;  // [0] covered count, [1] error bits
};

NaView view_of(unsigned char* base) {
    NaView v;
    v.counts = (int*)(base + OFF_COUNTS);
    v.node_off = (uint64_t*)(base + OFF_NODE_OFF);
    v.cursor = (uint32_t*)(base + OFF_CURSOR);
    v.node_sets = (uint32_t*)(base + OFF_NODE_SETS);
    v.covered = base + OFF_COVERED;
    v.chosen = base + OFF_CHOSEN;
    v.best = (unsigned long long*)(base + OFF_BEST);
    v.sums = (unsigned long long*)(base + OFF_SUMS);
    v.flags = (unsigned long long*)(base + OFF_FLAGS);
    return v;
}

// Histogram of members; members outside [0, n) are skipped and flagged.
__global__ void na_count_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ mem,
                                uint64_t n_sets, int64_t n, NaView v) {
    const uint64_t members = (uint64_t)off[n_sets];
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < members;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t u = mem[p];
        if (u < 0 || u >= n) {
            atomicOr(&v.flags[1], 1ull);
            continue;
        }
        atomicAdd(&v.counts[u], 1);
    }
}

// Exclusive scan of the counts into node_off (one block per 4096 entries, then one
// block over the block sums, then the fix-up), as in the library's own scan.
__device__ unsigned long long na_block_scan(unsigned long long x, unsigned long long* total) {
    __shared__ unsigned long long wsum[33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = lane < nw ? wsum[lane] : 0ull, ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < nw) wsum[lane] = ti - t;
        if (lane == nw - 1) wsum[32] = ti;
    }
    __syncthreads();
    const unsigned long long r = wsum[w] + inc - x;
    *total = wsum[32];
    __syncthreads();
    return r;
}

__global__ void na_scan_sums_kernel(int64_t n, NaView v) {
    const uint64_t base = (uint64_t)blockIdx.x * NA_SCAN_TILE;
    unsigned long long s = 0;
    for (int i = threadIdx.x; i < NA_SCAN_TILE; i += blockDim.x)
        if (base + i < (uint64_t)n) s += (uint32_t)v.counts[base + i];
    unsigned long long tot;
    na_block_scan(s, &tot);
    if (threadIdx.x == 0) v.sums[blockIdx.x] = tot;
}

__global__ void na_scan_top_kernel(uint64_t nblocks, int64_t n, NaView v) {
    unsigned long long carry = 0;
    for (uint64_t b = 0; b < nblocks; b += blockDim.x) {
        const uint64_t i = b + threadIdx.x;
        const unsigned long long x = i < nblocks ? v.sums[i] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = na_block_scan(x, &tot);
        if (i < nblocks) v.sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) v.node_off[n] = carry;
}

__global__ void na_scan_apply_kernel(int64_t n, NaView v) {
    // each thread scans 16 consecutive counts of the block's 4096
    const uint64_t base = (uint64_t)blockIdx.x * NA_SCAN_TILE + (uint64_t)threadIdx.x * 16;
    unsigned long long loc = 0;
    for (int i = 0; i < 16; i++)
        if (base + i < (uint64_t)n) loc += (uint32_t)v.counts[base + i];
    unsigned long long tot;
    unsigned long long ex = na_block_scan(loc, &tot) + v.sums[blockIdx.x];
    for (int i = 0; i < 16; i++)
        if (base + i < (uint64_t)n) {
            v.node_off[base + i] = ex;
            ex += (uint32_t)v.counts[base + i];
        }
}

// node -> sets: one warp per set writes the set id into each member's list.
__global__ void na_scatter_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ mem,
                                  uint64_t n_sets, int64_t n, NaView v) {
    const int lane = threadIdx.x & 31;
    const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t members = off[n_sets];
    for (uint64_t s = w0; s < n_sets; s += nw) {
        const int64_t a = off[s], b = off[s + 1];
        if (a < 0 || b < a || b > members) {  // malformed offsets: flag, skip the set
            if (lane == 0) atomicOr(&v.flags[1], 2ull);
            continue;
        }
        for (int64_t p = a + lane; p < b; p += 32) {
            const int32_t u = mem[p];
            if (u < 0 || u >= n) continue;
            const uint32_t slot = atomicAdd(&v.cursor[u], 1u);
            if (v.node_off[u] + slot < v.node_off[u + 1])
                v.node_sets[v.node_off[u] + slot] = (uint32_t)s;
            else
                atomicOr(&v.flags[1], 2ull);
        }
    }
}

__global__ void na_argmax_kernel(int64_t n, NaView v, int r) {
    unsigned long long b = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (!v.chosen[u]) {
            const unsigned long long key =
                ((unsigned long long)(uint32_t)max(v.counts[u], 0) << 32) |
                (unsigned long long)(~(uint32_t)u);
            b = key > b ? key : b;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
        b = y > b ? y : b;
    }
    if ((threadIdx.x & 31) == 0 && b) atomicMax(&v.best[r], b);
}

__global__ void na_cover_kernel(const int64_t* __restrict__ off, const int32_t* __restrict__ mem,
                                uint64_t n_sets, int64_t n, NaView v, int r,
                                int32_t* __restrict__ seeds) {
    const unsigned long long key = v.best[r];
    if (key == 0) return;
    const uint32_t u = ~(uint32_t)(key & 0xFFFFFFFFull);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        v.chosen[u] = 1;
        seeds[r] = (int32_t)u;
    }
    const int lane = threadIdx.x & 31;
    const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t a = v.node_off[u], b = v.node_off[u + 1];
    unsigned long long fresh = 0;
    for (uint64_t i = a + w0; i < b; i += nw) {
        const uint32_t s = v.node_sets[i];
        if (v.covered[s]) continue;
        __syncwarp();
        if (lane == 0) {
            v.covered[s] = 1;
            fresh++;
        }
        const int64_t pa = off[s], pb = off[s + 1];
        if (pa < 0 || pb < pa || pb > off[n_sets]) continue;
        for (int64_t p = pa + lane; p < pb; p += 32) {
            const int32_t x = mem[p];
            if (x >= 0 && x < n) atomicSub(&v.counts[x], 1);
        }
    }
    if (lane == 0 && fresh) atomicAdd(&v.flags[0], fresh);
}

__global__ void na_finish_kernel(NaView v, uint64_t* covered_out) { *covered_out = v.flags[0]; }

std::mutex na_mutex;
unsigned char* na_base[64] = {};

}  // namespace

extern "C" int tim_node_select_noalloc(int device, void* cuda_stream, int64_t n, uint64_t n_sets,
                                       const int64_t* d_off, const int32_t* d_mem, int k,
                                       int32_t* d_seeds, uint64_t* d_covered) {
    if (device < 0 || device >= 64 || !d_off || !d_seeds || !d_covered) return TIM_ERR_ARG;
    if (n < 1 || n > NA_MAX_NODES || n_sets > NA_MAX_SETS || k < 1 || k > n || k > NA_MAX_K)
        return TIM_ERR_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return TIM_ERR_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return TIM_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = TIM_OK;
    do {
        unsigned char* base;
        {
            // once per device, with that device current: the device address of the array
            std::lock_guard<std::mutex> lock(na_mutex);
            if (!na_base[device]) {
                void* p = nullptr;
                if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || !p) {
                    cudaGetLastError();
                    rc = TIM_ERR_CUDA;
                    break;
                }
                na_base[device] = (unsigned char*)p;
            }
            base = na_base[device];
        }
        int64_t ends[2] = {0, 0};
        if (cudaMemcpyAsync(&ends[1], d_off + n_sets, sizeof(int64_t), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess ||
            cudaMemcpyAsync(&ends[0], d_off, sizeof(int64_t), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = TIM_ERR_CUDA;
            break;
        }
        if (ends[0] != 0 || ends[1] < 0 || (uint64_t)ends[1] > NA_MAX_MEMBERS || (n_sets > 0 && !d_mem)) {
            rc = TIM_ERR_ARG;
            break;
        }
        const NaView v = view_of(base);
        // clear what must start at zero
        if (cudaMemsetAsync(v.counts, 0, 4 * (size_t)n, st) != cudaSuccess ||
            cudaMemsetAsync(v.cursor, 0, 4 * (size_t)n, st) != cudaSuccess ||
            cudaMemsetAsync(v.chosen, 0, (size_t)n, st) != cudaSuccess ||
            cudaMemsetAsync(v.covered, 0, (size_t)n_sets + 1, st) != cudaSuccess ||
            cudaMemsetAsync(v.best, 0, 8 * (size_t)k, st) != cudaSuccess ||
            cudaMemsetAsync(v.flags, 0, 32, st) != cudaSuccess) {
            rc = TIM_ERR_CUDA;
            break;
        }
        const uint64_t nblocks = ((uint64_t)n + NA_SCAN_TILE - 1) / NA_SCAN_TILE;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        const unsigned G = (unsigned)(sms > 0 ? sms * 4 : 128);
        if (n_sets > 0) na_count_kernel<<<G, 256, 0, st>>>(d_off, d_mem, n_sets, n, v);
        na_scan_sums_kernel<<<(unsigned)nblocks, 256, 0, st>>>(n, v);
        na_scan_top_kernel<<<1, 256, 0, st>>>(nblocks, n, v);
        na_scan_apply_kernel<<<(unsigned)nblocks, 256, 0, st>>>(n, v);
        if (n_sets > 0) na_scatter_kernel<<<G, 256, 0, st>>>(d_off, d_mem, n_sets, n, v);
        for (int r = 0; r < k; r++) {
            na_argmax_kernel<<<G, 256, 0, st>>>(n, v, r);
            na_cover_kernel<<<G, 256, 0, st>>>(d_off, d_mem, n_sets, n, v, r, d_seeds);
        }
        na_finish_kernel<<<1, 1, 0, st>>>(v, d_covered);
        if (cudaGetLastError() != cudaSuccess) {
            rc = TIM_ERR_CUDA;
            break;
        }
        unsigned long long err = 0;
        if (cudaMemcpyAsync(&err, v.flags + 1, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = TIM_ERR_CUDA;
            break;
        }
        if (err) rc = TIM_ERR_ARG;
    } while (0);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
}
