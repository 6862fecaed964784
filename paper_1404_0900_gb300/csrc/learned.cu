// learned.cu -- the learned start round of Algorithm 2 (Section 3.2): kernels that
// pool graph features, and the forward, backward and Adam kernels of the small network
// that maps them to a predicted stopping round.
//
// The network is tiny (d_in x 64 x 64 x 1, about 5K parameters) and its batches are a
// few thousand graphs, so one training step is some 10 MFLOP: far too little work to
// feed the tensor cores. The kernels are plain fp32 FMA over shared-memory tiles, with
// the weight matrices rounded to bfloat16 after every update (the precision the weights
// are kept in) and every sum accumulated in fp32. Reductions over samples run in a
// fixed order (per-block partials, then a block-ordered sum), so gradients and
// training runs are reproducible bit for bit.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace {

constexpr int H = TIM_MLP_HIDDEN;     // hidden units
constexpr int DMAX = TIM_MLP_MAX_IN;  // largest input width
constexpr int SB = 32;                // samples per block
constexpr int FB_THREADS = 256;
constexpr int FEAT_THREADS = 256;
constexpr int FEAT_WARPS = FEAT_THREADS / 32;
constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------------ graph features

__global__ void feat_outdeg_kernel(const uint32_t* __restrict__ src, uint64_t m,
                                   uint32_t* __restrict__ outdeg) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&outdeg[src[e]], 1u);
}

// One warp per node (grid-stride in a fixed order): the four per-node features, summed
// per warp in fp64 and maxed, then per block in warp order.
__global__ void __launch_bounds__(FEAT_THREADS)
feat_node_kernel(const uint64_t* __restrict__ rowptr, const uint32_t* __restrict__ src,
                 const uint32_t* __restrict__ thr, int model, uint64_t n,
                 const uint32_t* __restrict__ outdeg, double* __restrict__ part_sum,
                 float* __restrict__ part_max) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t nwarps = (uint64_t)gridDim.x * FEAT_WARPS;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    float mx[4] = {0.f, 0.f, 0.f, 0.f};  // every feature is >= 0
    for (uint64_t v = blockIdx.x * (uint64_t)FEAT_WARPS + wib; v < n; v += nwarps) {
        const uint64_t a = rowptr[v], b = rowptr[v + 1];
        unsigned long long hop = 0, tsum = 0;
        for (uint64_t j = a + lane; j < b; j += 32) {
            const uint32_t u = src[j];
            hop += rowptr[u + 1] - rowptr[u];
            if (model == TIM_IC) tsum += thr[j];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hop += __shfl_xor_sync(FULL, hop, o);
            tsum += __shfl_xor_sync(FULL, tsum, o);
        }
        // LT thresholds are the inclusive cumulative in-weights: the last one is the total
        if (model == TIM_LT) tsum = b > a ? thr[b - 1] : 0u;
        const double f[4] = {log1p((double)(b - a)), log1p((double)outdeg[v]),
                             (double)tsum * 0x1p-32, log1p((double)hop)};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            s[q] += f[q];
            mx[q] = fmaxf(mx[q], (float)f[q]);
        }
    }
    __shared__ double ws[FEAT_WARPS][4];
    __shared__ float wm[FEAT_WARPS][4];
    if (lane == 0)
        for (int q = 0; q < 4; q++) {
            ws[wib][q] = s[q];
            wm[wib][q] = mx[q];
        }
    __syncthreads();
    if (threadIdx.x < 4) {
        const int q = threadIdx.x;
        double t = 0.0;
        float m = 0.f;
        for (int w = 0; w < FEAT_WARPS; w++) {
            t += ws[w][q];
            m = fmaxf(m, wm[w][q]);
        }
        part_sum[blockIdx.x * 4 + q] = t;
        part_max[blockIdx.x * 4 + q] = m;
    }
}

__global__ void feat_final_kernel(const double* __restrict__ part_sum,
                                  const float* __restrict__ part_max, int nblocks, uint64_t n,
                                  float* __restrict__ out) {
    const int q = threadIdx.x;
    if (q >= 4) return;
    double t = 0.0;
    float m = 0.f;
    for (int b = 0; b < nblocks; b++) {
        t += part_sum[b * 4 + q];
        m = fmaxf(m, part_max[b * 4 + q]);
    }
    out[2 * q] = (float)(t / (double)n);
    out[2 * q + 1] = m;
}

// ------------------------------------------------------------------------ network

struct Layout {
    int d;
    int oW1, ob1, oW2, ob2, oW3, ob3, P;
};

__host__ __device__ inline Layout layout_of(int d) {
    Layout L;
    L.d = d;
    L.oW1 = 0;
    L.ob1 = H * d;
    L.oW2 = L.ob1 + H;
    L.ob2 = L.oW2 + H * H;
    L.oW3 = L.ob2 + H;
    L.ob3 = L.oW3 + H;
    L.P = L.ob3 + 1;
    return L;
}

__device__ inline bool is_weight(const Layout& L, int p) {
    return p < L.ob1 || (p >= L.oW2 && p < L.ob2) || (p >= L.oW3 && p < L.ob3);
}

__device__ inline float gelu_f(float t) { return 0.5f * t * (1.0f + erff(t * 0.70710678118654752f)); }

__device__ inline float gelu_grad_f(float t) {
    return 0.5f * (1.0f + erff(t * 0.70710678118654752f)) +
           t * expf(-0.5f * t * t) * 0.39894228040143268f;
}

// shared-memory plan of mlp_fb_kernel, in floats
constexpr int SM_W1T = 0;                 // [DMAX][H]   W1 transposed
constexpr int SM_B1 = SM_W1T + DMAX * H;  // [H]
constexpr int SM_W2T = SM_B1 + H;         // [H][H]      W2t[j][i] = W2[i][j]
constexpr int SM_W2R = SM_W2T + H * H;    // [H][H]      W2 row-major
constexpr int SM_B2 = SM_W2R + H * H;     // [H]
constexpr int SM_W3 = SM_B2 + H;          // [H]
constexpr int SM_B3 = SM_W3 + H;          // [4]
constexpr int SM_X = SM_B3 + 4;           // [SB][DMAX]  normalised inputs
constexpr int SM_A1 = SM_X + SB * DMAX;   // [SB][H]     pre-activations, layer 1
constexpr int SM_H1 = SM_A1 + SB * H;
constexpr int SM_A2 = SM_H1 + SB * H;
constexpr int SM_H2 = SM_A2 + SB * H;
constexpr int SM_D2 = SM_H2 + SB * H;     // d loss / d a2
constexpr int SM_D1 = SM_D2 + SB * H;     // d loss / d a1
constexpr int SM_Z = SM_D1 + SB * H;      // [SB] outputs, then d loss / d z
constexpr int SM_L = SM_Z + SB;           // [SB] per-sample loss terms
constexpr int SM_FLOATS = SM_L + SB;
constexpr size_t SM_BYTES = (size_t)SM_FLOATS * sizeof(float);

struct FbArgs {
    const float* wq;      // parameters with the weight matrices rounded to bfloat16
    const float* in_mu;   // [d]
    const float* in_isd;  // [d]
    float out_mu, out_sd, inv_out_sd;
    const float* x;       // [N][d]
    const float* y;       // [N] targets (backward)
    uint32_t N;
    float inv_n;
    float* out;           // [N] predictions (forward only)
    float* part;          // [gridDim.x][P] gradient partials (backward)
    float* part_loss;     // [gridDim.x]
};

// One block = SB samples. Forward through both hidden layers; with BACKWARD, the loss
// terms and this block's share of the gradient, each partial written by one thread in
// a fixed sample order.
template <bool BACKWARD>
__global__ void __launch_bounds__(FB_THREADS) mlp_fb_kernel(FbArgs a, int d) {
    extern __shared__ float sm[];
    const Layout L = layout_of(d);
    const int t = threadIdx.x;
    const uint32_t base = blockIdx.x * SB;
    float* W1t = sm + SM_W1T;
    float* b1 = sm + SM_B1;
    float* W2t = sm + SM_W2T;
    float* W2r = sm + SM_W2R;
    float* b2 = sm + SM_B2;
    float* W3 = sm + SM_W3;
    float* X = sm + SM_X;
    float* A1 = sm + SM_A1;
    float* H1 = sm + SM_H1;
    float* A2 = sm + SM_A2;
    float* H2 = sm + SM_H2;
    float* D2 = sm + SM_D2;
    float* D1 = sm + SM_D1;
    float* Z = sm + SM_Z;
    float* Ls = sm + SM_L;

    for (int i = t; i < H * d; i += FB_THREADS) W1t[(i % d) * H + i / d] = a.wq[L.oW1 + i];
    for (int i = t; i < H * H; i += FB_THREADS) {
        const float w = a.wq[L.oW2 + i];
        W2r[i] = w;
        W2t[(i % H) * H + i / H] = w;
    }
    if (t < H) {
        b1[t] = a.wq[L.ob1 + t];
        b2[t] = a.wq[L.ob2 + t];
        W3[t] = a.wq[L.oW3 + t];
    }
    if (t == 0) sm[SM_B3] = a.wq[L.ob3];
    for (int i = t; i < SB * d; i += FB_THREADS) {
        const int s = i / d, k = i % d;
        const uint32_t g = base + s;
        X[s * DMAX + k] = g < a.N ? (a.x[(size_t)g * d + k] - a.in_mu[k]) * a.in_isd[k] : 0.f;
    }
    __syncthreads();

    const int j = t & (H - 1);  // unit of this thread
    const int s0 = t >> 6;      // first sample; samples s0, s0 + 4, ...
    for (int s = s0; s < SB; s += FB_THREADS / H) {
        float acc = b1[j];
        for (int k = 0; k < d; k++) acc = fmaf(W1t[k * H + j], X[s * DMAX + k], acc);
        A1[s * H + j] = acc;
        H1[s * H + j] = gelu_f(acc);
    }
    __syncthreads();
    for (int s = s0; s < SB; s += FB_THREADS / H) {
        float acc = b2[j];
        for (int k = 0; k < H; k++) acc = fmaf(W2t[k * H + j], H1[s * H + k], acc);
        A2[s * H + j] = acc;
        H2[s * H + j] = gelu_f(acc);
    }
    __syncthreads();
    {
        const int w = t >> 5, lane = t & 31;
        for (int q = 0; q < SB / (FB_THREADS / 32); q++) {
            const int s = w * (SB / (FB_THREADS / 32)) + q;
            float v = W3[lane] * H2[s * H + lane];
            v = fmaf(W3[lane + 32], H2[s * H + lane + 32], v);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            if (lane == 0) {
                const float z = v + sm[SM_B3];
                const uint32_t g = base + s;
                if (!BACKWARD) {
                    if (g < a.N) a.out[g] = a.out_mu + a.out_sd * z;
                } else {
                    const float diff = g < a.N ? z - (a.y[g] - a.out_mu) * a.inv_out_sd : 0.f;
                    Z[s] = diff * a.inv_n;
                    Ls[s] = 0.5f * diff * diff * a.inv_n;
                }
            }
        }
    }
    if (!BACKWARD) return;
    __syncthreads();
    float* part = a.part + (size_t)blockIdx.x * L.P;
    if (t < H) {  // output layer
        float g = 0.f;
        for (int s = 0; s < SB; s++) g = fmaf(Z[s], H2[s * H + t], g);
        part[L.oW3 + t] = g;
    } else if (t == H) {
        float g = 0.f, l = 0.f;
        for (int s = 0; s < SB; s++) {
            g += Z[s];
            l += Ls[s];
        }
        part[L.ob3] = g;
        a.part_loss[blockIdx.x] = l;
    }
    for (int s = s0; s < SB; s += FB_THREADS / H)
        D2[s * H + j] = Z[s] * W3[j] * gelu_grad_f(A2[s * H + j]);
    __syncthreads();
    // layer 2: gW2[i][j] = sum_s D2[s][i] H1[s][j]
    for (int i = s0; i < H; i += FB_THREADS / H) {
        float g = 0.f;
        for (int s = 0; s < SB; s++) g = fmaf(D2[s * H + i], H1[s * H + j], g);
        part[L.oW2 + i * H + j] = g;
    }
    if (t < H) {
        float g = 0.f;
        for (int s = 0; s < SB; s++) g += D2[s * H + t];
        part[L.ob2 + t] = g;
    }
    // back through W2: D1[s][j] = (sum_i W2[i][j] D2[s][i]) gelu'(A1[s][j])
    for (int s = s0; s < SB; s += FB_THREADS / H) {
        float acc = 0.f;
        for (int i = 0; i < H; i++) acc = fmaf(W2r[i * H + j], D2[s * H + i], acc);
        D1[s * H + j] = acc * gelu_grad_f(A1[s * H + j]);
    }
    __syncthreads();
    // layer 1: gW1[j][k] = sum_s D1[s][j] X[s][k]
    for (int i = t; i < H * d; i += FB_THREADS) {
        const int jj = i % H, k = i / H;
        float g = 0.f;
        for (int s = 0; s < SB; s++) g = fmaf(D1[s * H + jj], X[s * DMAX + k], g);
        part[L.oW1 + jj * d + k] = g;
    }
    if (t < H) {
        float g = 0.f;
        for (int s = 0; s < SB; s++) g += D1[s * H + t];
        part[L.ob1 + t] = g;
    }
}

// Sum the per-block partials in block order. With adam != 0, one Adam step on the fp32
// master copy and the bfloat16-rounded working copy; else the gradient goes to `grad`.
struct ReduceArgs {
    const float* part;
    const float* part_loss;
    int nb;
    float* grad;      // gradient out (no Adam)
    float* loss_out;  // summed loss (may be null)
    int adam;
    float* params;    // fp32 master
    float* wq;        // working copy
    float* m;
    float* v;
    float lr, c1, c2;  // c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
};

__global__ void mlp_reduce_kernel(ReduceArgs r, int d) {
    const Layout L = layout_of(d);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && r.loss_out) {
        float l = 0.f;
        for (int b = 0; b < r.nb; b++) l += r.part_loss[b];
        *r.loss_out = l;
    }
    if (p >= L.P) return;
    float g = 0.f;
    for (int b = 0; b < r.nb; b++) g += r.part[(size_t)b * L.P + p];
    if (!r.adam) {
        r.grad[p] = g;
        return;
    }
    const float m = 0.9f * r.m[p] + 0.1f * g;
    const float v = 0.999f * r.v[p] + 0.001f * g * g;
    r.m[p] = m;
    r.v[p] = v;
    const float w = r.params[p] - r.lr * (m * r.c1) / (sqrtf(v * r.c2) + 1e-8f);
    r.params[p] = w;
    r.wq[p] = is_weight(L, p) ? __bfloat162float(__float2bfloat16_rn(w)) : w;
}

__global__ void mlp_round_kernel(const float* __restrict__ params, float* __restrict__ wq,
                                 int d) {
    const Layout L = layout_of(d);
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.P) return;
    const float w = params[p];
    wq[p] = is_weight(L, p) ? __bfloat162float(__float2bfloat16_rn(w)) : w;
}

}  // namespace

struct tim_mlp {
    tim_ctx* ctx = nullptr;
    int d = 0;
    Layout L{};
    DevBuf params, wq, m, v, scal;  // scal: in_mu[DMAX], in_isd[DMAX]
    DevBuf x, y, out, part, ploss;
    DevBuf gbuf;  // gradient (tim_mlp_grad) or loss history (tim_mlp_train)
    float out_mu = 0.f, out_sd = 1.f;
    int step = 0;
};

static int mlp_upload(tim_mlp* mlp, const float* x, const float* y, uint64_t N) {
    tim_ctx* ctx = mlp->ctx;
    const size_t nb = (size_t)((N + SB - 1) / SB);
    TIM_TRY(tim_ensure(ctx, mlp->x, (size_t)N * mlp->d * sizeof(float)));
    TIM_TRY(tim_ensure(ctx, mlp->out, ((size_t)N + 1) * sizeof(float)));
    CUDA_TRY(ctx, cudaMemcpyAsync(mlp->x.p, x, (size_t)N * mlp->d * sizeof(float),
                                  cudaMemcpyHostToDevice, ctx->stream));
    if (y) {
        TIM_TRY(tim_ensure(ctx, mlp->y, (size_t)N * sizeof(float)));
        TIM_TRY(tim_ensure(ctx, mlp->part, nb * mlp->L.P * sizeof(float)));
        TIM_TRY(tim_ensure(ctx, mlp->ploss, nb * sizeof(float)));
        CUDA_TRY(ctx, cudaMemcpyAsync(mlp->y.p, y, (size_t)N * sizeof(float),
                                      cudaMemcpyHostToDevice, ctx->stream));
    }
    return TIM_OK;
}

static FbArgs fb_args(tim_mlp* mlp, uint64_t N) {
    FbArgs a;
    a.wq = (const float*)mlp->wq.p;
    a.in_mu = (const float*)mlp->scal.p;
    a.in_isd = (const float*)mlp->scal.p + DMAX;
    a.out_mu = mlp->out_mu;
    a.out_sd = mlp->out_sd;
    a.inv_out_sd = 1.0f / mlp->out_sd;
    a.x = (const float*)mlp->x.p;
    a.y = (const float*)mlp->y.p;
    a.N = (uint32_t)N;
    a.inv_n = (float)(1.0 / (double)N);
    a.out = (float*)mlp->out.p;
    a.part = (float*)mlp->part.p;
    a.part_loss = (float*)mlp->ploss.p;
    return a;
}

static int check_samples(tim_mlp* mlp, const float* x, uint64_t N) {
    if (!x || N == 0 || N > (1u << 24))
        return tim_fail(mlp->ctx, TIM_ERR_ARG, "need 1 <= N <= 2^24 samples and an input array");
    return TIM_OK;
}

// Forward and backward over the uploaded batch, partials reduced into grad (no Adam)
// or into one Adam step at mlp->step.
static int mlp_step(tim_mlp* mlp, uint64_t N, bool adam, float lr, float* d_loss_out) {
    tim_ctx* ctx = mlp->ctx;
    const unsigned nb = (unsigned)((N + SB - 1) / SB);
    mlp_fb_kernel<true><<<nb, FB_THREADS, SM_BYTES, ctx->stream>>>(fb_args(mlp, N), mlp->d);
    LAUNCH_CHECK(ctx, "mlp_fb_kernel");
    ReduceArgs r;
    r.part = (const float*)mlp->part.p;
    r.part_loss = (const float*)mlp->ploss.p;
    r.nb = (int)nb;
    r.grad = (float*)mlp->out.p;  // unused with Adam
    r.loss_out = d_loss_out;
    r.adam = adam ? 1 : 0;
    r.params = (float*)mlp->params.p;
    r.wq = (float*)mlp->wq.p;
    r.m = (float*)mlp->m.p;
    r.v = (float*)mlp->v.p;
    r.lr = lr;
    r.c1 = r.c2 = 1.f;
    if (adam) {
        mlp->step++;
        r.c1 = (float)(1.0 / (1.0 - pow(0.9, (double)mlp->step)));
        r.c2 = (float)(1.0 / (1.0 - pow(0.999, (double)mlp->step)));
    } else {
        TIM_TRY(tim_ensure(ctx, mlp->gbuf, (size_t)mlp->L.P * sizeof(float)));
        r.grad = (float*)mlp->gbuf.p;
    }
    mlp_reduce_kernel<<<(mlp->L.P + 255) / 256, 256, 0, ctx->stream>>>(r, mlp->d);
    LAUNCH_CHECK(ctx, "mlp_reduce_kernel");
    return TIM_OK;
}

extern "C" {

int tim_graph_features(tim_ctx* ctx, float* host_out) {
    if (!ctx || !host_out) return TIM_ERR_ARG;
    if (!ctx->have_graph) return tim_fail(ctx, TIM_ERR_STATE, "no graph loaded");
    if (!ctx->have_feat) {
        DeviceGuard g(ctx->device);
        const uint64_t n = (uint64_t)ctx->n, m = (uint64_t)ctx->m;
        const int nb = ctx->num_sms * 4;
        TIM_TRY(tim_ensure(ctx, ctx->scratch_a, (size_t)(n + 1) * sizeof(uint32_t)));
        TIM_TRY(tim_ensure(ctx, ctx->scratch_b,
                           (size_t)nb * 4 * (sizeof(double) + sizeof(float)) + 64));
        uint32_t* outdeg = (uint32_t*)ctx->scratch_a.p;
        double* psum = (double*)ctx->scratch_b.p;
        float* pmax = (float*)(psum + (size_t)nb * 4);
        float* dout = pmax + (size_t)nb * 4;
        CUDA_TRY(ctx, cudaMemsetAsync(outdeg, 0, (size_t)(n + 1) * sizeof(uint32_t), ctx->stream));
        if (m > 0) {
            feat_outdeg_kernel<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(
                (const uint32_t*)ctx->src.p, m, outdeg);
            LAUNCH_CHECK(ctx, "feat_outdeg_kernel");
        }
        feat_node_kernel<<<nb, FEAT_THREADS, 0, ctx->stream>>>(
            (const uint64_t*)ctx->rowptr.p, (const uint32_t*)ctx->src.p,
            (const uint32_t*)ctx->thr.p, ctx->model, n, outdeg, psum, pmax);
        LAUNCH_CHECK(ctx, "feat_node_kernel");
        feat_final_kernel<<<1, 32, 0, ctx->stream>>>(psum, pmax, nb, n, dout);
        LAUNCH_CHECK(ctx, "feat_final_kernel");
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->feat, dout, sizeof ctx->feat, cudaMemcpyDeviceToHost,
                                      ctx->stream));
        TIM_TRY(tim_sync(ctx));
        ctx->have_feat = true;
    }
    memcpy(host_out, ctx->feat, sizeof ctx->feat);
    return TIM_OK;
}

int tim_mlp_create(tim_mlp** out, tim_ctx* ctx, int d_in) {
    if (!out || !ctx) return TIM_ERR_ARG;
    *out = nullptr;
    if (d_in < 1 || d_in > DMAX) return tim_fail(ctx, TIM_ERR_ARG, "d_in must be in [1, 32]");
    DeviceGuard g(ctx->device);
    CUDA_TRY(ctx, cudaFuncSetAttribute(mlp_fb_kernel<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_BYTES));
    CUDA_TRY(ctx, cudaFuncSetAttribute(mlp_fb_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_BYTES));
    tim_mlp* mlp = new tim_mlp;
    mlp->ctx = ctx;
    mlp->d = d_in;
    mlp->L = layout_of(d_in);
    const size_t pb = (size_t)mlp->L.P * sizeof(float);
    int rc = TIM_OK;
    for (DevBuf* b : {&mlp->params, &mlp->wq, &mlp->m, &mlp->v})
        if (rc == TIM_OK && (rc = tim_ensure(ctx, *b, pb)) == TIM_OK)
            rc = tim_cuda_check(ctx, cudaMemsetAsync(b->p, 0, pb, ctx->stream), "memset");
    if (rc == TIM_OK) rc = tim_ensure(ctx, mlp->scal, 2 * DMAX * sizeof(float));
    if (rc == TIM_OK) {
        std::vector<float> s(2 * DMAX, 0.f);
        for (int i = 0; i < DMAX; i++) s[DMAX + i] = 1.f;
        rc = tim_cuda_check(ctx, cudaMemcpyAsync(mlp->scal.p, s.data(), s.size() * sizeof(float),
                                                 cudaMemcpyHostToDevice, ctx->stream),
                            "copy scaling");
        if (rc == TIM_OK) rc = tim_sync(ctx);
    }
    if (rc != TIM_OK) {
        tim_mlp_destroy(mlp);
        return rc;
    }
    *out = mlp;
    return TIM_OK;
}

int tim_mlp_destroy(tim_mlp* mlp) {
    if (!mlp) return TIM_OK;
    DeviceGuard g(mlp->ctx->device);
    for (DevBuf* b : {&mlp->params, &mlp->wq, &mlp->m, &mlp->v, &mlp->scal, &mlp->x, &mlp->y,
                      &mlp->out, &mlp->part, &mlp->ploss, &mlp->gbuf})
        tim_free(*b);
    delete mlp;
    return TIM_OK;
}

uint64_t tim_mlp_param_count(const tim_mlp* mlp) { return mlp ? (uint64_t)mlp->L.P : 0; }

int tim_mlp_set_params(tim_mlp* mlp, const float* params, uint64_t count) {
    if (!mlp || !params) return TIM_ERR_ARG;
    tim_ctx* ctx = mlp->ctx;
    if (count != (uint64_t)mlp->L.P) return tim_fail(ctx, TIM_ERR_ARG, "wrong parameter count");
    DeviceGuard g(ctx->device);
    const size_t pb = (size_t)mlp->L.P * sizeof(float);
    CUDA_TRY(ctx, cudaMemcpyAsync(mlp->params.p, params, pb, cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(mlp->m.p, 0, pb, ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync(mlp->v.p, 0, pb, ctx->stream));
    mlp_round_kernel<<<(mlp->L.P + 255) / 256, 256, 0, ctx->stream>>>(
        (const float*)mlp->params.p, (float*)mlp->wq.p, mlp->d);
    LAUNCH_CHECK(ctx, "mlp_round_kernel");
    mlp->step = 0;
    return tim_sync(ctx);
}

int tim_mlp_get_params(tim_mlp* mlp, float* params, uint64_t count) {
    if (!mlp || !params) return TIM_ERR_ARG;
    tim_ctx* ctx = mlp->ctx;
    if (count != (uint64_t)mlp->L.P) return tim_fail(ctx, TIM_ERR_ARG, "wrong parameter count");
    DeviceGuard g(ctx->device);
    CUDA_TRY(ctx, cudaMemcpyAsync(params, mlp->params.p, (size_t)count * sizeof(float),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    return tim_sync(ctx);
}

int tim_mlp_set_scaling(tim_mlp* mlp, const float* in_mu, const float* in_isd, float out_mu,
                        float out_sd) {
    if (!mlp || !in_mu || !in_isd) return TIM_ERR_ARG;
    tim_ctx* ctx = mlp->ctx;
    if (!(out_sd != 0.f) || !isfinite(out_sd) || !isfinite(out_mu))
        return tim_fail(ctx, TIM_ERR_ARG, "out_sd must be finite and non-zero");
    DeviceGuard g(ctx->device);
    std::vector<float> s(2 * DMAX, 0.f);
    for (int i = 0; i < DMAX; i++) s[DMAX + i] = 1.f;
    for (int i = 0; i < mlp->d; i++) {
        s[i] = in_mu[i];
        s[DMAX + i] = in_isd[i];
    }
    CUDA_TRY(ctx, cudaMemcpyAsync(mlp->scal.p, s.data(), s.size() * sizeof(float),
                                  cudaMemcpyHostToDevice, ctx->stream));
    mlp->out_mu = out_mu;
    mlp->out_sd = out_sd;
    return tim_sync(ctx);
}

int tim_mlp_grad(tim_mlp* mlp, const float* x, const float* y, uint64_t n_samples, float* loss,
                 float* grad) {
    if (!mlp || !y) return TIM_ERR_ARG;
    TIM_TRY(check_samples(mlp, x, n_samples));
    tim_ctx* ctx = mlp->ctx;
    DeviceGuard g(ctx->device);
    TIM_TRY(mlp_upload(mlp, x, y, n_samples));
    float* d_loss = (float*)mlp->out.p + n_samples;
    TIM_TRY(mlp_step(mlp, n_samples, false, 0.f, d_loss));
    if (grad)
        CUDA_TRY(ctx, cudaMemcpyAsync(grad, mlp->gbuf.p, (size_t)mlp->L.P * sizeof(float),
                                      cudaMemcpyDeviceToHost, ctx->stream));
    float l = 0.f;
    CUDA_TRY(ctx, cudaMemcpyAsync(&l, d_loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    TIM_TRY(tim_sync(ctx));
    if (loss) *loss = l;
    return TIM_OK;
}

int tim_mlp_train(tim_mlp* mlp, const float* x, const float* y, uint64_t n_samples, int steps,
                  float lr, float* loss_history) {
    if (!mlp || !y) return TIM_ERR_ARG;
    TIM_TRY(check_samples(mlp, x, n_samples));
    tim_ctx* ctx = mlp->ctx;
    if (steps < 0 || !(lr > 0.f) || !isfinite(lr))
        return tim_fail(ctx, TIM_ERR_ARG, "need steps >= 0 and lr > 0");
    DeviceGuard g(ctx->device);
    TIM_TRY(mlp_upload(mlp, x, y, n_samples));
    TIM_TRY(tim_ensure(ctx, mlp->gbuf, ((size_t)steps + 1) * sizeof(float)));
    float* hist = (float*)mlp->gbuf.p;
    for (int s = 0; s < steps; s++) TIM_TRY(mlp_step(mlp, n_samples, true, lr, hist + s));
    if (loss_history && steps > 0)
        CUDA_TRY(ctx, cudaMemcpyAsync(loss_history, hist, (size_t)steps * sizeof(float),
                                      cudaMemcpyDeviceToHost, ctx->stream));
    return tim_sync(ctx);
}

int tim_mlp_predict(tim_mlp* mlp, const float* x, uint64_t n_samples, float* out) {
    if (!mlp || !out) return TIM_ERR_ARG;
    TIM_TRY(check_samples(mlp, x, n_samples));
    tim_ctx* ctx = mlp->ctx;
    DeviceGuard g(ctx->device);
    TIM_TRY(mlp_upload(mlp, x, nullptr, n_samples));
    const unsigned nb = (unsigned)((n_samples + SB - 1) / SB);
    mlp_fb_kernel<false><<<nb, FB_THREADS, SM_BYTES, ctx->stream>>>(fb_args(mlp, n_samples),
                                                                     mlp->d);
    LAUNCH_CHECK(ctx, "mlp_fb_kernel");
    CUDA_TRY(ctx, cudaMemcpyAsync(out, mlp->out.p, (size_t)n_samples * sizeof(float),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    return tim_sync(ctx);
}

}  // extern "C"

// Start rounds i0 of Algorithm 2 for the graphs of ctxs[] with the given k, in one
// network launch on the first context's stream (features come from each context's
// cache, computed on first use).
int tim_learned_start_rounds(tim_mlp* mlp, tim_ctx* const* ctxs, const int* ks, int nq,
                             int* i0) {
    if (!mlp || mlp->d != TIM_START_FEATURES)
        return tim_fail(ctxs[0], TIM_ERR_ARG, "the start-round network takes 12 features");
    std::vector<float> x((size_t)nq * TIM_START_FEATURES), y(nq);
    for (int q = 0; q < nq; q++) {
        tim_ctx* c = ctxs[q];
        float* row = x.data() + (size_t)q * TIM_START_FEATURES;
        TIM_TRY(tim_graph_features(c, row));
        row[8] = (float)log((double)c->n);
        row[9] = (float)log((double)std::max<int64_t>(c->m, 1));
        row[10] = (float)log((double)ks[q]);
        row[11] = (float)c->model;
    }
    TIM_TRY(tim_mlp_predict(mlp, x.data(), (uint64_t)nq, y.data()));
    for (int q = 0; q < nq; q++) {
        tim_ctx* c = ctxs[q];
        const int rounds = tim_host_rounds(c->n);
        const double t =
            (double)y[q] + log2((double)std::max<int64_t>(c->m, 1) / (double)ks[q]);
        int r = isfinite(t) ? (int)std::min(std::max(floor(t) + 1.0, 1.0), 64.0) : 1;
        i0[q] = std::max(1, std::min(r, std::max(rounds, 1)));
    }
    return TIM_OK;
}
