// graph.cu -- G^T (Table 1 of the paper) on the device: the in-CSR of G with the
// in-edges of every node ascending by source, and the per-edge thresholds of the
// diffusion model.
//
// Build: one pass writes (destination, source, weight bits) for every out-edge, in
// out-CSR order (ascending source); a stable radix sort by destination of these triples
// turns them into the in-lists, each ascending by source, with no gather afterwards;
// the in-CSR offsets are the boundaries between destinations in the sorted keys.
//   IC (Section 2.1): thr = floor(p * 2^32) for p < 1, 0xFFFFFFFF (always live) for
//                     p >= 1; an in-edge is live iff its coin word < thr.
//   LT (Section 6):   thr = inclusive prefix over the in-list of floor(b * 2^32),
//                     saturated at 2^32 - 1; the triggering in-edge of a node is the
//                     first whose prefix exceeds the node's draw.
#include "common.cuh"

namespace {

__global__ void check_rowptr_kernel(const int64_t* __restrict__ rowptr, int64_t n, int64_t m,
                                    int* __restrict__ err) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = rowptr[u], b = rowptr[u + 1];
        if (b < a || a < 0 || b > m || (u == 0 && a != 0) || (u == n - 1 && b != m))
            atomicOr(err, TIM_DEV_ERR_GRAPH);
    }
}

// Sort input per out-CSR edge e: key = destination and b = the weight's bits are read by
// the sort's first pass straight from the caller's arrays; this kernel checks the
// destinations and writes a = the source (one warp per source node u over its
// out-edges; the offsets are checked by check_rowptr_kernel only at the end of the load,
// so they are clamped to [0, m) here: an invalid graph is rejected and its sources are
// never used), and for the triggering model, which has no per-edge weight, b = the edge
// id e.
__global__ void edges_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ dst,
                             const float* __restrict__ w, int64_t n, int64_t m,  // w null: ids
                             uint32_t* __restrict__ srcs, uint32_t* __restrict__ wbits,
                             int* __restrict__ err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = dst[e];
        if (v < 0 || v >= n) atomicOr(err, TIM_DEV_ERR_GRAPH);
        if (!w) wbits[e] = (uint32_t)e;
    }
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const int64_t b = min(max(rowptr[u], (int64_t)0), m);
        const int64_t f = min(max(rowptr[u + 1], b), m);
        for (int64_t e = b + lane; e < f; e += 32) srcs[e] = (uint32_t)u;
    }
}

// floor(p 2^32) of an edge weight (bits) as a 64-bit integer; invalid weights (outside
// [0, 1]) count as 0 and set *bad. In single precision: multiplying by 2^32 only moves
// the exponent, so p 2^32 is exact, and conversion toward zero is the floor.
__device__ __forceinline__ unsigned long long weight_scaled(uint32_t wb, bool* bad) {
    float p = __uint_as_float(wb);
    *bad = !(p >= 0.0f && p <= 1.0f);
    if (*bad) p = 0.0f;
    return __float2ull_rz(p * 4294967296.0f);
}

// IC threshold: floor(p 2^32), p >= 1 (2^32) as 2^32 - 1 (always live)
__device__ __forceinline__ uint32_t ic_threshold(uint32_t wb) {
    bool bad;
    const unsigned long long scaled = weight_scaled(wb, &bad);
    return scaled > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)scaled;
}

// Everything the sorted (destination, source, weight) triples give, one pass per in-edge
// (sorted position) that also reads its predecessor: the source (range and self-loop
// checks), the in-CSR offsets at destination boundaries, the duplicate check (sources
// strictly ascending inside an in-list), the model's threshold (weight checks), and for
// IC whether a node's in-edges carry different thresholds.
__global__ void in_edges_kernel(const uint32_t* __restrict__ sorted_dst,
                                const uint32_t* __restrict__ sorted_src,
                                const uint32_t* __restrict__ sorted_wbits, int64_t n, int64_t m,
                                int model, uint64_t* __restrict__ rowptr,
                                uint32_t* __restrict__ src, uint32_t* __restrict__ thr,
                                unsigned long long* __restrict__ lt_t,
                                uint32_t* __restrict__ posof, uint8_t* __restrict__ nonuni,
                                int* __restrict__ err) {
    // keys outside [0, n) come from an invalid graph (already flagged): clamped, so that
    // nothing is written out of bounds
    const uint32_t vmax = (uint32_t)(n - 1);
    for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < m;
         pos += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = min(sorted_dst[pos], vmax);
        uint32_t u = sorted_src[pos];
        const uint32_t wb = sorted_wbits[pos];
        if (u >= (uint64_t)n) {  // offsets that miss this edge (an invalid graph)
            atomicOr(err, TIM_DEV_ERR_GRAPH);
            u = 0;
        }
        if (u == v) atomicOr(err, TIM_DEV_ERR_GRAPH);
        src[pos] = u;
        // the in-CSR offsets: rowptr[w] = pos for every w in (previous key, v]
        const int64_t prev = pos > 0 ? (int64_t)min(sorted_dst[pos - 1], vmax) : -1;
        for (int64_t w = prev + 1; w <= (int64_t)v; w++) rowptr[w] = (uint64_t)pos;
        if (pos == m - 1)
            for (int64_t w = (int64_t)v + 1; w <= n; w++) rowptr[w] = (uint64_t)m;
        const bool same = prev == (int64_t)v;  // the predecessor is in the same in-list
        if (same) {
            uint32_t pu = sorted_src[pos - 1];
            if (pu >= (uint64_t)n) pu = 0;
            if (u <= pu) atomicOr(err, TIM_DEV_ERR_GRAPH);
        }
        if (model == TIM_TRIG) {  // no weight; record where out-edge wb landed
            thr[pos] = 0u;
            posof[wb] = (uint32_t)pos;
            continue;
        }
        bool bad;
        const unsigned long long scaled = weight_scaled(wb, &bad);
        if (bad) atomicOr(err, TIM_DEV_ERR_WEIGHT);
        if (model == TIM_IC) {
            const uint32_t t = scaled > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)scaled;
            thr[pos] = t;
            if (same && ic_threshold(sorted_wbits[pos - 1]) != t) nonuni[v] = 1;
        } else {
            lt_t[pos] = scaled;
        }
    }
}

// LT thresholds from E, the exclusive scan of t over all in-edges: the inclusive
// prefix of t over v's in-list at position j is E[j] + t[j] - E[beg(v)], saturated at
// 2^32 - 1. The weight check compares v's total sum of t with floor((1 + 1e-5) 2^32)
// (sum of floor(b 2^32) <= 2^32 sum b, so a valid in-list always passes). One thread per
// in-edge; also marks nodes whose in-edges do not all carry the same t.
__global__ void lt_thr_kernel(const uint64_t* __restrict__ rowptr, const uint32_t* __restrict__ dst_sorted,
                              int64_t m, const unsigned long long* __restrict__ lt_t,
                              const uint64_t* __restrict__ E, uint32_t* __restrict__ thr,
                              uint8_t* __restrict__ nonuni, int* __restrict__ err) {
    const unsigned long long bound = (unsigned long long)((1.0 + 1e-5) * 4294967296.0);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = dst_sorted[j];
        const uint64_t beg = rowptr[v], end = rowptr[v + 1];
        const unsigned long long c = E[j] + lt_t[j] - E[beg];
        thr[j] = c > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)c;
        if ((uint64_t)j + 1 == end && c > bound) atomicOr(err, TIM_DEV_ERR_WEIGHT);
        if ((uint64_t)j > beg && lt_t[j] != lt_t[j - 1]) nonuni[v] = 1;
    }
}

// Per-node threshold word: IC: low word = the first in-edge's threshold, bit 32 set when
// all in-edges share it (empty in-lists included); LT: bit 32 set, low word = t, when
// all in-edges share t < 2^32 (empty in-lists get 0).
__global__ void node_thr_kernel(const uint64_t* __restrict__ rowptr, int64_t n, int model,
                                const uint32_t* __restrict__ thr,
                                const unsigned long long* __restrict__ lt_t,
                                const uint8_t* __restrict__ nonuni,
                                unsigned long long* __restrict__ node_thr) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = rowptr[v], b = rowptr[v + 1];
        if (model == TIM_IC) {
            const uint32_t t0 = b > a ? thr[a] : 0u;
            node_thr[v] = (unsigned long long)t0 | (nonuni[v] ? 0ull : (1ull << 32));
        } else if (model == TIM_TRIG) {
            node_thr[v] = 0ull;
        } else {
            const unsigned long long t0 = b > a ? lt_t[a] : 0ull;
            const bool same = b > a && !nonuni[v] && t0 <= 0xFFFFFFFFull;
            node_thr[v] = same ? ((1ull << 32) | t0) : 0ull;
        }
    }
}

// IC: nodes under the geometric-skip rule get a gap table Q_0..Q_31 (Q_0 = (2^32 - t)
// 2^32, Q_(b+1) = floor(Q_b^2 / 2^64)) and 1 + its index in bits 33..63 of node_thr.
// With tab == nullptr only counts them.
__global__ void skip_tables_kernel(const uint64_t* __restrict__ rowptr, int64_t n,
                                   unsigned long long* __restrict__ node_thr,
                                   unsigned long long* __restrict__ tab, unsigned long long cap,
                                   unsigned long long* __restrict__ counter) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long nt = node_thr[v];
        if (!tim_skip_rule(nt, rowptr[v + 1] - rowptr[v])) continue;
        const unsigned long long idx = atomicAdd(counter, 1ull);
        if (!tab || idx >= cap) continue;
        unsigned long long q = (0x100000000ull - (unsigned long long)(uint32_t)nt) << 32;
        for (int b = 0; b < 32; b++) {
            tab[idx * 32 + b] = q;
            q = __umul64hi(q, q);
        }
        node_thr[v] = (nt & 0x1FFFFFFFFull) | ((idx + 1ull) << 33);
    }
}

// Triggering model, per node v: the inclusive cumulative threshold of each of its
// options (floor(p * 2^32) summed in option order, saturated at 2^32 - 1), the node of
// each option, and the checks p in [0, 1] and sum p <= 1 + 1e-5.
__global__ void trig_node_kernel(const uint64_t* __restrict__ node_opt, int64_t n,
                                 const float* __restrict__ opt_prob,
                                 uint32_t* __restrict__ opt_cum, uint32_t* __restrict__ opt_node,
                                 int* __restrict__ err) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        double tot = 0.0;
        unsigned long long acc = 0;
        for (uint64_t o = node_opt[v]; o < node_opt[v + 1]; o++) {
            const float p = opt_prob[o];
            if (!(p >= 0.0f && p <= 1.0f)) {
                atomicOr(err, TIM_DEV_ERR_WEIGHT);
                continue;
            }
            tot += (double)p;
            acc += (unsigned long long)((double)p * 4294967296.0);  // floor: p >= 0
            opt_cum[o] = acc > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)acc;
            opt_node[o] = (uint32_t)v;
        }
        if (tot > 1.0 + 1e-5) atomicOr(err, TIM_DEV_ERR_WEIGHT);
    }
}

// Triggering model, per option o: the in-CSR positions of its out-CSR edge ids, each of
// which must end in the option's node, and the option of every entry (the sort key that
// groups the entries again after they are sorted by position).
__global__ void trig_pos_kernel(uint64_t n_opts, const uint64_t* __restrict__ opt_off,
                                const int64_t* __restrict__ opt_edges,
                                const uint32_t* __restrict__ opt_node,
                                const int32_t* __restrict__ out_dst, int64_t m,
                                const uint32_t* __restrict__ posof,
                                uint32_t* __restrict__ opt_pos, uint32_t* __restrict__ opt_of,
                                int* __restrict__ err) {
    for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < n_opts;
         o += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = opt_node[o];
        for (uint64_t i = opt_off[o]; i < opt_off[o + 1]; i++) {
            const int64_t e = opt_edges[i];
            opt_of[i] = (uint32_t)o;
            if (e < 0 || e >= m || (uint32_t)out_dst[e] != v) {
                atomicOr(err, TIM_DEV_ERR_GRAPH);
                opt_pos[i] = 0u;
                continue;
            }
            opt_pos[i] = posof[e];
        }
    }
}

int bit_length(uint64_t x) {
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

}  // namespace

int tim_trig_build(tim_ctx* ctx, const int32_t* d_out_dst, const uint64_t* d_node_opt,
                   const float* d_opt_prob, uint64_t n_opts, const uint64_t* d_opt_off,
                   const int64_t* d_opt_edges, uint64_t n_ent) {
    const int64_t n = ctx->n, m = ctx->m;
    TIM_TRY(tim_zero_scalars(ctx));
    DevScalars* ds = tim_dscal(ctx);
    TIM_TRY(tim_ensure(ctx, ctx->opt_cum, (n_opts + 1) * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->opt_node, (n_opts + 1) * sizeof(uint32_t)));
    const unsigned G = (unsigned)(ctx->num_sms * 8);
    trig_node_kernel<<<G, 256, 0, ctx->stream>>>(d_node_opt, n, d_opt_prob,
                                                 (uint32_t*)ctx->opt_cum.p,
                                                 (uint32_t*)ctx->opt_node.p, &ds->err);
    LAUNCH_CHECK(ctx, "trig_node_kernel");
    if (n_opts) {
        DevBuf of, pad;
        int rc = tim_ensure(ctx, of, (n_ent + 1) * sizeof(uint32_t));
        if (rc == TIM_OK) rc = tim_ensure(ctx, pad, (n_ent + 1) * sizeof(uint32_t));
        if (rc == TIM_OK) {
            trig_pos_kernel<<<G, 256, 0, ctx->stream>>>(
                n_opts, d_opt_off, d_opt_edges, (const uint32_t*)ctx->opt_node.p, d_out_dst, m,
                (const uint32_t*)ctx->ld_posof.p, (uint32_t*)ctx->opt_pos.p, (uint32_t*)of.p,
                &ds->err);
            rc = tim_cuda_check(ctx, cudaGetLastError(), "trig_pos_kernel");
            ctx->launches++;
        }
        // each option's positions ascending (by position, then stably by option): the
        // forward cascades test an in-edge's membership by binary search; the RR walk
        // does not depend on the order
        if (rc == TIM_OK)
            rc = tim_radix_sort_triples(ctx, (uint32_t*)ctx->opt_pos.p, (uint32_t*)of.p,
                                        (uint32_t*)pad.p, n_ent, bit_length((uint64_t)m));
        if (rc == TIM_OK)
            rc = tim_radix_sort_triples(ctx, (uint32_t*)of.p, (uint32_t*)ctx->opt_pos.p,
                                        (uint32_t*)pad.p, n_ent, bit_length(n_opts));
        if (rc == TIM_OK) rc = tim_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sort");
        tim_free(of);
        tim_free(pad);
        TIM_TRY(rc);
    }
    TIM_TRY(tim_read_scalars(ctx));
    if (ctx->h_scal->err & TIM_DEV_ERR_WEIGHT)
        return tim_fail(ctx, TIM_ERR_ARG, "invalid triggering probabilities");
    if (ctx->h_scal->err)
        return tim_fail(ctx, TIM_ERR_ARG, "a triggering option lists an edge that does not end "
                                          "in its node");
    return TIM_OK;
}

int tim_graph_build(tim_ctx* ctx, int64_t n, int64_t m, const int64_t* d_rowptr,
                    const int32_t* d_dst, const float* d_w, int model) {
    if (n < 2 || n > 0x7FFFFFFFll || m < 0 || m > 0xFFFFFFF0ll)
        return tim_fail(ctx, TIM_ERR_ARG, "n must be in [2, 2^31) and m in [0, 2^32 - 16)");
    if (model != TIM_IC && model != TIM_LT && model != TIM_TRIG)
        return tim_fail(ctx, TIM_ERR_ARG, "unknown model");
    ctx->have_graph = false;
    ctx->have_kpt = false;
    ctx->select_open = false;
    ctx->have_feat = false;
    ctx->have_out = false;
    ctx->n_sets = ctx->members = 0;
    TIM_TRY(tim_zero_scalars(ctx));
    DevScalars* ds = tim_dscal(ctx);
    const int T = 256;
    const unsigned G = (unsigned)(ctx->num_sms * 8);

    TIM_TRY(tim_ensure(ctx, ctx->rowptr, (size_t)(n + 1) * sizeof(uint64_t)));
    TIM_TRY(tim_ensure(ctx, ctx->src, (size_t)(m + 4) * sizeof(uint32_t)));
    TIM_TRY(tim_ensure(ctx, ctx->thr, (size_t)(m + 4) * sizeof(uint32_t)));
    // every in-edge is written below; only the padding after the last one (read by
    // 16-byte group loads) needs zeros
    CUDA_TRY(ctx, cudaMemsetAsync((uint32_t*)ctx->src.p + m, 0, 4 * sizeof(uint32_t), ctx->stream));
    CUDA_TRY(ctx, cudaMemsetAsync((uint32_t*)ctx->thr.p + m, 0, 4 * sizeof(uint32_t), ctx->stream));

    // temporaries of the build, kept by the context so that reloading allocates nothing
    DevBuf& keys = ctx->ld_keys;
    DevBuf& srcs = ctx->ld_vals;
    DevBuf& wbits = ctx->ld_srcof;
    DevBuf& lt_t = ctx->ld_lt_t;
    DevBuf& lt_e = ctx->ld_lt_e;
    DevBuf& nonuni = ctx->ld_nonuni;
    int rc = TIM_OK;
    do {
        if ((rc = tim_ensure(ctx, keys, (size_t)(m + 1) * sizeof(uint32_t)))) break;
        if ((rc = tim_ensure(ctx, srcs, (size_t)(m + 1) * sizeof(uint32_t)))) break;
        if ((rc = tim_ensure(ctx, wbits, (size_t)(m + 1) * sizeof(uint32_t)))) break;
        if (model == TIM_LT &&
            (rc = tim_ensure(ctx, lt_t, (size_t)(m + 1) * sizeof(unsigned long long))))
            break;
        check_rowptr_kernel<<<G, T, 0, ctx->stream>>>(d_rowptr, n, m, &ds->err);
        ctx->launches++;
        if (m > 0) {
            edges_kernel<<<G, T, 0, ctx->stream>>>(d_rowptr, d_dst, d_w, n, m, (uint32_t*)srcs.p,
                                                   (uint32_t*)wbits.p, &ds->err);
            ctx->launches++;
            int bits = 0;
            while (bits < 32 && ((int64_t)1 << bits) < n) bits++;
            // destinations and weight bits straight from the caller's arrays (an invalid
            // destination has been flagged and only has to stay in bounds below)
            if ((rc = tim_radix_sort_triples_from(
                     ctx, (const uint32_t*)d_dst, (const uint32_t*)srcs.p,
                     d_w ? (const uint32_t*)d_w : (const uint32_t*)wbits.p, (uint32_t*)keys.p,
                     (uint32_t*)srcs.p, (uint32_t*)wbits.p, (uint64_t)m, bits)))
                break;
            if (model == TIM_TRIG &&
                (rc = tim_ensure(ctx, ctx->ld_posof, (size_t)(m + 1) * sizeof(uint32_t))))
                break;
            if ((rc = tim_ensure(ctx, nonuni, (size_t)(n + 1)))) break;
            if ((rc = tim_cuda_check(ctx, cudaMemsetAsync(nonuni.p, 0, (size_t)(n + 1), ctx->stream),
                                     "memset")))
                break;
            in_edges_kernel<<<G, T, 0, ctx->stream>>>(
                (const uint32_t*)keys.p, (const uint32_t*)srcs.p, (const uint32_t*)wbits.p, n, m,
                model, (uint64_t*)ctx->rowptr.p, (uint32_t*)ctx->src.p, (uint32_t*)ctx->thr.p,
                (unsigned long long*)lt_t.p, (uint32_t*)ctx->ld_posof.p, (uint8_t*)nonuni.p,
                &ds->err);
            ctx->launches++;
        } else if ((rc = tim_cuda_check(ctx, cudaMemsetAsync(ctx->rowptr.p, 0,
                                                             (size_t)(n + 1) * sizeof(uint64_t),
                                                             ctx->stream),
                                        "memset"))) {
            break;
        }
        if (m == 0) {  // no in-edges: every node's list is uniform (empty)
            if ((rc = tim_ensure(ctx, nonuni, (size_t)(n + 1)))) break;
            if ((rc = tim_cuda_check(ctx, cudaMemsetAsync(nonuni.p, 0, (size_t)(n + 1),
                                                          ctx->stream),
                                     "memset")))
                break;
        }
        if (m > 0 && model == TIM_LT) {
            if ((rc = tim_ensure(ctx, lt_e, (size_t)(m + 1) * sizeof(uint64_t)))) break;
            if ((rc = tim_scan_u64(ctx, (const unsigned long long*)lt_t.p, (uint64_t*)lt_e.p,
                                   (uint64_t)m)))
                break;
            lt_thr_kernel<<<G, T, 0, ctx->stream>>>(
                (const uint64_t*)ctx->rowptr.p, (const uint32_t*)keys.p, m,
                (const unsigned long long*)lt_t.p, (const uint64_t*)lt_e.p, (uint32_t*)ctx->thr.p,
                (uint8_t*)nonuni.p, &ds->err);
            ctx->launches++;
        }
        if ((rc = tim_ensure(ctx, ctx->node_thr, (size_t)(n + 1) * 8))) break;
        node_thr_kernel<<<G, T, 0, ctx->stream>>>(
            (const uint64_t*)ctx->rowptr.p, n, model, (const uint32_t*)ctx->thr.p,
            (const unsigned long long*)lt_t.p, (const uint8_t*)nonuni.p,
            (unsigned long long*)ctx->node_thr.p);
        ctx->launches++;
        if (model == TIM_IC) {
            // count the skip-rule nodes, then give each its gap table
            if ((rc = tim_ensure(ctx, lt_e, 2 * sizeof(unsigned long long)))) break;
            auto* ctr = (unsigned long long*)lt_e.p;
            if ((rc = tim_cuda_check(ctx, cudaMemsetAsync(ctr, 0, 16, ctx->stream), "memset")))
                break;
            skip_tables_kernel<<<G, T, 0, ctx->stream>>>((const uint64_t*)ctx->rowptr.p, n,
                                                          (unsigned long long*)ctx->node_thr.p,
                                                          nullptr, 0, ctr);
            ctx->launches++;
            unsigned long long nskip = 0;
            if ((rc = tim_cuda_check(ctx, cudaMemcpyAsync(&nskip, ctr, 8, cudaMemcpyDeviceToHost,
                                                          ctx->stream), "copy")))
                break;
            if ((rc = tim_sync(ctx))) break;
            if ((rc = tim_ensure(ctx, ctx->qtab, (size_t)(nskip + 1) * 32 * 8))) break;
            skip_tables_kernel<<<G, T, 0, ctx->stream>>>(
                (const uint64_t*)ctx->rowptr.p, n, (unsigned long long*)ctx->node_thr.p,
                (unsigned long long*)ctx->qtab.p, nskip, ctr + 1);
            ctx->launches++;
        }
        if ((rc = tim_cuda_check(ctx, cudaGetLastError(), "graph kernels"))) break;
        if ((rc = tim_read_scalars(ctx))) break;
    } while (0);
    if (rc) return rc;
    if (ctx->h_scal->err & TIM_DEV_ERR_BOUNDS)
        return tim_fail(ctx, TIM_ERR_CUDA, "graph build: an index check of the sort failed");
    if (ctx->h_scal->err & TIM_DEV_ERR_WEIGHT)
        return tim_fail(ctx, TIM_ERR_ARG, "invalid edge weights for the model");
    if (ctx->h_scal->err & TIM_DEV_ERR_GRAPH)
        return tim_fail(ctx, TIM_ERR_ARG,
                        "invalid graph (offsets, node range, self-loop or duplicate edge)");
    ctx->n = n;
    ctx->m = m;
    ctx->model = model;
    ctx->have_graph = true;
    return TIM_OK;
}

