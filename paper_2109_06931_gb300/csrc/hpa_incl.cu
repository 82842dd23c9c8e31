// Inclusive metrics (Section 6.1, statistic generation: measured values are
// propagated up the calling context tree).
//  (a) structure tree inside each launch context: every key is expanded to
//      its node and all ancestors up to the function node, then aggregated
//      exactly by the shared plan / leaf / emit kernels (hpa_agg.cu);
//  (b) host calling-context tree: per-context exclusive totals, then one
//      bottom-up pass in which the last child to finish carries the sum to
//      its parent (no level loop, no waiting).

#include <algorithm>

#include "hpa_host.h"

namespace hpa {

__global__ void k_cct_exclusive(const uint32_t* kctx, const uint8_t* kstall, const uint64_t* kval,
                                const uint64_t* n_keys, uint64_t cap, uint32_t n_cct, uint32_t S,
                                unsigned long long* out, DevStatus* st) {
    const uint64_t K = min(*n_keys, cap);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = kctx[i], r = kstall[i];
        if (c >= n_cct || r >= S) { raise_status(st, 1 /* HPA_E_INVALID_ARG */, 1); continue; }
        atomicAdd(&out[(size_t)c * S + r], (unsigned long long)kval[i]);
    }
}

__global__ void k_cct_children(const uint32_t* parent, uint32_t n, uint32_t* nchild, uint32_t* pend, DevStatus* st) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint32_t p = parent[v];
        if (p == NO_PARENT) continue;
        if (p >= n || p == v) { raise_status(st, 2 /* HPA_E_INVALID_TABLE */, 2); continue; }
        atomicAdd(&nchild[p], 1u);
        atomicAdd(&pend[p], 1u);
    }
}

// A leaf starts a walk; at each parent the child's inclusive row is added
// (64-bit atomics in L2), then the parent's pending-children counter drops.
// The thread that brings it to zero is the last child: every other child's
// additions are visible to it (fence before the decrement, fence after), so
// it continues upward with the parent's now final row.
__global__ void k_cct_peel(const uint32_t* parent, uint32_t n, const uint32_t* nchild, uint32_t* pend,
                           uint32_t S, unsigned long long* out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (nchild[v] != 0) continue;
        uint32_t x = v;
        for (uint32_t steps = 0; steps < n; ++steps) {
            const uint32_t p = parent[x];
            if (p == NO_PARENT || p >= n || p == x) break;
            for (uint32_t r = 0; r < S; ++r) {
                const unsigned long long a = __ldcg(&out[(size_t)x * S + r]);
                if (a) atomicAdd(&out[(size_t)p * S + r], a);
            }
            __threadfence();
            if (atomicSub(&pend[p], 1u) != 1u) break;
            __threadfence();
            x = p;
        }
    }
}

// nodes whose children never all finished lie on or above a cycle
__global__ void k_cct_check(const uint32_t* pend, uint32_t n, DevStatus* st) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (pend[v] != 0) raise_status(st, 2 /* HPA_E_INVALID_TABLE */, 3);
}

}  // namespace hpa

using namespace hpa;

hpa_status hpa_handle::stage_single_output(AggWork& w, uint32_t bin, uint32_t n_ctx, const hpa_profile& o) {
    hpa_status st = ensure_staging(sizeof(BufDev) + 64 + 1024);
    if (st) return st;
    Carve hs{(char*)staging};
    BufDev* hb = hs.take<BufDev>(1);
    uint64_t* htile = hs.take<uint64_t>(2);
    uint32_t* hgrp = hs.take<uint32_t>(2);
    BufDev d{};
    d.n_ctx = n_ctx; d.n_stall = o.n_stall; d.grp_base = 0; d.bin = bin;
    d.key_ctx = o.key_ctx; d.key_node = o.key_node; d.key_stall = o.key_stall; d.val = o.val;
    d.n_keys = o.n_keys; d.capacity = o.capacity;
    *hb = d;
    htile[0] = htile[1] = 0;
    hgrp[0] = 0; hgrp[1] = n_ctx;
    if ((st = upload_staging(hs.off))) return st;
    char* ds = (char*)d_staging;
    w.bufs = (const BufDev*)(ds + ((char*)hb - (char*)staging));
    w.buf_tile = (const uint64_t*)(ds + ((char*)htile - (char*)staging));
    w.buf_grp = (const uint32_t*)(ds + ((char*)hgrp - (char*)staging));
    w.n_tiles = 0;
    return HPA_OK;
}

extern "C" hpa_status hpa_propagate_inclusive(hpa_handle* h, uint32_t binary_id, const hpa_profile* p,
                                              hpa_profile* tree_out, const hpa_cct* cct, uint64_t* cct_out) {
    hpa::Trace trace_("hpa.propagate_inclusive");
    if (!h || !p) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = h->binary(binary_id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", binary_id);
    if (!p->n_keys || (p->capacity && (!p->key_ctx || !p->key_node || !p->key_stall || !p->val)))
        return h->fail(HPA_E_INVALID_ARG, "input profile arrays missing");
    if (p->n_stall == 0 || p->n_stall > HPA_MAX_STALL || p->n_ctx == 0)
        return h->fail(HPA_E_INVALID_ARG, "input profile has no n_ctx / n_stall (produce it with hpa_attribute_samples)");
    hpa_status st;
    if (tree_out) {
        if (!tree_out->n_keys || (tree_out->capacity && (!tree_out->key_ctx || !tree_out->key_node ||
                                                          !tree_out->key_stall || !tree_out->val)))
            return h->fail(HPA_E_INVALID_ARG, "tree_out arrays missing");
        const uint64_t N = p->capacity * (uint64_t)(B->max_depth + 1);
        if (N >= 0xFFFFFFF0ull) return h->fail(HPA_E_INVALID_ARG, "expanded record bound %llu too large; pass the key count as capacity",
                                               (unsigned long long)N);
        const uint32_t sb = ceil_log2_u64(p->n_stall);
        const uint32_t nb = ceil_log2_u64((uint64_t)B->n_nodes + 1);
        if (nb + sb > 32) return h->fail(HPA_E_INVALID_ARG, "(n_nodes + 1) * 2^stall_bits exceeds 2^32");
        AggWork w{};
        if ((st = h->carve_work(w, N, p->n_ctx, 1, LEAF_CAP_SMALL, sb, nb + sb, true, true))) return st;
        tree_out->n_ctx = p->n_ctx;
        tree_out->n_stall = p->n_stall;
        tree_out->n_nodes = B->n_nodes;
        if ((st = h->stage_single_output(w, binary_id, p->n_ctx, *tree_out))) return st;
        ExpandSrc x{p->key_ctx, p->key_node, p->key_stall, p->val, p->n_keys, p->capacity,
                    B->d_node_parent, B->d_node_depth, B->n_nodes, p->n_ctx};
        run_expand_aggregate(w, x, h->stream, h->sms, &h->launches);
        if ((st = h->cuda(cudaGetLastError(), "structure inclusive launch"))) return st;
    }
    if (cct) {
        if (!cct->parent || !cct_out || cct->n_nodes == 0) return h->fail(HPA_E_INVALID_ARG, "cct arrays missing");
        if (cct->n_nodes < p->n_ctx) return h->fail(HPA_E_INVALID_ARG, "cct has fewer nodes than the profile has contexts");
        const uint32_t n = cct->n_nodes, S = p->n_stall;
        Carve probe{nullptr};
        probe.take<uint32_t>(n);
        probe.take<uint32_t>(n);
        // the CCT counters use their own small allocation so that they never
        // alias the aggregation scratch of a tree_out call queued before
        if ((size_t)n * 8 + 512 > h->cct_cap) {
            if ((st = h->cuda(cudaStreamSynchronize(h->stream), "sync"))) return st;
            if (h->cct_scratch) cudaFree(h->cct_scratch);
            h->cct_scratch = nullptr;
            h->cct_cap = 0;
            if (cudaMalloc(&h->cct_scratch, (size_t)n * 8 + 512) != cudaSuccess) {
                cudaGetLastError();
                return h->fail(HPA_E_OOM, "cct counters");
            }
            h->cct_cap = (size_t)n * 8 + 512;
        }
        Carve c{(char*)h->cct_scratch};
        uint32_t* nchild = c.take<uint32_t>(n);
        uint32_t* pend = c.take<uint32_t>(n);
        cudaStream_t s = h->stream;
        cudaMemsetAsync(h->cct_scratch, 0, c.off, s);
        cudaMemsetAsync(cct_out, 0, (size_t)n * S * 8, s);
        const int kb = (int)std::max<uint64_t>(1, std::min<uint64_t>((p->capacity + 255) / 256, (uint64_t)h->sms * 8));
        const int nbk = (int)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)h->sms * 8));
        k_cct_exclusive<<<kb, 256, 0, s>>>(p->key_ctx, p->key_stall, p->val, p->n_keys, p->capacity, n, S,
                                           (unsigned long long*)cct_out, h->d_status);
        k_cct_children<<<nbk, 256, 0, s>>>(cct->parent, n, nchild, pend, h->d_status);
        k_cct_peel<<<nbk, 256, 0, s>>>(cct->parent, n, nchild, pend, S, (unsigned long long*)cct_out);
        k_cct_check<<<nbk, 256, 0, s>>>(pend, n, h->d_status);
        h->launches += 4;
        if ((st = h->cuda(cudaGetLastError(), "cct inclusive launch"))) return st;
    }
    return HPA_OK;
}
