// Warp issue rate and stall shares per (launch context, function) (Section
// 7: W = (S - S_stall) / S, read per kernel and per function).
//
// The profile's keys are regrouped by (context, function of the node,
// stall) through the aggregation's own grouping, leaves and key placement
// (64-bit values), which gives exact sums in (context, function, stall)
// order; a head flag per (context, function) run, a scan of the flags and
// one thread per run then give each row's S, S_issued, W and stall shares.
// UNKNOWN keys belong to no function and are left out.

#include <algorithm>

#include "hpa_host.h"

namespace hpa {

struct FuncSrc {
    const uint32_t* ctx;
    const uint32_t* node;
    const uint8_t* stall;
    const uint64_t* val;
    const uint64_t* n_keys;
    uint64_t cap;
    const uint32_t* node_func;
    uint32_t M, n_ctx, S;
};

__global__ void k_fn_hist(AggWork w, FuncSrc x) {
    const uint64_t K = min(*x.n_keys, x.cap);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = x.ctx[i], n = x.node[i];
        if (n == UNKNOWN) continue;
        if (c >= x.n_ctx || n >= x.M || x.stall[i] >= x.S) { atomicAdd(&w.buf_bad[0], 1ull); continue; }
        atomicAdd(&w.grp_hist[c], 1u);
    }
}

__global__ void k_fn_scatter(AggWork w, FuncSrc x) {
    const uint64_t K = min(*x.n_keys, x.cap);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = x.ctx[i], n = x.node[i], r = x.stall[i];
        if (n == UNKNOWN || c >= x.n_ctx || n >= x.M || r >= x.S) continue;
        const uint32_t slot = atomicAdd(&w.grp_cursor[(size_t)c << w.cur_shift], 1u);
        w.rec_sub[slot] = (x.node_func[n] << w.sb) | r;
        w.rec_v64[slot] = x.val[i];
    }
}

// head of a (context, function) run in the regrouped keys
__global__ void k_issue_heads(const uint32_t* kc, const uint32_t* kf, const uint64_t* n_keys, uint64_t cap,
                              uint32_t* head) {
    const uint64_t K = min(*n_keys, cap);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x)
        head[i] = i < K && (i == 0 || kc[i] != kc[i - 1] || kf[i] != kf[i - 1]) ? 1u : 0u;
}

__global__ void k_issue_rows(const uint32_t* kc, const uint32_t* kf, const uint8_t* ks, const uint64_t* kv,
                             const uint64_t* n_keys, uint64_t cap, const uint32_t* row, uint32_t S,
                             uint32_t issued_mask, hpa_issue_rows o, DevStatus* st) {
    const uint64_t K = min(*n_keys, cap);
    const uint64_t n_rows = row[cap];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *o.n_rows = n_rows;
        if (n_rows > o.capacity) raise_status(st, 4 /* HPA_E_CAPACITY */, 0);
    }
    if (n_rows > o.capacity) return;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
        if (!(i == 0 || kc[i] != kc[i - 1] || kf[i] != kf[i - 1])) continue;
        const uint64_t r = row[i];
        uint64_t tot = 0, iss = 0;
        uint64_t j = i;
        for (; j < K && kc[j] == kc[i] && kf[j] == kf[i]; ++j) {
            tot += kv[j];
            if ((issued_mask >> ks[j]) & 1u) iss += kv[j];
        }
        o.ctx[r] = kc[i];
        o.func[r] = kf[i];
        o.S[r] = tot;
        o.S_issued[r] = iss;
        o.W[r] = (float)((double)iss / (double)tot);
        if (o.frac) {
            for (uint32_t q = 0; q < S; ++q) o.frac[r * S + q] = 0.0f;
            for (uint64_t m = i; m < j; ++m) o.frac[r * S + ks[m]] = (float)((double)kv[m] / (double)tot);
        }
    }
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_issue_by_function(hpa_handle* h, uint32_t binary_id, const hpa_profile* p,
                                            hpa_issue_rows* out) {
    hpa::Trace trace_("hpa.issue_by_function");
    if (!h || !p || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = h->binary(binary_id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", binary_id);
    if (!p->n_keys || (p->capacity && (!p->key_ctx || !p->key_node || !p->key_stall || !p->val)))
        return h->fail(HPA_E_INVALID_ARG, "profile arrays missing");
    if (p->n_stall == 0 || p->n_stall > HPA_MAX_STALL || p->n_ctx == 0)
        return h->fail(HPA_E_INVALID_ARG, "profile has no n_ctx / n_stall (produce it with hpa_attribute_samples)");
    if (!out->n_rows || (out->capacity && (!out->ctx || !out->func || !out->S || !out->S_issued || !out->W)))
        return h->fail(HPA_E_INVALID_ARG, "output arrays missing");
    const uint64_t K = p->capacity;
    if (K >= 0xFFFFFFF0ull) return h->fail(HPA_E_INVALID_ARG, "too many keys in one call");
    if (K == 0) return h->cuda(cudaMemsetAsync(out->n_rows, 0, sizeof(uint64_t), h->stream), "issue rate");
    const uint32_t sb = ceil_log2_u64(p->n_stall);
    const uint32_t fb = ceil_log2_u64((uint64_t)B->n_funcs + 1);
    if (fb + sb > 32) return h->fail(HPA_E_INVALID_ARG, "(n_funcs + 1) * 2^stall_bits exceeds 2^32");
    // the regrouped keys (ctx, function, stall, sum) and the run flags
    Carve probe{nullptr};
    probe.take<uint32_t>(K + 1);
    probe.take<uint32_t>(K + 1);
    probe.take<uint8_t>(K + 1);
    probe.take<uint64_t>(K + 1);
    probe.take<uint64_t>(2);
    probe.take<uint32_t>(K + 1);
    probe.take<uint32_t>(scan_tmp_words(K + 1));
    if (probe.off + 256 > h->aux_cap) {
        hpa_status st = h->cuda(cudaStreamSynchronize(h->stream), "sync");
        if (st) return st;
        if (h->aux_scratch) cudaFree(h->aux_scratch);
        h->aux_scratch = nullptr;
        h->aux_cap = 0;
        if (cudaMalloc(&h->aux_scratch, probe.off + 256) != cudaSuccess) {
            cudaGetLastError();
            return h->fail(HPA_E_OOM, "issue-rate keys of %zu bytes", probe.off + 256);
        }
        h->aux_cap = probe.off + 256;
    }
    Carve c{(char*)h->aux_scratch};
    hpa_profile g{};
    g.capacity = K;
    g.key_ctx = c.take<uint32_t>(K + 1);
    g.key_node = c.take<uint32_t>(K + 1);
    g.key_stall = c.take<uint8_t>(K + 1);
    g.val = c.take<uint64_t>(K + 1);
    g.n_keys = c.take<uint64_t>(2);
    g.n_stall = p->n_stall;
    uint32_t* head = c.take<uint32_t>(K + 1);
    uint32_t* stmp = c.take<uint32_t>(scan_tmp_words(K + 1));
    AggWork w{};
    hpa_status st = h->carve_work(w, K, p->n_ctx, 1, LEAF_CAP_SMALL, sb, fb + sb, true, true);
    if (st) return st;
    if ((st = h->stage_single_output(w, binary_id, p->n_ctx, g))) return st;
    w.emit_totals = 0;
    FuncSrc x{p->key_ctx, p->key_node, p->key_stall, p->val, p->n_keys, K, B->cg.node_func, B->n_nodes, p->n_ctx,
              p->n_stall};
    cudaStream_t s = h->stream;
    clear_work(w, s);
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((K + 255) / 256, (uint64_t)h->sms * 8));
    k_fn_hist<<<blocks, 256, 0, s>>>(w, x);
    run_plan(w, s, h->sms, &h->launches, false);
    k_fn_scatter<<<blocks, 256, 0, s>>>(w, x);
    h->launches += 2;
    run_group_tail(w, s, h->sms, &h->launches);
    k_issue_heads<<<blocks, 256, 0, s>>>(g.key_ctx, g.key_node, g.n_keys, K, head);
    scan_u32(head, head, K, stmp, s, &h->launches);
    k_issue_rows<<<blocks, 256, 0, s>>>(g.key_ctx, g.key_node, g.key_stall, g.val, g.n_keys, K, head, p->n_stall,
                                        h->opt.issued_mask ? h->opt.issued_mask : 1u, *out, h->d_status);
    h->launches += 2;
    return h->cuda(cudaGetLastError(), "issue rate launch");
}
