// Ratio of two raw metrics per key (Section 4.5: a quantity known once per
// kernel invocation is recovered from two raw metrics summed over threads and
// ranks like any other -- the quantity summed over invocations and the count
// of invocations -- by dividing the two sums).
//
// The keys of both groups of profiles are regrouped by context through the
// aggregation's own plan, leaves and key placement (64-bit values), with the
// group in the lowest subkey bit: (node, stall, group) sorts the two sums of
// a key next to each other.  A head flag per (context, node, stall) run, a
// scan of the flags and one thread per run then give each row's numerator,
// denominator and ratio.

#include <algorithm>
#include <vector>

#include "hpa_host.h"
#include "hpa_warpagg.cuh"

namespace hpa {

struct RatioProf {
    const uint32_t* ctx;
    const uint32_t* node;
    const uint8_t* stall;
    const uint64_t* val;
    const uint64_t* n_keys;
    uint64_t cap;
    uint64_t base;       // first flattened index
};

struct RatioSrc {
    const RatioProf* prof;
    const uint64_t* prof_base;   // [P + 1]
    uint32_t P, P_num;
    uint64_t total;              // sum of capacities
    uint32_t M, n_ctx, S, sb;    // UNKNOWN coded as node M; sb = stall bits
};

// key i of the flattened profiles: false past the profile's keys; *bad for a
// key with an id out of range
__device__ __forceinline__ bool ratio_fetch(const RatioSrc& x, uint64_t i, uint32_t& c, uint32_t& sub, uint64_t& v,
                                            bool& bad) {
    const uint32_t p = upper_index<uint64_t>(x.prof_base, x.P, i);
    const RatioProf& d = x.prof[p];
    const uint64_t j = i - d.base;
    bad = false;
    if (j >= min(*d.n_keys, d.cap)) return false;
    c = d.ctx[j];
    const uint32_t n = d.node[j];
    const uint32_t r = d.stall[j];
    if (c >= x.n_ctx || r >= x.S || (n != UNKNOWN && n >= x.M)) { bad = true; return false; }
    const uint32_t node = n == UNKNOWN ? x.M : n;
    sub = (((node << x.sb) | r) << 1) | (p >= x.P_num ? 1u : 0u);
    v = d.val[j];
    return true;
}

// Both passes walk the flattened keys warp by warp (the loop is uniform in a
// warp); the profiles are sorted by context, so warp-aggregated counting
// mostly takes one atomic per warp.
__global__ void k_ratio_hist(AggWork w, RatioSrc x) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); i0 < x.total; i0 += stride) {
        const uint64_t i = i0 + (threadIdx.x & 31u);
        uint32_t c = 0, sub;
        uint64_t v;
        bool bad = false;
        const bool ok = i < x.total && ratio_fetch(x, i, c, sub, v, bad);
        if (bad) atomicAdd(&w.buf_bad[0], 1ull);
        warp_agg_inc(ok ? &w.grp_hist[c] : nullptr);
    }
}

__global__ void k_ratio_scatter(AggWork w, RatioSrc x) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); i0 < x.total; i0 += stride) {
        const uint64_t i = i0 + (threadIdx.x & 31u);
        uint32_t c = 0, sub = 0;
        uint64_t v = 0;
        bool bad = false;
        const bool ok = i < x.total && ratio_fetch(x, i, c, sub, v, bad);
        const uint32_t slot = warp_agg_inc(ok ? &w.grp_cursor[(size_t)c << w.cur_shift] : nullptr);
        if (!ok) continue;
        w.rec_sub[slot] = sub;
        w.rec_v64[slot] = v;
    }
}

// head of a (context, node, stall) run in the regrouped keys, whose stall
// field holds (stall << 1 | group)
__global__ void k_ratio_heads(const uint32_t* kc, const uint32_t* kn, const uint8_t* ks, const uint64_t* n_keys,
                              uint64_t cap, uint32_t* head) {
    const uint64_t K = min(*n_keys, cap);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x)
        head[i] = i < K && (i == 0 || kc[i] != kc[i - 1] || kn[i] != kn[i - 1] || (ks[i] >> 1) != (ks[i - 1] >> 1))
                      ? 1u : 0u;
}

__global__ void k_ratio_rows(const uint32_t* kc, const uint32_t* kn, const uint8_t* ks, const uint64_t* kv,
                             const uint64_t* n_keys, uint64_t cap, const uint32_t* row, hpa_ratio_rows o,
                             DevStatus* st) {
    const uint64_t K = min(*n_keys, cap);
    const uint64_t n_rows = row[cap];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *o.n_keys = n_rows;
        if (n_rows > o.capacity) raise_status(st, 4 /* HPA_E_CAPACITY */, 0);
    }
    if (n_rows > o.capacity) return;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
        if (!(i == 0 || kc[i] != kc[i - 1] || kn[i] != kn[i - 1] || (ks[i] >> 1) != (ks[i - 1] >> 1))) continue;
        // a run holds at most two keys: the numerator group's sum, then the denominator's
        uint64_t num = 0, den = 0;
        for (uint64_t j = i; j < K && j < i + 2 && kc[j] == kc[i] && kn[j] == kn[i] && (ks[j] >> 1) == (ks[i] >> 1); ++j) {
            if (ks[j] & 1u) den += kv[j];
            else num += kv[j];
        }
        const uint64_t r = row[i];
        o.key_ctx[r] = kc[i];
        o.key_node[r] = kn[i];
        o.key_stall[r] = (uint8_t)(ks[i] >> 1);
        o.num[r] = num;
        o.den[r] = den;
        o.ratio[r] = den ? (float)((double)num / (double)den) : __int_as_float(0x7fc00000);
    }
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_ratio_of_sums(hpa_handle* h, uint32_t binary_id, const hpa_profile* const* num,
                                        uint32_t n_num, const hpa_profile* const* den, uint32_t n_den,
                                        hpa_ratio_rows* out) {
    hpa::Trace trace_("hpa.ratio_of_sums");
    if (!h || !out || (n_num && !num) || (n_den && !den)) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = h->binary(binary_id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", binary_id);
    const uint32_t P = n_num + n_den;
    if (P == 0) return h->fail(HPA_E_INVALID_ARG, "no profiles");
    std::vector<const hpa_profile*> ps(P);
    uint64_t N = 0;
    uint32_t G = 0, S = 0;
    for (uint32_t p = 0; p < P; ++p) {
        const hpa_profile* q = p < n_num ? num[p] : den[p - n_num];
        if (!q || !q->n_keys || (q->capacity && (!q->key_ctx || !q->key_node || !q->key_stall || !q->val)))
            return h->fail(HPA_E_INVALID_ARG, "profile %u arrays missing", p);
        if (q->n_stall == 0 || q->n_stall > HPA_MAX_STALL || q->n_ctx == 0)
            return h->fail(HPA_E_INVALID_ARG, "profile %u has no n_ctx / n_stall", p);
        ps[p] = q;
        N += q->capacity;
        G = std::max(G, q->n_ctx);
        S = std::max(S, q->n_stall);
    }
    if (!out->n_keys || (out->capacity && (!out->key_ctx || !out->key_node || !out->key_stall || !out->num ||
                                           !out->den || !out->ratio)))
        return h->fail(HPA_E_INVALID_ARG, "output arrays missing");
    if (N >= 0xFFFFFFF0ull) return h->fail(HPA_E_INVALID_ARG, "too many keys in one call");
    if (N == 0) return h->cuda(cudaMemsetAsync(out->n_keys, 0, sizeof(uint64_t), h->stream), "ratio");
    const uint32_t M = B->n_nodes;
    const uint32_t sb = ceil_log2_u64(S);
    const uint32_t nb = ceil_log2_u64((uint64_t)M + 1);
    if (nb + sb + 1 > 32) return h->fail(HPA_E_INVALID_ARG, "(n_nodes + 1) * 2^(stall_bits + 1) exceeds 2^32");
    // the regrouped keys (ctx, node, stall << 1 | group, sum) and the run flags
    auto layout = [&](Carve& c, hpa_profile& g, uint32_t*& head, uint32_t*& stmp) {
        g.key_ctx = c.take<uint32_t>(N + 1);
        g.key_node = c.take<uint32_t>(N + 1);
        g.key_stall = c.take<uint8_t>(N + 1);
        g.val = c.take<uint64_t>(N + 1);
        g.n_keys = c.take<uint64_t>(2);
        head = c.take<uint32_t>(N + 1);
        stmp = c.take<uint32_t>(scan_tmp_words(N + 1));
    };
    hpa_profile g{};
    uint32_t *head = nullptr, *stmp = nullptr;
    Carve probe{nullptr};
    layout(probe, g, head, stmp);
    if (probe.off + 256 > h->aux_cap) {
        hpa_status st = h->cuda(cudaStreamSynchronize(h->stream), "sync");
        if (st) return st;
        if (h->aux_scratch) cudaFree(h->aux_scratch);
        h->aux_scratch = nullptr;
        h->aux_cap = 0;
        if (cudaMalloc(&h->aux_scratch, probe.off + 256) != cudaSuccess) {
            cudaGetLastError();
            return h->fail(HPA_E_OOM, "ratio keys of %zu bytes", probe.off + 256);
        }
        h->aux_cap = probe.off + 256;
    }
    Carve c{(char*)h->aux_scratch};
    layout(c, g, head, stmp);
    g.capacity = N;
    g.n_stall = 2 * S;
    AggWork w{};
    hpa_status st = h->carve_work(w, N, G, 1, LEAF_CAP_SMALL, sb + 1, nb + sb + 1, true, true);
    if (st) return st;
    // descriptors: profiles, their flattened bases, and the single output
    if ((st = h->ensure_staging(P * sizeof(RatioProf) + (P + 1) * 8 + sizeof(BufDev) + 4096))) return st;
    Carve hs{(char*)h->staging};
    RatioProf* hp = hs.take<RatioProf>(P);
    uint64_t* hbase = hs.take<uint64_t>(P + 1);
    BufDev* hb = hs.take<BufDev>(1);
    uint64_t* htile = hs.take<uint64_t>(2);
    uint32_t* hgrp = hs.take<uint32_t>(2);
    uint64_t base = 0;
    for (uint32_t p = 0; p < P; ++p) {
        const hpa_profile* q = ps[p];
        hp[p] = RatioProf{q->key_ctx, q->key_node, q->key_stall, q->val, q->n_keys, q->capacity, base};
        hbase[p] = base;
        base += q->capacity;
    }
    hbase[P] = base;
    BufDev d{};
    d.n_ctx = G; d.n_stall = 2 * S; d.grp_base = 0; d.bin = binary_id;
    d.key_ctx = g.key_ctx; d.key_node = g.key_node; d.key_stall = g.key_stall; d.val = g.val;
    d.n_keys = g.n_keys; d.capacity = N;
    *hb = d;
    htile[0] = htile[1] = 0;
    hgrp[0] = 0; hgrp[1] = G;
    if ((st = h->upload_staging(hs.off))) return st;
    char* ds = (char*)h->d_staging;
    auto dev = [&](void* hostp) { return ds + ((char*)hostp - (char*)h->staging); };
    w.bufs = (const BufDev*)dev(hb);
    w.buf_tile = (const uint64_t*)dev(htile);
    w.buf_grp = (const uint32_t*)dev(hgrp);
    w.n_tiles = 0;
    w.emit_totals = 0;
    RatioSrc x{(const RatioProf*)dev(hp), (const uint64_t*)dev(hbase), P, n_num, N, M, G, S, sb};
    cudaStream_t s = h->stream;
    clear_work(w, s);
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((N + 255) / 256, (uint64_t)h->sms * 8));
    k_ratio_hist<<<blocks, 256, 0, s>>>(w, x);
    run_plan(w, s, h->sms, &h->launches, false);
    k_ratio_scatter<<<blocks, 256, 0, s>>>(w, x);
    h->launches += 2;
    run_group_tail(w, s, h->sms, &h->launches);
    k_ratio_heads<<<blocks, 256, 0, s>>>(g.key_ctx, g.key_node, g.key_stall, g.n_keys, N, head);
    scan_u32(head, head, N, stmp, s, &h->launches);
    k_ratio_rows<<<blocks, 256, 0, s>>>(g.key_ctx, g.key_node, g.key_stall, g.val, g.n_keys, N, head, *out,
                                        h->d_status);
    h->launches += 2;
    return h->cuda(cudaGetLastError(), "ratio launch");
}
