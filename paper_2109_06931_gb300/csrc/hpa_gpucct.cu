// Approximate GPU calling context trees (Section 6.3, steps 1-4), one
// launch context per CTA.
//
// Per context c (the keys of c in a profile sorted by (ctx, node, stall)):
//  step 1  exclusive cost of every condensed node and the measured weight of
//          every call site: samples at its call instruction, all stall reasons;
//  step 2  a function with samples whose incoming edges all have zero
//          measured weight gets weight 1 on each incoming edge, and the rule
//          repeats through its callers that have no measured incoming weight
//          (frontier-parallel closure in shared scratch);
//  step 3  the SCC condensation is static (Tarjan at load time); a condensed
//          node left with cost but zero incoming weight gets the step-2 rule
//          again on the condensed graph (FIXUP2);
//  step 4  bottom-up over the condensed DAG's levels (sinks first):
//          incl(v) = excl(v) + sum_{e out of v} w(e)/W(head(e)) * incl(head(e)),
//          a(e) = w(e)/W(head(e)) * incl(head(e)); the ratio of each edge is
//          computed once, then one thread per (node of the level, stall
//          reason), then one per node for its total column.
// Counts are accumulated exactly (integers in FP64, < 2^53); ratios and
// products are FP64; results are rounded once to FP32.

#include <algorithm>

#include "hpa_host.h"

namespace hpa {

constexpr int GPUCCT_THREADS = 1024;   // one CTA per requested context (per SM)

struct CctSlot {
    double* incl;        // [V][M]
    unsigned long long* fS;   // [F]
    unsigned long long* w;    // [E] measured
    unsigned long long* w2;   // [E] after fix-ups
    unsigned long long* W;    // [V]
    double* ratio;       // [E] w(e) / W(head(e)) of external edges
    uint8_t* flags;      // [E]
    uint32_t* inZ;       // [F]
    uint8_t* meas_in;    // [F]
    uint32_t* inZ2;      // [V]
    uint8_t* cneed;      // [V]
    uint32_t* front[2];  // [V] each
};

struct CctArgs {
    DevCallGraph g;
    const uint32_t* key_ctx;
    const uint32_t* key_node;
    const uint8_t* key_stall;
    const uint64_t* key_val;
    const uint64_t* n_keys;
    uint64_t key_cap;
    uint32_t S, M;           // stall reasons, S + 1
    uint32_t n_req;
    const uint32_t* req_ctx;
    float* out_incl;
    float* out_a;
    uint8_t* out_flags;
    char* slots;
    size_t slot_bytes;
    DevStatus* status;
};

__host__ __device__ inline size_t slot_layout(const DevCallGraph& g, uint32_t M, char* base, CctSlot* s) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~size_t(255);
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    CctSlot t;
    t.incl = (double*)take((size_t)g.V * M * 8);
    t.fS = (unsigned long long*)take((size_t)g.F * 8);
    t.w = (unsigned long long*)take((size_t)g.E * 8);
    t.w2 = (unsigned long long*)take((size_t)g.E * 8);
    t.W = (unsigned long long*)take((size_t)g.V * 8);
    t.ratio = (double*)take((size_t)g.E * 8);
    t.flags = (uint8_t*)take(g.E);
    t.inZ = (uint32_t*)take((size_t)g.F * 4);
    t.meas_in = (uint8_t*)take(g.F);
    t.inZ2 = (uint32_t*)take((size_t)g.V * 4);
    t.cneed = (uint8_t*)take(g.V);
    t.front[0] = (uint32_t*)take((size_t)g.V * 4);
    t.front[1] = (uint32_t*)take((size_t)g.V * 4);
    if (s) *s = t;
    return (off + 255) & ~size_t(255);
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_gpucct(CctArgs A) {
    const DevCallGraph& g = A.g;
    __shared__ uint32_t s_cnt[2];
    __shared__ uint64_t s_range[2];
    CctSlot T;
    slot_layout(g, A.M, A.slots + (size_t)blockIdx.x * A.slot_bytes, &T);
    const uint32_t tid = threadIdx.x;
    const uint64_t K = min(*A.n_keys, A.key_cap);

    for (uint32_t q = blockIdx.x; q < A.n_req; q += gridDim.x) {
        const uint32_t c = A.req_ctx[q];
        if (tid == 0) {
            uint64_t lo = 0, hi = K;
            while (lo < hi) { const uint64_t m = (lo + hi) >> 1; if (A.key_ctx[m] < c) lo = m + 1; else hi = m; }
            uint64_t lo2 = lo, hi2 = K;
            while (lo2 < hi2) { const uint64_t m = (lo2 + hi2) >> 1; if (A.key_ctx[m] <= c) lo2 = m + 1; else hi2 = m; }
            s_range[0] = lo; s_range[1] = lo2;
        }
        for (size_t i = tid; i < (size_t)g.V * A.M; i += THREADS) T.incl[i] = 0.0;
        for (uint32_t f = tid; f < g.F; f += THREADS) { T.fS[f] = 0; T.inZ[f] = 0; }
        for (uint32_t e = tid; e < g.E; e += THREADS) { T.w[e] = 0; T.flags[e] = g.edge_intra[e] ? HPA_EDGE_INTRA_SCC : 0; }
        for (uint32_t v = tid; v < g.V; v += THREADS) { T.inZ2[v] = 0; T.cneed[v] = 0; }
        __syncthreads();
        // step 1: exclusive costs and measured call-site weights
        for (uint64_t i = s_range[0] + tid; i < s_range[1]; i += THREADS) {
            const uint32_t n = A.key_node[i];
            if (n == UNKNOWN) continue;
            const uint32_t r = A.key_stall[i];
            if (n >= g.M || r >= A.S) { raise_status(A.status, 1 /* HPA_E_INVALID_ARG */, 10); continue; }
            const uint64_t v = A.key_val[i];
            const uint32_t f = g.node_func[n];
            atomicAdd(&T.incl[(size_t)g.cnode_of_func[f] * A.M + r], (double)v);
            atomicAdd(&T.fS[f], (unsigned long long)v);
            const uint32_t e = g.node_cs[n];
            if (e != UNKNOWN) atomicAdd(&T.w[e], (unsigned long long)v);
        }
        __syncthreads();
        for (uint32_t f = tid; f < g.F; f += THREADS) {
            uint8_t m = 0;
            for (uint32_t j = g.fin_off[f]; j < g.fin_off[f + 1]; ++j) m |= T.w[g.fin_edge[j]] > 0;
            T.meas_in[f] = m;
        }
        for (uint32_t e = tid; e < g.E; e += THREADS) T.w2[e] = T.w[e];
        if (tid == 0) s_cnt[0] = 0;
        __syncthreads();
        // step 2: zero-weight fix-up, closure through callers
        for (uint32_t f = tid; f < g.F; f += THREADS)
            if (T.fS[f] > 0 && g.fin_off[f + 1] > g.fin_off[f] && !T.meas_in[f]) {
                T.inZ[f] = 1;
                T.front[0][atomicAdd(&s_cnt[0], 1u)] = f;
            }
        __syncthreads();
        int cur = 0;
        while (true) {
            const uint32_t cnt = s_cnt[cur];
            if (cnt == 0) break;
            if (tid == 0) s_cnt[cur ^ 1] = 0;
            __syncthreads();
            for (uint32_t k = tid; k < cnt; k += THREADS) {
                const uint32_t f = T.front[cur][k];
                for (uint32_t j = g.fin_off[f]; j < g.fin_off[f + 1]; ++j) {
                    const uint32_t e = g.fin_edge[j];
                    T.w2[e] = 1;
                    T.flags[e] |= HPA_EDGE_FIXUP;
                    const uint32_t h = g.cs_caller[e];
                    if (g.fin_off[h + 1] > g.fin_off[h] && !T.meas_in[h] && atomicCAS(&T.inZ[h], 0u, 1u) == 0u)
                        T.front[cur ^ 1][atomicAdd(&s_cnt[cur ^ 1], 1u)] = h;
                }
            }
            __syncthreads();
            cur ^= 1;
        }
        // step 3: condensed graph, incoming weights, FIXUP2
        for (uint32_t v = tid; v < g.V; v += THREADS) {
            unsigned long long Wv = 0;
            for (uint32_t j = g.cin_off[v]; j < g.cin_off[v + 1]; ++j) Wv += T.w2[g.cin_edge[j]];
            T.W[v] = Wv;
        }
        for (uint32_t f = tid; f < g.F; f += THREADS)
            if (T.fS[f] > 0 || T.inZ[f]) T.cneed[g.cnode_of_func[f]] = 1;
        if (tid == 0) s_cnt[0] = 0;
        __syncthreads();
        for (uint32_t v = tid; v < g.V; v += THREADS)
            if (g.cnode_live[v] && T.cneed[v] && g.cin_off[v + 1] > g.cin_off[v] && T.W[v] == 0) {
                T.inZ2[v] = 1;
                T.front[0][atomicAdd(&s_cnt[0], 1u)] = v;
            }
        __syncthreads();
        cur = 0;
        bool any2 = s_cnt[0] > 0;
        while (true) {
            const uint32_t cnt = s_cnt[cur];
            if (cnt == 0) break;
            if (tid == 0) s_cnt[cur ^ 1] = 0;
            __syncthreads();
            for (uint32_t k = tid; k < cnt; k += THREADS) {
                const uint32_t v = T.front[cur][k];
                for (uint32_t j = g.cin_off[v]; j < g.cin_off[v + 1]; ++j) {
                    const uint32_t e = g.cin_edge[j];
                    T.w2[e] = 1;
                    T.flags[e] |= HPA_EDGE_FIXUP2;
                    const uint32_t u = g.cnode_of_func[g.cs_caller[e]];
                    if (g.cin_off[u + 1] > g.cin_off[u] && T.W[u] == 0 && atomicCAS(&T.inZ2[u], 0u, 1u) == 0u)
                        T.front[cur ^ 1][atomicAdd(&s_cnt[cur ^ 1], 1u)] = u;
                }
            }
            __syncthreads();
            cur ^= 1;
        }
        if (any2) {
            for (uint32_t v = tid; v < g.V; v += THREADS) {
                unsigned long long Wv = 0;
                for (uint32_t j = g.cin_off[v]; j < g.cin_off[v + 1]; ++j) Wv += T.w2[g.cin_edge[j]];
                T.W[v] = Wv;
            }
            __syncthreads();
        }
        // step 4: the ratio of every external edge once, then the levels
        // bottom-up: one thread per (node of the level, stall reason), then one
        // per node for its total column and its edges' total shares
        for (uint32_t e = tid; e < g.E; e += THREADS) {
            if (g.edge_intra[e]) continue;
            const uint32_t hd = g.cnode_of_func[g.cs_callee[e]];
            T.ratio[e] = T.W[hd] ? (double)T.w2[e] / (double)T.W[hd] : 0.0;
        }
        __syncthreads();
        float* outA = A.out_a + (size_t)q * g.E * A.M;
        const uint32_t S = A.S;
        for (uint32_t lev = 0; lev < g.n_levels; ++lev) {
            const uint32_t k0 = g.level_off[lev], nk = g.level_off[lev + 1] - k0;
            for (uint32_t it = tid; it < nk * S; it += THREADS) {
                const uint32_t v = g.level_node[k0 + it / S], r = it % S;
                double acc = T.incl[(size_t)v * A.M + r];
                for (uint32_t j = g.cout_off[v]; j < g.cout_off[v + 1]; ++j) {
                    const uint32_t e = g.cout_edge[j];
                    const double x = T.ratio[e] * T.incl[(size_t)g.cout_head[j] * A.M + r];
                    acc += x;
                    outA[(size_t)e * A.M + r] = (float)x;
                }
                T.incl[(size_t)v * A.M + r] = acc;
            }
            __syncthreads();
            for (uint32_t k = k0 + tid; k < k0 + nk; k += THREADS) {
                const uint32_t v = g.level_node[k];
                double* iv = T.incl + (size_t)v * A.M;
                double tot = 0.0;
                for (uint32_t r = 0; r < S; ++r) tot += iv[r];
                iv[S] = tot;
                for (uint32_t j = g.cout_off[v]; j < g.cout_off[v + 1]; ++j) {
                    const uint32_t e = g.cout_edge[j];
                    outA[(size_t)e * A.M + S] = (float)(T.ratio[e] * T.incl[(size_t)g.cout_head[j] * A.M + S]);
                }
            }
            __syncthreads();
        }
        // outputs: condensed-node rows, zero shares of internal SCC edges, flags
        float* outI = A.out_incl + (size_t)q * g.V * A.M;
        for (size_t i = tid; i < (size_t)g.V * A.M; i += THREADS)
            outI[i] = g.cnode_live[i / A.M] ? (float)T.incl[i] : 0.0f;
        for (uint32_t e = tid; e < g.E; e += THREADS) {
            if (g.edge_intra[e])
                for (uint32_t r = 0; r < A.M; ++r) outA[(size_t)e * A.M + r] = 0.0f;
            A.out_flags[(size_t)q * g.E + e] = T.flags[e];
        }
        __syncthreads();
    }
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_apportion_callgraph(hpa_handle* h, uint32_t binary_id, const hpa_profile* p,
                                              hpa_gpucct* out) {
    hpa::Trace trace_("hpa.apportion_callgraph");
    if (!h || !p || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = h->binary(binary_id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", binary_id);
    if (!p->n_keys || (p->capacity && (!p->key_ctx || !p->key_node || !p->key_stall || !p->val)))
        return h->fail(HPA_E_INVALID_ARG, "profile arrays missing");
    if (p->n_stall == 0 || p->n_stall > HPA_MAX_STALL)
        return h->fail(HPA_E_INVALID_ARG, "profile has no n_stall (produce it with hpa_attribute_samples)");
    if (out->n_req == 0) return HPA_OK;
    if (!out->req_ctx || !out->incl || !out->a || !out->flags) return h->fail(HPA_E_INVALID_ARG, "gpucct arrays missing");
    const DevCallGraph& g = B->cg;
    if (g.F == 0) return h->fail(HPA_E_INVALID_ARG, "binary has no functions");
    CctArgs A{};
    A.g = g;
    A.key_ctx = p->key_ctx; A.key_node = p->key_node; A.key_stall = p->key_stall; A.key_val = p->val;
    A.n_keys = p->n_keys; A.key_cap = p->capacity;
    A.S = p->n_stall; A.M = p->n_stall + 1;
    A.n_req = out->n_req; A.req_ctx = out->req_ctx;
    A.out_incl = out->incl; A.out_a = out->a; A.out_flags = out->flags;
    A.status = h->d_status;
    A.slot_bytes = slot_layout(g, A.M, nullptr, nullptr);
    const uint32_t grid = std::min<uint32_t>(out->n_req, (uint32_t)h->sms);
    hpa_status st = h->ensure_scratch(A.slot_bytes * grid + 256);
    if (st) return st;
    A.slots = (char*)h->scratch;
    k_gpucct<GPUCCT_THREADS><<<grid, GPUCCT_THREADS, 0, h->stream>>>(A);
    h->launches += 1;
    return h->cuda(cudaGetLastError(), "apportion launch");
}
