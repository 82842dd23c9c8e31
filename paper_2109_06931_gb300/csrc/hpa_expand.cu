// hpa_expand_gpucct: the GPU calling context tree of one context
// materialised as a tree (Section 6.3, step 4: apportioning the condensed
// call graph is the same as splitting it into a tree in which every call
// path from a root carries the product of the call-site ratios along it).
// Breadth-first, level by level: the roots are the condensed nodes without
// external callers, in node order; a tree node for condensed node v at scale
// s has, for every external call site e of v in call-site order, the child
// h = callee's condensed node at scale s * r(e), with
// r(e) = a(e) / incl(h) (total column) from the apportioning result.  Children
// with zero scale or zero inclusive cost are not materialised.  A tree node's
// inclusive cost is incl(h) * scale.  At most `budget` nodes are written;
// a level that does not fit entirely is cut in order and flagged.

#include "hpa_host.h"

namespace hpa {

struct TreeArgs {
    DevCallGraph cg;
    const float* incl;   // [V][S1] of the context
    const float* a;      // [E][S1]
    uint32_t S1;
    uint32_t budget;
    uint32_t* parent;
    uint32_t* cnode;
    uint32_t* edge;
    float* scale;
    float* out_incl;     // [budget][S1]
    uint64_t* n_nodes;
    uint32_t* truncated;
    double* s64;         // [budget] scales in FP64 while expanding
    uint32_t* cnt;       // [budget + 1] children per frontier node -> exclusive offsets
    uint32_t* lvl;       // [4] frontier start, frontier end, nodes used, truncated
};

__device__ __forceinline__ double ratio(const TreeArgs& t, uint32_t e, uint32_t& h) {
    h = t.cg.cnode_of_func[t.cg.cs_callee[e]];
    const float ih = t.incl[(size_t)h * t.S1 + t.S1 - 1];
    if (!(ih > 0.f)) return 0.0;
    return (double)t.a[(size_t)e * t.S1 + t.S1 - 1] / (double)ih;
}

__device__ __forceinline__ void put(const TreeArgs& t, uint32_t pos, uint32_t par, uint32_t v, uint32_t e, double s) {
    t.parent[pos] = par;
    t.cnode[pos] = v;
    t.edge[pos] = e;
    t.s64[pos] = s;
    t.scale[pos] = (float)s;
    for (uint32_t r = 0; r < t.S1; ++r) t.out_incl[(size_t)pos * t.S1 + r] = (float)(t.incl[(size_t)v * t.S1 + r] * s);
}

// roots: live condensed nodes with no external caller and a nonzero cost
__global__ void __launch_bounds__(1024) k_tree_roots(TreeArgs t) {
    __shared__ uint32_t sw[33];
    uint32_t used = 0;
    for (uint32_t base = 0; base < t.cg.V; base += 1024) {
        const uint32_t v = base + threadIdx.x;
        const bool root = v < t.cg.V && t.cg.cnode_live[v] && t.cg.cin_off[v + 1] == t.cg.cin_off[v] &&
                          t.incl[(size_t)v * t.S1 + t.S1 - 1] > 0.f;
        uint32_t tot;
        const uint32_t pos = used + block_exclusive_scan<uint32_t, 1024>(root ? 1u : 0u, sw, &tot);
        if (root && pos < t.budget) put(t, pos, HPA_NO_PARENT, v, HPA_NO_PARENT, 1.0);
        used += tot;
    }
    if (threadIdx.x == 0) {
        const uint32_t n = min(used, t.budget);
        t.lvl[0] = 0; t.lvl[1] = n; t.lvl[2] = n; t.lvl[3] = used > t.budget;
    }
}

__global__ void k_tree_count(TreeArgs t) {
    const uint32_t f0 = t.lvl[0], f1 = t.lvl[1];
    for (uint32_t i = f0 + blockIdx.x * blockDim.x + threadIdx.x; i < f1; i += gridDim.x * blockDim.x) {
        const uint32_t v = t.cnode[i];
        const double s = t.s64[i];
        uint32_t c = 0;
        for (uint32_t k = t.cg.cout_off[v]; k < t.cg.cout_off[v + 1]; ++k) {
            uint32_t h;
            const double r = ratio(t, t.cg.cout_edge[k], h);
            c += s * r > 0.0;
        }
        t.cnt[i - f0] = c;
    }
}

// exclusive scan of the frontier's child counts (one CTA; frontier <= budget)
__global__ void __launch_bounds__(1024) k_tree_scan(TreeArgs t) {
    __shared__ uint32_t sw[33];
    const uint32_t n = t.lvl[1] - t.lvl[0];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < n ? t.cnt[i] : 0;
        uint32_t tot;
        const uint32_t e = block_exclusive_scan<uint32_t, 1024>(x, sw, &tot);
        if (i < n) t.cnt[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) t.cnt[n] = carry;
}

__global__ void k_tree_write(TreeArgs t) {
    const uint32_t f0 = t.lvl[0], f1 = t.lvl[1], used = t.lvl[2];
    for (uint32_t i = f0 + blockIdx.x * blockDim.x + threadIdx.x; i < f1; i += gridDim.x * blockDim.x) {
        const uint32_t v = t.cnode[i];
        const double s = t.s64[i];
        uint64_t pos = (uint64_t)used + t.cnt[i - f0];
        for (uint32_t k = t.cg.cout_off[v]; k < t.cg.cout_off[v + 1]; ++k) {
            const uint32_t e = t.cg.cout_edge[k];
            uint32_t h;
            const double r = ratio(t, e, h);
            if (!(s * r > 0.0)) continue;
            if (pos < t.budget) put(t, (uint32_t)pos, i, h, e, s * r);
            ++pos;
        }
    }
}

__global__ void k_tree_advance(TreeArgs t) {
    const uint32_t n = t.lvl[1] - t.lvl[0];
    const uint64_t want = (uint64_t)t.lvl[2] + t.cnt[n];
    const uint32_t end = (uint32_t)(want < (uint64_t)t.budget ? want : (uint64_t)t.budget);
    if (want > t.budget) t.lvl[3] = 1;
    t.lvl[0] = t.lvl[2];
    t.lvl[1] = end;
    t.lvl[2] = end;
}

__global__ void k_tree_finish(TreeArgs t) {
    *t.n_nodes = t.lvl[2];
    *t.truncated = t.lvl[3];
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_expand_gpucct(hpa_handle* h, uint32_t binary_id, const hpa_gpucct* g, uint32_t n_stall,
                                        uint32_t q, hpa_cct_tree* out) {
    hpa::Trace trace_("hpa.expand_gpucct");
    if (!h || !g || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = h->binary(binary_id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", binary_id);
    if (q >= g->n_req || !g->incl || !g->a) return h->fail(HPA_E_INVALID_ARG, "no apportioning result %u", q);
    if (n_stall == 0 || n_stall > HPA_MAX_STALL) return h->fail(HPA_E_INVALID_ARG, "n_stall must be in [1, %u]", HPA_MAX_STALL);
    if (out->budget == 0 || !out->parent || !out->cnode || !out->edge || !out->scale || !out->incl ||
        !out->n_nodes || !out->truncated)
        return h->fail(HPA_E_INVALID_ARG, "tree output arrays missing");
    const uint32_t S1 = n_stall + 1;
    TreeArgs t{};
    t.cg = B->cg;
    t.incl = g->incl + (size_t)q * B->n_cnodes * S1;
    t.a = g->a + (size_t)q * B->n_calls * S1;
    t.S1 = S1;
    t.budget = out->budget;
    t.parent = out->parent; t.cnode = out->cnode; t.edge = out->edge; t.scale = out->scale;
    t.out_incl = out->incl; t.n_nodes = out->n_nodes; t.truncated = out->truncated;
    auto layout = [&](Carve& c) {
        t.s64 = c.take<double>(out->budget);
        t.cnt = c.take<uint32_t>((size_t)out->budget + 1);
        t.lvl = c.take<uint32_t>(4);
    };
    Carve probe{nullptr};
    layout(probe);
    hpa_status st = h->ensure_scratch(probe.off + 256);
    if (st) return st;
    Carve c{(char*)h->scratch};
    layout(c);
    cudaStream_t s = h->stream;
    const int blocks = h->sms * 4;
    k_tree_roots<<<1, 1024, 0, s>>>(t);
    for (uint32_t L = 0; L < B->cdag_levels; ++L) {
        k_tree_count<<<blocks, 256, 0, s>>>(t);
        k_tree_scan<<<1, 1024, 0, s>>>(t);
        k_tree_write<<<blocks, 256, 0, s>>>(t);
        k_tree_advance<<<1, 1, 0, s>>>(t);
    }
    k_tree_finish<<<1, 1, 0, s>>>(t);
    h->launches += 2 + 4ull * B->cdag_levels;
    return h->cuda(cudaGetLastError(), "GPU CCT expansion launch");
}
