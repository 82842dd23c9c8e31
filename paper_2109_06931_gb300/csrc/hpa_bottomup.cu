// hpa_bottom_up_view: the bottom-up view of a profile (Section 7): the costs
// of each function divided among the calling contexts in which it is
// called.  A node of the view is a function followed by a caller chain --
// the call sites met walking up the calling context tree from a launch
// context, its own site first -- and holds, per stall reason, the values of
// the keys of that function whose context's chain begins with it.
//
// Level by level over the keys: every live key carries the view node it
// reached at the previous level and the CCT node whose call site labels the
// next one.  A level's nodes are the distinct (previous node, label) pairs,
// found with a 64-bit hash table whose slots keep the smallest key index
// (so a node is numbered by the first key, in profile order, that reaches
// it: an exclusive scan of "key is its node's representative" flags).  A
// bit mask of stall reasons per node and a scan of their popcounts place
// each (node, stall) value, which the keys add up with 64-bit atomics --
// exact, so the order of the additions does not matter.  Call sites are
// first replaced by their representative CCT node so that a label is 32
// bits.

#include "hpa_hash.cuh"
#include "hpa_host.h"

namespace hpa {

constexpr uint32_t BU_DEAD = 0xFFFFFFFEu;   // key without a node at this level (UNKNOWN, or chain ended)

struct BuArgs {
    // profile
    const uint32_t* ctx;
    const uint32_t* node;
    const uint8_t* stall;
    const uint64_t* val;
    const uint64_t* n_keys;
    uint64_t kcap;                // capacity of the key arrays (reads stay below it)
    uint64_t K;                   // max(kcap, 1): length of the per-key scratch and scans
    uint32_t n_ctx, n_stall, M;
    const uint32_t* node_func;
    // calling context tree
    uint32_t n_cct;
    const uint32_t* cparent;
    const uint16_t* cmodule;
    const uint64_t* coffset;
    uint32_t* site_rep;           // [n_cct]
    // per key
    uint32_t* at;                 // view node reached at the previous level
    uint32_t* anc;                // CCT node labelling the next level
    uint32_t* rep;                // representative key, then the node's rank within the level
    uint32_t* rank;               // [K + 1]
    uint32_t* mask;               // [K] stall reasons present per node of the level
    uint32_t* voff;               // [K + 1]
    unsigned long long* tkeys;
    uint32_t* tvals;
    uint32_t tmask;
    unsigned long long* bases;    // [2] nodes, values before this level
    DevStatus* status;
};

__device__ __forceinline__ uint64_t bu_keys(const BuArgs& a) { return min(*a.n_keys, a.kcap); }

__global__ void k_bu_sites(BuArgs a, int pass) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < a.n_cct; v += gridDim.x * blockDim.x) {
        const unsigned long long key = ((unsigned long long)a.cmodule[v] << 48) | (a.coffset[v] & 0xFFFFFFFFFFFFull);
        if (pass == 0) {
            const uint32_t p = a.cparent[v];
            if ((p != HPA_NO_PARENT && p >= v) || a.cmodule[v] == 0xFFFFu || (a.coffset[v] >> 48))
                raise_status(a.status, 2 /* HPA_E_INVALID_TABLE */, (int32_t)v);
            const uint32_t slot = ut_insert(a.tkeys, a.tvals, a.tmask, key, v);
            if (slot > a.tmask) raise_status(a.status, 8 /* HPA_E_INTERNAL */, 3);
            a.site_rep[v] = slot;
        } else {
            const uint32_t slot = a.site_rep[v];
            const uint32_t r = slot <= a.tmask ? a.tvals[slot] : v;
            a.site_rep[v] = r < a.n_cct ? r : v;
        }
    }
}

__global__ void k_bu_keys_init(BuArgs a) {
    const uint64_t Kd = bu_keys(a);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < Kd; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = a.ctx[i], n = a.node[i];
        if (c >= a.n_ctx || c >= a.n_cct || a.stall[i] >= a.n_stall || (n != UNKNOWN && n >= a.M)) {
            atomicAdd(&a.status->bad, 1ull);
            raise_status(a.status, 3 /* HPA_E_INVALID_SAMPLE */, 0);
            a.at[i] = BU_DEAD;
            continue;
        }
        a.at[i] = n == UNKNOWN ? BU_DEAD : HPA_NO_PARENT;
        a.anc[i] = c;
    }
}

__device__ __forceinline__ bool bu_live(const BuArgs& a, uint64_t i, uint32_t lev, unsigned long long* key) {
    const uint32_t at = a.at[i];
    if (at == BU_DEAD) return false;
    uint32_t label;
    if (lev == 0) {
        label = a.node_func[a.node[i]];
    } else {
        const uint32_t c = a.anc[i];
        if (c == HPA_NO_PARENT) return false;
        label = a.site_rep[c];
    }
    *key = ((unsigned long long)at << 32) | label;
    return true;
}

// insertion keeps each key's slot in rep[]; the next pass reads the slot's
// representative (the smallest key index inserted there)
__global__ void k_bu_insert(BuArgs a, uint32_t lev) {
    const uint64_t Kd = bu_keys(a);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < Kd; i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long key;
        uint32_t slot = HPA_NO_PARENT;
        if (bu_live(a, i, lev, &key)) {
            slot = ut_insert(a.tkeys, a.tvals, a.tmask, key, (uint32_t)i);
            if (slot > a.tmask) raise_status(a.status, 8, 4);
        }
        a.rep[i] = slot;
    }
}

__global__ void k_bu_find(BuArgs a, uint32_t lev) {
    const uint64_t Kd = bu_keys(a);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.K; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t slot = i < Kd ? a.rep[i] : HPA_NO_PARENT;
        const uint32_t r = slot <= a.tmask ? a.tvals[slot] : HPA_NO_PARENT;
        a.rep[i] = r;
        a.rank[i] = r == (uint32_t)i;
    }
}

__global__ void k_bu_nodes(BuArgs a, uint32_t lev, hpa_bottom_up o) {
    const uint64_t Kd = bu_keys(a);
    const unsigned long long base = a.bases[0];
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < Kd; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = a.rep[i];
        if (r >= a.K) continue;                      // no node at this level (or a raised status)
        const uint32_t local = a.rank[r];
        a.rep[i] = local;
        atomicOr(&a.mask[local], 1u << a.stall[i]);
        const unsigned long long id = base + local;
        if (r != (uint32_t)i || id >= o.cap_nodes) continue;
        o.parent[id] = a.at[i];
        o.func[id] = a.node_func[a.node[i]];
        o.module[id] = lev == 0 ? (uint16_t)0xFFFFu : a.cmodule[a.anc[i]];
        o.offset[id] = lev == 0 ? 0ull : a.coffset[a.anc[i]];
    }
}

__global__ void k_bu_popc(BuArgs a) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < a.K; j += (uint64_t)gridDim.x * blockDim.x)
        a.voff[j] = __popc(a.mask[j]);
}

__global__ void k_bu_values(BuArgs a, uint32_t lev, hpa_bottom_up o) {
    const uint64_t Kd = bu_keys(a);
    const unsigned long long nb = a.bases[0], vb = a.bases[1];
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < Kd; i += (uint64_t)gridDim.x * blockDim.x) {
        if (a.at[i] == BU_DEAD) continue;
        if (lev > 0 && a.anc[i] == HPA_NO_PARENT) { a.at[i] = BU_DEAD; continue; }
        const uint32_t local = a.rep[i];
        if (local >= a.K) { a.at[i] = BU_DEAD; continue; }   // only after a raised status
        const uint32_t s = a.stall[i];
        const unsigned long long pos = vb + a.voff[local] + __popc(a.mask[local] & ((1u << s) - 1u));
        if (pos < o.cap_values) {
            atomicAdd((unsigned long long*)&o.val[pos], (unsigned long long)a.val[i]);
            o.val_node[pos] = (uint32_t)(nb + local);
            o.val_stall[pos] = (uint8_t)s;
        }
        a.at[i] = (uint32_t)(nb + local);
        if (lev > 0) a.anc[i] = a.cparent[a.anc[i]];
    }
}

__global__ void k_bu_level_end(BuArgs a, uint32_t lev, hpa_bottom_up o) {
    if (o.level_off) o.level_off[lev] = a.bases[0];
    a.bases[0] += a.rank[a.K];
    a.bases[1] += a.voff[a.K];
    if (a.bases[0] >= BU_DEAD) raise_status(a.status, 4 /* HPA_E_CAPACITY */, 1);   // ids are 32-bit
}

__global__ void k_bu_finish(BuArgs a, hpa_bottom_up o) {
    if (o.level_off) o.level_off[o.levels + 1] = a.bases[0];
    o.counts[0] = a.bases[0];
    o.counts[1] = a.bases[1];
    if (a.bases[0] > o.cap_nodes || a.bases[1] > o.cap_values) raise_status(a.status, 4 /* HPA_E_CAPACITY */, 0);
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_bottom_up_view(hpa_handle* h, uint32_t binary_id, const hpa_profile* p,
                                         const hpa_cct_nodes* cct, hpa_bottom_up* out) {
    hpa::Trace trace_("hpa.bottom_up_view");
    if (!h || !p || !cct || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = h->binary(binary_id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", binary_id);
    if (!p->n_keys || (p->capacity && (!p->key_ctx || !p->key_node || !p->key_stall || !p->val)))
        return h->fail(HPA_E_INVALID_ARG, "input profile arrays missing");
    if (p->n_stall == 0 || p->n_stall > HPA_MAX_STALL || p->n_ctx == 0)
        return h->fail(HPA_E_INVALID_ARG, "input profile has no n_ctx / n_stall (produce it with hpa_attribute_samples)");
    if (!cct->parent || !cct->module || !cct->offset || cct->n_nodes == 0)
        return h->fail(HPA_E_INVALID_ARG, "calling context tree arrays missing");
    if (cct->n_nodes < p->n_ctx) return h->fail(HPA_E_INVALID_ARG, "the tree has fewer nodes than the profile has contexts");
    if (!out->counts || (out->cap_nodes && (!out->parent || !out->func || !out->module || !out->offset)) ||
        (out->cap_values && (!out->val_node || !out->val_stall || !out->val)))
        return h->fail(HPA_E_INVALID_ARG, "output arrays missing");
    if (out->levels > 1024) return h->fail(HPA_E_INVALID_ARG, "levels must be <= 1024");
    const uint64_t K = std::max<uint64_t>(p->capacity, 1);
    if (K >= 0x7FFFFFFFull || cct->n_nodes >= 0x7FFFFFFFu)
        return h->fail(HPA_E_INVALID_ARG, "profile capacity and tree nodes must be < 2^31");
    uint32_t tlog = 1;
    while ((1ull << tlog) < 2 * std::max<uint64_t>(K, cct->n_nodes)) ++tlog;
    const uint64_t TS = 1ull << tlog;
    BuArgs a{};
    uint32_t* scan_tmp = nullptr;
    auto layout = [&](Carve& c) {
        a.site_rep = c.take<uint32_t>(cct->n_nodes);
        a.at = c.take<uint32_t>(K + 1);
        a.anc = c.take<uint32_t>(K + 1);
        a.rep = c.take<uint32_t>(K + 1);
        a.rank = c.take<uint32_t>(K + 1);
        a.mask = c.take<uint32_t>(K + 1);
        a.voff = c.take<uint32_t>(K + 1);
        a.tkeys = c.take<unsigned long long>(TS);
        a.tvals = c.take<uint32_t>(TS);
        a.bases = c.take<unsigned long long>(2);
        scan_tmp = c.take<uint32_t>(scan_tmp_words(K + 1));
    };
    Carve probe{nullptr};
    layout(probe);
    hpa_status st = h->ensure_scratch(probe.off + 256);
    if (st) return st;
    Carve c{(char*)h->scratch};
    layout(c);
    a.ctx = p->key_ctx; a.node = p->key_node; a.stall = p->key_stall; a.val = p->val; a.n_keys = p->n_keys;
    a.kcap = p->capacity; a.K = K; a.n_ctx = p->n_ctx; a.n_stall = p->n_stall; a.M = B->n_nodes; a.node_func = B->cg.node_func;
    a.n_cct = cct->n_nodes; a.cparent = cct->parent; a.cmodule = cct->module; a.coffset = cct->offset;
    a.tmask = (uint32_t)(TS - 1); a.status = h->d_status;
    cudaStream_t s = h->stream;
    const int blocks = h->sms * 8;
    const hpa_bottom_up o = *out;
    if (o.cap_values) cudaMemsetAsync(o.val, 0, o.cap_values * 8, s);
    cudaMemsetAsync(a.bases, 0, 16, s);
    cudaMemsetAsync(a.tkeys, 0xFF, TS * 8, s);
    cudaMemsetAsync(a.tvals, 0xFF, TS * 4, s);
    k_bu_sites<<<blocks, 256, 0, s>>>(a, 0);
    k_bu_sites<<<blocks, 256, 0, s>>>(a, 1);
    k_bu_keys_init<<<blocks, 256, 0, s>>>(a);
    uint64_t n_launch = 4;
    for (uint32_t lev = 0; lev <= o.levels; ++lev) {
        cudaMemsetAsync(a.tkeys, 0xFF, TS * 8, s);
        cudaMemsetAsync(a.tvals, 0xFF, TS * 4, s);
        cudaMemsetAsync(a.mask, 0, (K + 1) * 4, s);
        k_bu_insert<<<blocks, 256, 0, s>>>(a, lev);
        k_bu_find<<<blocks, 256, 0, s>>>(a, lev);
        scan_u32(a.rank, a.rank, K, scan_tmp, s, &h->launches);
        k_bu_nodes<<<blocks, 256, 0, s>>>(a, lev, o);
        k_bu_popc<<<blocks, 256, 0, s>>>(a);
        scan_u32(a.voff, a.voff, K, scan_tmp, s, &h->launches);
        k_bu_values<<<blocks, 256, 0, s>>>(a, lev, o);
        k_bu_level_end<<<1, 1, 0, s>>>(a, lev, o);
        n_launch += 6;
    }
    k_bu_finish<<<1, 1, 0, s>>>(a, o);
    h->launches += n_launch;
    return h->cuda(cudaGetLastError(), "bottom-up view launch");
}
