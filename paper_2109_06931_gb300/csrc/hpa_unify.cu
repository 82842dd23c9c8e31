// hpa_unify_ccts: call-path profile unification (Section 6.1): the calling
// context trees of several profiles merged into one tree, and every input
// node mapped to its node of the merged tree.  A node is identified by its
// parent's merged node and its call site (load module, offset).
//
// Representatives instead of a sequential walk: the site of a node is
// represented by the first node (in the concatenated input order) with the
// same (module, offset), and a node by the first node with the same (parent's
// representative, site's representative) -- both found with 64-bit keys in
// open-addressing tables (compare-and-swap on the key, minimum of the node
// index).  Nodes are keyed level by level (depth from pointer jumping), so a
// parent's representative is final before its children are keyed.  Merged
// ids are the ranks of the representatives: the order of first occurrence.

#include "hpa_hash.cuh"
#include "hpa_host.h"

namespace hpa {

struct UnifyDesc {
    const uint32_t* parent;
    const uint16_t* module;
    const uint64_t* offset;
    uint64_t base;
};

struct UnifyArgs {
    const UnifyDesc* ccts;
    const uint64_t* bases;    // [n + 1]
    uint32_t n;
    uint64_t N;
    uint32_t* gparent;        // global parent index or HPA_NO_PARENT
    uint32_t* anc[2];
    uint32_t* dep[2];
    uint32_t* site_rep;
    uint32_t* rep;
    uint32_t* rank;           // [N + 1] is-representative flags -> exclusive scan
    unsigned long long* skeys;
    uint32_t* svals;
    unsigned long long* nkeys;
    uint32_t* nvals;
    uint32_t tmask;
    uint32_t* maxdep;
    DevStatus* status;
};

__global__ void k_un_init(UnifyArgs a) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.N; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = upper_index<uint64_t>(a.bases, a.n, i);
        const UnifyDesc& d = a.ccts[p];
        const uint64_t j = i - d.base;
        const uint32_t par = d.parent[j];
        uint32_t g = HPA_NO_PARENT;
        if (par != HPA_NO_PARENT) {
            if (par >= j) raise_status(a.status, 2 /* HPA_E_INVALID_TABLE */, (int32_t)p);
            else g = (uint32_t)(d.base + par);
        }
        if (d.module[j] == 0xFFFFu || (d.offset[j] >> 48)) raise_status(a.status, 2, (int32_t)p);
        a.gparent[i] = g;
        a.anc[0][i] = g;
        a.dep[0][i] = g != HPA_NO_PARENT;
    }
}

// one pointer-jumping round: depth += depth of the current ancestor, ancestor = its ancestor
__global__ void k_un_jump(UnifyArgs a, int from) {
    const uint32_t* an = a.anc[from];
    const uint32_t* de = a.dep[from];
    uint32_t* an2 = a.anc[from ^ 1];
    uint32_t* de2 = a.dep[from ^ 1];
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.N; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = an[i];
        if (x == HPA_NO_PARENT) { an2[i] = x; de2[i] = de[i]; continue; }
        an2[i] = an[x];
        de2[i] = de[i] + de[x];
    }
}

__global__ void k_un_sites(UnifyArgs a, int pass, int cur) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.N; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = upper_index<uint64_t>(a.bases, a.n, i);
        const UnifyDesc& d = a.ccts[p];
        const uint64_t j = i - d.base;
        const unsigned long long key = ((unsigned long long)d.module[j] << 48) | (d.offset[j] & 0xFFFFFFFFFFFFull);
        if (pass == 0) {                                // the slot waits in site_rep for pass 1
            const uint32_t slot = ut_insert(a.skeys, a.svals, a.tmask, key, (uint32_t)i);
            if (slot > a.tmask) raise_status(a.status, 8 /* HPA_E_INTERNAL */, 1);
            a.site_rep[i] = slot;
            atomicMax(a.maxdep, a.dep[cur][i]);
        } else {
            const uint32_t slot = a.site_rep[i];
            a.site_rep[i] = slot <= a.tmask ? a.svals[slot] : 0xFFFFFFFFu;
        }
    }
}

__global__ void k_un_level(UnifyArgs a, uint32_t level, int cur, int pass) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.N; i += (uint64_t)gridDim.x * blockDim.x) {
        if (a.dep[cur][i] != level) continue;
        const uint32_t g = a.gparent[i];
        const uint32_t pk = g == HPA_NO_PARENT ? 0xFFFFFFFFu : a.rep[g];
        if (a.site_rep[i] >= a.N) { if (pass) a.rep[i] = HPA_NO_PARENT; continue; }   // only after a raised status
        const unsigned long long key = ((unsigned long long)pk << 32) | a.site_rep[i];
        if (pass == 0) {                                // the slot waits in rep for pass 1
            const uint32_t slot = ut_insert(a.nkeys, a.nvals, a.tmask, key, (uint32_t)i);
            if (slot > a.tmask) raise_status(a.status, 8, 2);
            a.rep[i] = slot;
        } else {
            const uint32_t slot = a.rep[i];
            a.rep[i] = slot <= a.tmask ? a.nvals[slot] : HPA_NO_PARENT;
        }
    }
}

__global__ void k_un_flags(UnifyArgs a) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.N; i += (uint64_t)gridDim.x * blockDim.x)
        a.rank[i] = a.rep[i] == (uint32_t)i;
}

__global__ void k_un_output(UnifyArgs a, hpa_cct_unified o) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.N; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = a.rep[i];
        o.uid[i] = r < a.N ? a.rank[r] : HPA_NO_PARENT;     // r >= N only after a raised status
        if (r != (uint32_t)i) continue;
        const uint32_t u = a.rank[i];
        if (u >= o.capacity) continue;
        const uint32_t p = upper_index<uint64_t>(a.bases, a.n, i);
        const UnifyDesc& d = a.ccts[p];
        const uint64_t j = i - d.base;
        const uint32_t g = a.gparent[i];
        const uint32_t gr = g == HPA_NO_PARENT ? HPA_NO_PARENT : a.rep[g];
        o.parent[u] = gr < a.N ? a.rank[gr] : HPA_NO_PARENT;
        o.module[u] = d.module[j];
        o.offset[u] = d.offset[j];
    }
}

__global__ void k_un_finish(UnifyArgs a, hpa_cct_unified o) {
    const uint64_t nu = a.rank[a.N];
    *o.n_unified = nu;
    if (nu > o.capacity) raise_status(a.status, 4 /* HPA_E_CAPACITY */, 0);
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_unify_ccts(hpa_handle* h, const hpa_cct_nodes* ccts, uint32_t n, hpa_cct_unified* out) {
    hpa::Trace trace_("hpa.unify_ccts");
    if (!h || !ccts || !out || n == 0) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    if (!out->uid || !out->n_unified || (out->capacity && (!out->parent || !out->module || !out->offset)))
        return h->fail(HPA_E_INVALID_ARG, "unified CCT output arrays missing");
    uint64_t N = 0;
    for (uint32_t p = 0; p < n; ++p) {
        if (ccts[p].n_nodes && (!ccts[p].parent || !ccts[p].module || !ccts[p].offset))
            return h->fail(HPA_E_INVALID_ARG, "CCT %u arrays missing", p);
        N += ccts[p].n_nodes;
    }
    if (N == 0 || N >= 0x7FFFFFFFull) return h->fail(HPA_E_INVALID_ARG, "total CCT nodes must be in [1, 2^31)");
    uint32_t tlog = 1;
    while ((1ull << tlog) < 2 * N) ++tlog;
    const uint64_t TS = 1ull << tlog;
    UnifyArgs a{};
    uint32_t* scan_tmp = nullptr;
    auto layout = [&](Carve& c) {
        a.gparent = c.take<uint32_t>(N);
        a.anc[0] = c.take<uint32_t>(N); a.anc[1] = c.take<uint32_t>(N);
        a.dep[0] = c.take<uint32_t>(N); a.dep[1] = c.take<uint32_t>(N);
        a.site_rep = c.take<uint32_t>(N);
        a.rep = c.take<uint32_t>(N);
        a.rank = c.take<uint32_t>(N + 1);
        a.skeys = c.take<unsigned long long>(TS);
        a.svals = c.take<uint32_t>(TS);
        a.nkeys = c.take<unsigned long long>(TS);
        a.nvals = c.take<uint32_t>(TS);
        a.maxdep = c.take<uint32_t>(1);
        scan_tmp = c.take<uint32_t>(scan_tmp_words(N));
    };
    Carve probe{nullptr};
    layout(probe);
    hpa_status st = h->ensure_scratch(probe.off + 256);
    if (st) return st;
    Carve c{(char*)h->scratch};
    layout(c);
    // descriptors
    Carve sp{nullptr};
    sp.take<UnifyDesc>(n);
    sp.take<uint64_t>(n + 1);
    if ((st = h->ensure_staging(sp.off + 256))) return st;
    Carve hs{(char*)h->staging};
    UnifyDesc* hd = hs.take<UnifyDesc>(n);
    uint64_t* hb = hs.take<uint64_t>(n + 1);
    uint64_t base = 0;
    for (uint32_t p = 0; p < n; ++p) {
        hd[p] = UnifyDesc{ccts[p].parent, ccts[p].module, ccts[p].offset, base};
        hb[p] = base;
        base += ccts[p].n_nodes;
    }
    hb[n] = base;
    if ((st = h->upload_staging(hs.off))) return st;
    char* ds = (char*)h->d_staging;
    a.ccts = (const UnifyDesc*)(ds + ((char*)hd - (char*)h->staging));
    a.bases = (const uint64_t*)(ds + ((char*)hb - (char*)h->staging));
    a.n = n; a.N = N; a.tmask = (uint32_t)(TS - 1); a.status = h->d_status;
    cudaStream_t s = h->stream;
    const int blocks = h->sms * 8;
    cudaMemsetAsync(a.skeys, 0xFF, TS * 8, s);
    cudaMemsetAsync(a.svals, 0xFF, TS * 4, s);
    cudaMemsetAsync(a.nkeys, 0xFF, TS * 8, s);
    cudaMemsetAsync(a.nvals, 0xFF, TS * 4, s);
    cudaMemsetAsync(a.maxdep, 0, 4, s);
    k_un_init<<<blocks, 256, 0, s>>>(a);
    int cur = 0;
    uint32_t rounds = 0;
    for (uint64_t span = 1; span < N; span <<= 1, ++rounds) {  // ceil(log2 N) rounds reach every root
        k_un_jump<<<blocks, 256, 0, s>>>(a, cur);
        cur ^= 1;
    }
    k_un_sites<<<blocks, 256, 0, s>>>(a, 0, cur);
    k_un_sites<<<blocks, 256, 0, s>>>(a, 1, cur);
    uint32_t maxdep = 0;
    if ((st = h->cuda(cudaMemcpyAsync(&maxdep, a.maxdep, 4, cudaMemcpyDeviceToHost, s), "depth")) ||
        (st = h->cuda(cudaStreamSynchronize(s), "sync")))
        return st;
    for (uint32_t L = 0; L <= maxdep; ++L) {
        k_un_level<<<blocks, 256, 0, s>>>(a, L, cur, 0);
        k_un_level<<<blocks, 256, 0, s>>>(a, L, cur, 1);
    }
    k_un_flags<<<blocks, 256, 0, s>>>(a);
    scan_u32(a.rank, a.rank, N, scan_tmp, s, &h->launches);
    k_un_output<<<blocks, 256, 0, s>>>(a, *out);
    k_un_finish<<<1, 1, 0, s>>>(a, *out);
    h->launches += 6 + rounds + 2ull * (maxdep + 1);
    return h->cuda(cudaGetLastError(), "CCT unification launch");
}
