// Sparse layouts of several profiles (Section 6.2): the profile-major (PMS)
// and the calling-context-major (CMS) forms, built on the device.
//
// A calling context here is a (launch context, structure node) pair, a
// metric is a stall reason, a profile is one input key list.
//   PMS: for every profile, its contexts (planes) in order, each with the
//        (metric, value) entries it holds: prof_off -> plane_off -> values.
//   CMS: for every context of the union, its non-empty metrics (the sparse
//        metric index: metric id and start), each with the (profile, value)
//        entries of the profiles that hold it, in profile order.
// PMS is a reformat of the (already sorted) key lists: run heads and scans.
// CMS is a transpose: every key of every profile becomes a record whose sort
// key is (node, stall, profile) within its context -- the profile index
// occupies the lowest key bits -- and the aggregation's grouping, split and
// leaf sort put all records in (context, node, stall, profile) order; flags
// and scans over that order give the planes and the metric index.

#include "hpa_host.h"
#include "hpa_warpagg.cuh"

namespace hpa {

struct SpDesc {
    const uint32_t* ctx;
    const uint32_t* node;
    const uint8_t* stall;
    const uint64_t* val;
    const uint64_t* n_keys;
    uint64_t cap;
    uint64_t base;     // first flattened index
};

struct SpArgs {
    const SpDesc* prof;
    const uint64_t* prof_base;   // [P + 1]
    uint32_t P, pbits;
    uint64_t total;              // sum of capacities
    uint32_t M, n_ctx, sb, n_stall;
    // CMS entries in order, before the flags
    uint32_t* e_ctx;
    uint32_t* e_node;
    uint8_t* e_stall;
    uint32_t* f_key;             // [total + 1] heads -> exclusive scan
    uint32_t* f_plane;           // [total + 1]
    DevStatus* status;
};

__device__ __forceinline__ bool sp_fetch(const SpArgs& A, uint64_t i, uint32_t& p, uint64_t& j) {
    p = upper_index<uint64_t>(A.prof_base, A.P, i);
    j = i - A.prof[p].base;
    return j < min(*A.prof[p].n_keys, A.prof[p].cap);
}

// ---- CMS
// Both passes walk the flattened keys warp by warp (the loop is uniform in
// a warp) and count with warp-aggregated atomics: the profiles are sorted by
// context, so the lanes of a warp mostly share one.
__global__ void k_cms_hist(AggWork w, SpArgs A) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); i0 < A.total; i0 += stride) {
        const uint64_t i = i0 + (threadIdx.x & 31u);
        uint32_t* ctr = nullptr;
        uint32_t p;
        uint64_t j;
        if (i < A.total && sp_fetch(A, i, p, j)) {
            const SpDesc& d = A.prof[p];
            const uint32_t c = d.ctx[j], n = d.node[j];
            if (c >= A.n_ctx || d.stall[j] >= A.n_stall || (n != UNKNOWN && n >= A.M)) atomicAdd(&w.buf_bad[0], 1ull);
            else ctr = &w.grp_hist[c];
        }
        warp_agg_inc(ctr);
    }
}

__global__ void k_cms_scatter(AggWork w, SpArgs A) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); i0 < A.total; i0 += stride) {
        const uint64_t i = i0 + (threadIdx.x & 31u);
        uint32_t* ctr = nullptr;
        uint32_t p = 0, sub = 0;
        uint64_t j = 0;
        if (i < A.total && sp_fetch(A, i, p, j)) {
            const SpDesc& d = A.prof[p];
            const uint32_t c = d.ctx[j], n = d.node[j], r = d.stall[j];
            if (c < A.n_ctx && r < A.n_stall && (n == UNKNOWN || n < A.M)) {
                sub = (((n == UNKNOWN ? A.M : n) << A.sb) | r);
                ctr = &w.grp_cursor[(size_t)c << w.cur_shift];
            }
        }
        const uint32_t slot = warp_agg_inc(ctr);
        if (!ctr) continue;
        w.rec_sub[slot] = (sub << A.pbits) | p;
        w.rec_v64[slot] = A.prof[p].val[j];
    }
}

// leaves -> entries in (context, node, stall, profile) order
__global__ void k_cms_emit(AggWork w, SpArgs A, hpa_cms o) {
    const uint32_t n_leaves = w.item_nleaf[w.G];
    const uint32_t* leaf_out = w.leaf_d;
    const uint32_t kmask = (w.sbits >= 32) ? 0xFFFFFFFFu : ((1u << w.sbits) - 1);
    const uint32_t pmask = (1u << A.pbits) - 1, stmask = (1u << A.sb) - 1;
    for (uint32_t l = blockIdx.x; l < n_leaves; l += gridDim.x) {
        const uint32_t d = leaf_out[l + 1] - leaf_out[l];
        const uint32_t start = w.leaf_start[l], g0 = w.leaf_grp0[l];
        for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
            const uint32_t k = w.tmp_key[start + i];
            const uint32_t gl = (w.sbits >= 32) ? 0u : (k >> w.sbits);
            const uint32_t sk = k & kmask;
            const uint32_t sub = sk >> A.pbits, node = sub >> A.sb;
            const uint64_t pos = (uint64_t)leaf_out[l] + i;
            A.e_ctx[pos] = g0 + gl;
            A.e_node[pos] = node == A.M ? UNKNOWN : node;
            A.e_stall[pos] = (uint8_t)(sub & stmask);
            if (pos < o.cap_values) {
                o.pid[pos] = sk & pmask;
                o.val[pos] = w.tmp_val[start + i];
            }
        }
    }
}

__global__ void k_cms_flags(AggWork w, SpArgs A) {
    const uint64_t T = w.leaf_d[w.item_nleaf[w.G]];
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < A.total; j += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t fk = 0, fp = 0;
        if (j < T) {
            const bool first = j == 0;
            fp = first || A.e_ctx[j] != A.e_ctx[j - 1] || A.e_node[j] != A.e_node[j - 1];
            fk = fp || A.e_stall[j] != A.e_stall[j - 1];
        }
        A.f_key[j] = fk;
        A.f_plane[j] = fp;
    }
}

__global__ void k_cms_fill(AggWork w, SpArgs A, hpa_cms o) {
    const uint64_t T = w.leaf_d[w.item_nleaf[w.G]];
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < T; j += (uint64_t)gridDim.x * blockDim.x) {
        const bool first = j == 0;
        const bool fp = first || A.e_ctx[j] != A.e_ctx[j - 1] || A.e_node[j] != A.e_node[j - 1];
        const bool fk = fp || A.e_stall[j] != A.e_stall[j - 1];
        const uint64_t k = A.f_key[j], pl = A.f_plane[j];
        if (fk && k < o.cap_metrics) {
            o.metric_id[k] = A.e_stall[j];
            o.metric_off[k] = j;
        }
        if (fp && pl < o.cap_planes) {
            o.plane_ctx[pl] = A.e_ctx[j];
            o.plane_node[pl] = A.e_node[j];
            o.plane_off[pl] = k;
        }
    }
}

__global__ void k_cms_finish(AggWork w, SpArgs A, hpa_cms o) {
    const uint64_t T = w.leaf_d[w.item_nleaf[w.G]];
    const uint64_t nk = A.f_key[A.total], np = A.f_plane[A.total];
    o.counts[0] = np; o.counts[1] = nk; o.counts[2] = T;
    if (w.buf_bad[0]) {
        atomicAdd(&A.status->bad, w.buf_bad[0]);
        raise_status(A.status, 3 /* HPA_E_INVALID_SAMPLE */, 0);
    }
    if (np > o.cap_planes || nk > o.cap_metrics || T > o.cap_values) {
        raise_status(A.status, 4 /* HPA_E_CAPACITY */, 0);
        return;
    }
    o.plane_off[np] = nk;
    o.metric_off[nk] = T;
}

// ---- PMS
__global__ void k_pms_flags(SpArgs A) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < A.total; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t p;
        uint64_t j;
        const bool valid = sp_fetch(A, i, p, j);
        uint32_t head = 0;
        if (valid) {
            const SpDesc& d = A.prof[p];
            head = j == 0 || d.ctx[j] != d.ctx[j - 1] || d.node[j] != d.node[j - 1];
        }
        A.f_key[i] = valid;       // value slots
        A.f_plane[i] = head;      // planes
    }
}

__global__ void k_pms_fill(SpArgs A, hpa_pms o) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < A.total; i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t p;
        uint64_t j;
        if (!sp_fetch(A, i, p, j)) continue;
        const SpDesc& d = A.prof[p];
        const uint64_t v = A.f_key[i];
        const bool head = j == 0 || d.ctx[j] != d.ctx[j - 1] || d.node[j] != d.node[j - 1];
        if (v < o.cap_values) {
            o.metric_id[v] = d.stall[j];
            o.val[v] = d.val[j];
        }
        if (head) {
            const uint64_t pl = A.f_plane[i];
            if (pl < o.cap_planes) {
                o.plane_ctx[pl] = d.ctx[j];
                o.plane_node[pl] = d.node[j];
                o.plane_off[pl] = v;
            }
        }
    }
}

__global__ void k_pms_finish(SpArgs A, hpa_pms o) {
    const uint64_t np = A.f_plane[A.total], nv = A.f_key[A.total];
    for (uint32_t p = threadIdx.x; p <= A.P; p += blockDim.x) o.prof_off[p] = A.f_plane[A.prof_base[p]];
    if (threadIdx.x == 0) {
        o.counts[0] = np; o.counts[1] = nv;
        if (np > o.cap_planes || nv > o.cap_values) raise_status(A.status, 4 /* HPA_E_CAPACITY */, 0);
        else o.plane_off[np] = nv;
    }
}

}  // namespace hpa

using namespace hpa;

// common host part: validation, sizes, descriptors in the staging area
static hpa_status sp_setup(hpa_handle* h, const hpa_profile* const* ps, uint32_t P, SpArgs& A, uint64_t& N,
                           uint32_t& G, uint32_t& S, uint32_t& M) {
    if (P == 0) return h->fail(HPA_E_INVALID_ARG, "no profiles");
    N = 0; G = 0; S = 1; M = 0;
    for (uint32_t p = 0; p < P; ++p) {
        const hpa_profile* q = ps[p];
        if (!q || !q->n_keys || (q->capacity && (!q->key_ctx || !q->key_node || !q->key_stall || !q->val)))
            return h->fail(HPA_E_INVALID_ARG, "profile %u arrays missing", p);
        if (q->n_stall == 0 || q->n_stall > HPA_MAX_STALL || q->n_ctx == 0)
            return h->fail(HPA_E_INVALID_ARG, "profile %u has no n_ctx / n_stall", p);
        N += q->capacity;
        G = std::max(G, q->n_ctx);
        S = std::max(S, q->n_stall);
        M = std::max(M, q->n_nodes);
    }
    if (N >= 0xFFFFFFF0ull) return h->fail(HPA_E_INVALID_ARG, "too many keys");
    A.P = P; A.total = N; A.M = M; A.n_ctx = G; A.n_stall = S; A.status = h->d_status;
    return HPA_OK;
}

static hpa_status sp_stage(hpa_handle* h, const hpa_profile* const* ps, uint32_t P, SpArgs& A, uint32_t G,
                           AggWork* w) {
    Carve probe{nullptr};
    probe.take<SpDesc>(P);
    probe.take<uint64_t>(P + 1);
    probe.take<BufDev>(1);
    probe.take<uint64_t>(2);
    probe.take<uint32_t>(2);
    hpa_status st = h->ensure_staging(probe.off + 256);
    if (st) return st;
    Carve hs{(char*)h->staging};
    SpDesc* hp = hs.take<SpDesc>(P);
    uint64_t* hbase = hs.take<uint64_t>(P + 1);
    BufDev* hb = hs.take<BufDev>(1);
    uint64_t* htile = hs.take<uint64_t>(2);
    uint32_t* hgrp = hs.take<uint32_t>(2);
    uint64_t base = 0;
    for (uint32_t p = 0; p < P; ++p) {
        const hpa_profile* q = ps[p];
        hp[p] = SpDesc{q->key_ctx, q->key_node, q->key_stall, q->val, q->n_keys, q->capacity, base};
        hbase[p] = base;
        base += q->capacity;
    }
    hbase[P] = base;
    BufDev d{};
    d.n_ctx = G;
    *hb = d;
    htile[0] = htile[1] = 0;
    hgrp[0] = 0; hgrp[1] = G;
    if ((st = h->upload_staging(hs.off))) return st;
    char* ds = (char*)h->d_staging;
    auto dev = [&](void* hostp) { return ds + ((char*)hostp - (char*)h->staging); };
    A.prof = (const SpDesc*)dev(hp);
    A.prof_base = (const uint64_t*)dev(hbase);
    if (w) {
        w->bufs = (const BufDev*)dev(hb);
        w->buf_tile = (const uint64_t*)dev(htile);
        w->buf_grp = (const uint32_t*)dev(hgrp);
        w->n_tiles = 0;
    }
    return HPA_OK;
}

extern "C" hpa_status hpa_build_cms(hpa_handle* h, const hpa_profile* const* ps, uint32_t n_profiles, hpa_cms* out) {
    hpa::Trace trace_("hpa.build_cms");
    if (!h || !ps || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    if (!out->counts || (out->cap_planes && (!out->plane_ctx || !out->plane_node)) || !out->plane_off ||
        (out->cap_metrics && !out->metric_id) || !out->metric_off || (out->cap_values && (!out->pid || !out->val)))
        return h->fail(HPA_E_INVALID_ARG, "CMS output arrays missing");
    SpArgs A{};
    uint64_t N;
    uint32_t G, S, M;
    hpa_status st = sp_setup(h, ps, n_profiles, A, N, G, S, M);
    if (st) return st;
    const uint32_t sb = ceil_log2_u64(S), nb = ceil_log2_u64((uint64_t)M + 1), pbits = ceil_log2_u64(n_profiles);
    if (nb + sb + pbits > 32)
        return h->fail(HPA_E_INVALID_ARG, "(n_nodes + 1) * 2^stall_bits * 2^profile_bits exceeds 2^32");
    A.sb = sb; A.pbits = pbits;
    AggWork w{};
    uint32_t* flag_scan_tmp = nullptr;     // the flag scans run over N entries, beyond the work's scan buffer
    auto extra = [&](Carve& c) {
        A.e_ctx = c.take<uint32_t>(N + 1);
        A.e_node = c.take<uint32_t>(N + 1);
        A.e_stall = c.take<uint8_t>(N + 1);
        A.f_key = c.take<uint32_t>(N + 1);
        A.f_plane = c.take<uint32_t>(N + 1);
        flag_scan_tmp = c.take<uint32_t>(scan_tmp_words(N));
    };
    if ((st = h->carve_work(w, N, G, 1, LEAF_CAP_SMALL, sb + pbits, nb + sb + pbits, true, true))) return st;
    Carve probe{nullptr};
    probe.off = h->last_carve;
    extra(probe);
    if (probe.off > h->scratch_cap) {
        if ((st = h->ensure_scratch(probe.off + 256))) return st;
        if ((st = h->carve_work(w, N, G, 1, LEAF_CAP_SMALL, sb + pbits, nb + sb + pbits, true, true))) return st;
    }
    Carve c{(char*)h->scratch};
    c.off = h->last_carve;
    extra(c);
    if ((st = sp_stage(h, ps, n_profiles, A, G, &w))) return st;
    cudaStream_t s = h->stream;
    const int blocks = h->sms * 8;
    clear_work(w, s);
    k_cms_hist<<<blocks, 256, 0, s>>>(w, A);
    run_plan(w, s, h->sms, &h->launches, false);
    k_cms_scatter<<<blocks, 256, 0, s>>>(w, A);
    launch_big_partition(w, s, h->sms, &h->launches);
    launch_leaves(w, s, h->sms, &h->launches);
    scan_u32(w.leaf_d, w.leaf_d, w.L_max, w.scan_tmp, s, &h->launches);
    k_cms_emit<<<blocks, 256, 0, s>>>(w, A, *out);
    k_cms_flags<<<blocks, 256, 0, s>>>(w, A);
    scan_u32(A.f_key, A.f_key, N, flag_scan_tmp, s, &h->launches);
    scan_u32(A.f_plane, A.f_plane, N, flag_scan_tmp, s, &h->launches);
    k_cms_fill<<<blocks, 256, 0, s>>>(w, A, *out);
    k_cms_finish<<<1, 1, 0, s>>>(w, A, *out);
    h->launches += 7;
    return h->cuda(cudaGetLastError(), "CMS launch");
}

extern "C" hpa_status hpa_build_pms(hpa_handle* h, const hpa_profile* const* ps, uint32_t n_profiles, hpa_pms* out) {
    hpa::Trace trace_("hpa.build_pms");
    if (!h || !ps || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    if (!out->counts || !out->prof_off || (out->cap_planes && (!out->plane_ctx || !out->plane_node)) ||
        !out->plane_off || (out->cap_values && (!out->metric_id || !out->val)))
        return h->fail(HPA_E_INVALID_ARG, "PMS output arrays missing");
    SpArgs A{};
    uint64_t N;
    uint32_t G, S, M;
    hpa_status st = sp_setup(h, ps, n_profiles, A, N, G, S, M);
    if (st) return st;
    uint32_t* scan_tmp = nullptr;
    auto layout = [&](Carve& c) {
        A.f_key = c.take<uint32_t>(N + 1);
        A.f_plane = c.take<uint32_t>(N + 1);
        scan_tmp = c.take<uint32_t>(scan_tmp_words(N));
    };
    Carve probe{nullptr};
    layout(probe);
    if ((st = h->ensure_scratch(probe.off + 256))) return st;
    Carve c{(char*)h->scratch};
    layout(c);
    if ((st = sp_stage(h, ps, n_profiles, A, G, nullptr))) return st;
    cudaStream_t s = h->stream;
    const int blocks = h->sms * 8;
    k_pms_flags<<<blocks, 256, 0, s>>>(A);
    scan_u32(A.f_key, A.f_key, N, scan_tmp, s, &h->launches);
    scan_u32(A.f_plane, A.f_plane, N, scan_tmp, s, &h->launches);
    k_pms_fill<<<blocks, 256, 0, s>>>(A, *out);
    k_pms_finish<<<1, 256, 0, s>>>(A, *out);
    h->launches += 3;
    return h->cuda(cudaGetLastError(), "PMS launch");
}
