// C ABI of libhpa.so: handles, structure loading and validation, scratch
// management and the launch sequences of every entry point declared in
// include/hpa.h.

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hpa.h"
#include "hpa_internal.h"
#include "hpa_host.h"

using namespace hpa;

// ------------------------------------------------------------------ handle helpers
hpa_status hpa_handle::fail(hpa_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return st;
}

hpa_status hpa_handle::cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return HPA_OK;
    cudaGetLastError();
    return fail(HPA_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool hpa_handle::capturing() const {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

hpa_status hpa_handle::ensure_scratch(size_t bytes) {
    if (bytes <= scratch_cap) return HPA_OK;
    if (capturing())
        return fail(HPA_E_OOM, "scratch of %zu bytes needed during stream capture; call hpa_reserve first", bytes);
    hpa_status st = cuda(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    if (st) return st;
    if (scratch) cudaFree(scratch);
    scratch = nullptr;
    scratch_cap = 0;
    size_t want = bytes + bytes / 8 + (1 << 20);
    if (cudaMalloc(&scratch, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(HPA_E_OOM, "cannot allocate %zu bytes of device scratch", want);
    }
    scratch_cap = want;
    ++scratch_epoch;
    return HPA_OK;
}

hpa_status hpa_handle::ensure_staging(size_t bytes, bool for_graph) {
    const int k = for_graph ? 0 : staging_next;
    if (!for_graph) staging_next = staging_next % (N_STAGING - 1) + 1;
    StagingSlot& sl = stage_slots[k];
    if (!sl.ev && cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess)
        return cuda(cudaGetLastError(), "staging event");
    if (bytes > sl.cap) {
        if (capturing()) return fail(HPA_E_OOM, "descriptor staging must grow during stream capture");
        if (sl.live) cudaEventSynchronize(sl.ev);
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.dev) cudaFree(sl.dev);
        sl.host = nullptr; sl.dev = nullptr; sl.cap = 0; sl.live = false;
        size_t want = std::max<size_t>(bytes, 64 << 10);
        if (cudaMallocHost(&sl.host, want) != cudaSuccess || cudaMalloc(&sl.dev, want) != cudaSuccess) {
            cudaGetLastError();
            if (sl.host) cudaFreeHost(sl.host);
            if (sl.dev) cudaFree(sl.dev);
            sl.host = nullptr; sl.dev = nullptr;
            return fail(HPA_E_OOM, "cannot allocate %zu bytes of descriptor staging", want);
        }
        sl.cap = want;
        if (k == 0) ++scratch_epoch;           // graphs copy from slot 0's buffers
        // the other rotating slots come into being with the first one, so one
        // call prepares them all (for callers that capture later calls)
        for (int j = 1; j < N_STAGING && k != 0; ++j) {
            StagingSlot& o = stage_slots[j];
            if (o.cap || j == k) continue;
            if (!o.ev && cudaEventCreateWithFlags(&o.ev, cudaEventDisableTiming) != cudaSuccess)
                return cuda(cudaGetLastError(), "staging event");
            if (cudaMallocHost(&o.host, want) != cudaSuccess || cudaMalloc(&o.dev, want) != cudaSuccess) {
                cudaGetLastError();
                if (o.host) cudaFreeHost(o.host);
                if (o.dev) cudaFree(o.dev);
                o.host = nullptr; o.dev = nullptr;
                return fail(HPA_E_OOM, "cannot allocate %zu bytes of descriptor staging", want);
            }
            o.cap = want;
        }
    } else if (sl.live) {
        hpa_status st = cuda(cudaEventSynchronize(sl.ev), "cudaEventSynchronize");
        if (st) return st;
    }
    staging_slot = k;
    staging = sl.host;
    d_staging = sl.dev;
    staging_cap = sl.cap;
    return HPA_OK;
}

// upload the staged descriptors; the host must not touch the slot's buffer
// until its event has completed (ensure_staging waits for it)
hpa_status hpa_handle::upload_staging(size_t bytes) {
    hpa_status st = cuda(cudaMemcpyAsync(d_staging, staging, bytes, cudaMemcpyHostToDevice, stream), "upload descriptors");
    if (st) return st;
    StagingSlot& sl = stage_slots[staging_slot];
    st = cuda(cudaEventRecord(sl.ev, stream), "cudaEventRecord");
    sl.live = true;
    return st;
}

Binary* hpa_handle::binary(uint32_t id) {
    if (id >= bins.size() || !bins[id]) return nullptr;
    return bins[id];
}

// ------------------------------------------------------------------ create / destroy
extern "C" hpa_status hpa_create(hpa_handle** out, int device, void* cuda_stream, const hpa_options* opt) {
    if (!out) return HPA_E_INVALID_ARG;
    *out = nullptr;
    if (opt && (opt->leaf_hash > 1 || opt->leaf_emit > 1 || opt->small_leaves > 2 || opt->leaf_ranking > 3 || opt->grouping > 1 ||
                opt->cursor_pad > 7 ||
                (opt->leaf_capacity && opt->leaf_capacity != LEAF_CAP_SMALL && opt->leaf_capacity != LEAF_CAP_LARGE)))
        return HPA_E_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HPA_E_CUDA;
    }
    hpa_handle* h = new hpa_handle();
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    if (opt) h->opt = *opt;
    if (!h->opt.issued_mask) h->opt.issued_mask = 1u;
    if (!h->opt.timeout_iters) h->opt.timeout_iters = 1u << 22;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&h->d_status, sizeof(DevStatus)) != cudaSuccess ||
        cudaMemset(h->d_status, 0, sizeof(DevStatus)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return HPA_E_CUDA;
    }
    *out = h;
    return HPA_OK;
}

hpa_handle::~hpa_handle() {
    cudaStreamSynchronize(stream);
    for (Binary* b : bins) delete b;
    if (scratch) cudaFree(scratch);
    for (StagingSlot& sl : stage_slots) {
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.dev) cudaFree(sl.dev);
        if (sl.ev) cudaEventDestroy(sl.ev);
    }
    if (d_status) cudaFree(d_status);
    if (d_bins) cudaFree(d_bins);
    for (auto& g : graphs) if (g.exec) cudaGraphExecDestroy(g.exec);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    for (int i = 0; i < N_COPY_STREAMS; ++i) {
        if (copy_streams[i]) cudaStreamDestroy(copy_streams[i]);
        if (copy_join[i]) cudaEventDestroy(copy_join[i]);
    }
    if (copy_fork) cudaEventDestroy(copy_fork);
    for (auto& v : ev_pool) for (cudaEvent_t e : v) cudaEventDestroy(e);
    for (auto& v : ev_pending) for (cudaEvent_t e : v) cudaEventDestroy(e);
    if (host_io) cudaFree(host_io);
    if (pinned_io) cudaFreeHost(pinned_io);
    if (cct_scratch) cudaFree(cct_scratch);
    if (aux_scratch) cudaFree(aux_scratch);
}

extern "C" hpa_status hpa_destroy(hpa_handle* h) {
    if (!h) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    delete h;
    return HPA_OK;
}

extern "C" const char* hpa_last_error(hpa_handle* h) { return h ? h->err.c_str() : "null handle"; }

extern "C" uint64_t hpa_kernel_launches(hpa_handle* h) { return h ? h->launches : 0; }

extern "C" uint32_t hpa_build_flags(void) {
#ifdef HPA_CHECKED
    return HPA_BUILD_CHECKED;
#else
    return 0u;
#endif
}

cudaEvent_t* hpa_handle::phase_events(bool new_call) {
    std::vector<cudaEvent_t> v;
    if (!ev_pool.empty()) {
        v = std::move(ev_pool.back());
        ev_pool.pop_back();
    } else {
        v.resize(N_PHASES + 1);
        for (auto& e : v) cudaEventCreate(&e);
    }
    ev_pending.push_back(std::move(v));
    ev_counts.push_back(new_call);
    return ev_pending.back().data();
}

void hpa_handle::collect_phase_times() {
    for (size_t k = 0; k < ev_pending.size(); ++k) {
        auto& v = ev_pending[k];
        for (int i = 0; i < N_PHASES; ++i) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, v[i], v[i + 1]) == cudaSuccess) phase_ms[i] += ms;
            else cudaGetLastError();
        }
        if (ev_counts[k]) ++phase_calls;
        ev_pool.push_back(std::move(v));
    }
    ev_pending.clear();
    ev_counts.clear();
}

extern "C" hpa_status hpa_set_phase_timing(hpa_handle* h, int enable) {
    if (!h) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    h->collect_phase_times();
    h->timing = enable != 0;
    if (enable) {
        for (int i = 0; i < N_PHASES; ++i) h->phase_ms[i] = 0;
        h->phase_calls = 0;
    }
    return HPA_OK;
}

extern "C" hpa_status hpa_phase_times(hpa_handle* h, uint32_t n_max, double* ms, uint64_t* calls, uint32_t* n_phases) {
    if (!h) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    h->collect_phase_times();
    for (uint32_t i = 0; i < n_max && i < (uint32_t)N_PHASES; ++i) if (ms) ms[i] = h->phase_ms[i];
    if (calls) *calls = h->phase_calls;
    if (n_phases) *n_phases = N_PHASES;
    return HPA_OK;
}

extern "C" hpa_status hpa_sync(hpa_handle* h, uint64_t* bad) {
    if (!h) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    hpa_status st = h->cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (st) return st;
    h->collect_phase_times();
    DevStatus ds;
    st = h->cuda(cudaMemcpy(&ds, h->d_status, sizeof ds, cudaMemcpyDeviceToHost), "read device status");
    if (st) return st;
    if (bad) *bad = ds.bad;
    if (ds.code) {
        cudaMemset(h->d_status, 0, sizeof(DevStatus));
        const char* what = ds.code == HPA_E_INVALID_SAMPLE ? "invalid sample records"
                         : ds.code == HPA_E_CAPACITY ? "output capacity too small (n_keys holds the size needed)"
                         : ds.code == HPA_E_TIMEOUT ? "a bounded device wait gave up"
                         : ds.code == HPA_E_INTERNAL ? "internal invariant violated (detail >= 100: the index check that failed)"
                         : "device error";
        return h->fail(ds.code, "%s (detail %d, bad records %llu)", what, ds.where, (unsigned long long)ds.bad);
    }
    return HPA_OK;
}

// ------------------------------------------------------------------ structure
static hpa_status load_binary(hpa_handle* h, const hpa_structure* s, Binary* B);
static hpa_status check_structure(const hpa_structure* s, std::vector<uint32_t>& depth, uint32_t& max_depth,
                                  char* msg, size_t msg_len);

extern "C" hpa_status hpa_validate_structure(const hpa_structure* s, char* msg, size_t msg_len) {
    if (msg && msg_len) msg[0] = 0;
    if (!s) return HPA_E_INVALID_ARG;
    std::vector<uint32_t> depth;
    uint32_t max_depth = 0;
    return check_structure(s, depth, max_depth, msg, msg_len);
}

extern "C" hpa_status hpa_load_structure(hpa_handle* h, const hpa_structure* s, uint32_t* binary_id) {
    hpa::Trace trace_("hpa.load_structure");
    if (!h || !s || !binary_id) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = new Binary();
    hpa_status st = load_binary(h, s, B);
    if (st) { delete B; return st; }
    uint32_t id = 0;
    while (id < h->bins.size() && h->bins[id]) ++id;
    if (id == h->bins.size()) h->bins.push_back(nullptr);
    h->bins[id] = B;
    st = h->refresh_bin_table();
    if (st) { h->bins[id] = nullptr; delete B; return st; }
    *binary_id = id;
    return HPA_OK;
}

extern "C" hpa_status hpa_unload_structure(hpa_handle* h, uint32_t id) {
    if (!h) return HPA_E_INVALID_ARG;
    Binary* B = h->binary(id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", id);
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    delete B;
    h->bins[id] = nullptr;
    return h->refresh_bin_table();
}

hpa_status hpa_handle::refresh_bin_table() {
    std::vector<DevBinary> t(std::max<size_t>(1, bins.size()));
    for (size_t i = 0; i < bins.size(); ++i)
        if (bins[i]) t[i] = bins[i]->dev;
    hpa_status st = cuda(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
    if (st) return st;
    if (t.size() > d_bins_cap) {
        if (d_bins) cudaFree(d_bins);
        d_bins = nullptr;
        if (cudaMalloc(&d_bins, t.size() * sizeof(DevBinary)) != cudaSuccess) {
            cudaGetLastError();
            d_bins_cap = 0;
            return fail(HPA_E_OOM, "binary table");
        }
        d_bins_cap = t.size();
        ++scratch_epoch;
    }
    return cuda(cudaMemcpy(d_bins, t.data(), t.size() * sizeof(DevBinary), cudaMemcpyHostToDevice), "binary table");
}

Binary::~Binary() {
    for (void* p : dev_allocs) cudaFree(p);
}

// Host checks of a structure's tables (no device work): ranges sorted,
// non-empty, disjoint, spanning < 2^32 bytes; FUNC nodes exactly the roots,
// one per function; parents in range, of the same function, acyclic; call
// sites naming existing functions and CALL nodes of the caller.  Fills each
// node's depth.  On failure returns the status with a message in msg.
static hpa_status check_structure(const hpa_structure* s, std::vector<uint32_t>& depth, uint32_t& max_depth,
                                  char* msg, size_t msg_len) {
    auto bad = [&](hpa_status st, const char* fmt, ...) {
        if (msg && msg_len) {
            va_list ap;
            va_start(ap, fmt);
            vsnprintf(msg, msg_len, fmt, ap);
            va_end(ap);
        }
        return st;
    };
    const uint64_t R = s->n_ranges;
    const uint32_t M = s->n_nodes, F = s->n_funcs, E = s->n_calls;
    if (R == 0 || !s->range_lo || !s->range_hi || !s->range_node)
        return bad(HPA_E_INVALID_ARG, "structure needs at least one range");
    if (M == 0 || !s->node_parent || !s->node_kind || !s->node_func)
        return bad(HPA_E_INVALID_ARG, "structure needs node tables");
    if (R >= 0xFFFFFFFFull) return bad(HPA_E_INVALID_TABLE, "too many ranges");
    if (M >= 0x7FFFFFFFu) return bad(HPA_E_INVALID_TABLE, "too many nodes");
    if (E && (!s->cs_caller || !s->cs_callee || !s->cs_node))
        return bad(HPA_E_INVALID_ARG, "call-site tables missing");
    // ranges: sorted, non-empty, disjoint, span < 2^32
    for (uint64_t i = 0; i < R; ++i) {
        if (s->range_hi[i] <= s->range_lo[i])
            return bad(HPA_E_INVALID_TABLE, "range %llu is empty", (unsigned long long)i);
        if (i && s->range_lo[i] < s->range_hi[i - 1])
            return bad(HPA_E_INVALID_TABLE, "range %llu overlaps or is out of order", (unsigned long long)i);
        if (s->range_node[i] >= M)
            return bad(HPA_E_INVALID_TABLE, "range %llu names node %u >= n_nodes", (unsigned long long)i, s->range_node[i]);
    }
    const uint64_t base = s->range_lo[0];
    const uint64_t span = s->range_hi[R - 1] - base;
    if (span >= (1ull << 32)) return bad(HPA_E_INVALID_TABLE, "ranges span %llu bytes (limit 2^32)", (unsigned long long)span);
    // nodes: FUNC exactly the roots, parents of the same function, no cycles
    for (uint32_t v = 0; v < M; ++v) {
        const uint32_t p = s->node_parent[v];
        if (s->node_func[v] >= F) return bad(HPA_E_INVALID_TABLE, "node %u names function %u >= n_funcs", v, s->node_func[v]);
        if (s->node_kind[v] > HPA_NODE_CALL) return bad(HPA_E_INVALID_TABLE, "node %u has kind %u", v, s->node_kind[v]);
        const bool root = p == HPA_NO_PARENT;
        if (root != (s->node_kind[v] == HPA_NODE_FUNC))
            return bad(HPA_E_INVALID_TABLE, "node %u: FUNC nodes must be exactly the roots", v);
        if (!root) {
            if (p >= M) return bad(HPA_E_INVALID_TABLE, "node %u has parent %u >= n_nodes", v, p);
            if (s->node_func[p] != s->node_func[v]) return bad(HPA_E_INVALID_TABLE, "node %u and its parent belong to different functions", v);
        }
    }
    depth.assign(M, 0xFFFFFFFFu);
    std::vector<uint32_t> func_node(F, HPA_NO_PARENT);
    for (uint32_t v = 0; v < M; ++v) {
        if (s->node_parent[v] == HPA_NO_PARENT) {
            if (func_node[s->node_func[v]] != HPA_NO_PARENT)
                return bad(HPA_E_INVALID_TABLE, "function %u has two FUNC nodes", s->node_func[v]);
            func_node[s->node_func[v]] = v;
        }
    }
    max_depth = 0;
    {
        std::vector<uint32_t> path;
        for (uint32_t v = 0; v < M; ++v) {
            path.clear();
            uint32_t x = v;
            while (depth[x] == 0xFFFFFFFFu && s->node_parent[x] != HPA_NO_PARENT) {
                path.push_back(x);
                if (path.size() > M) return bad(HPA_E_INVALID_TABLE, "structure tree has a cycle");
                x = s->node_parent[x];
            }
            if (depth[x] == 0xFFFFFFFFu) depth[x] = 0;
            uint32_t d = depth[x];
            for (size_t i = path.size(); i-- > 0;) depth[path[i]] = ++d;
            max_depth = std::max(max_depth, d);
        }
    }
    // call sites
    for (uint32_t e = 0; e < E; ++e) {
        if (s->cs_caller[e] >= F || s->cs_callee[e] >= F)
            return bad(HPA_E_INVALID_TABLE, "call site %u names a function >= n_funcs", e);
        const uint32_t n = s->cs_node[e];
        if (n >= M || s->node_kind[n] != HPA_NODE_CALL || s->node_func[n] != s->cs_caller[e])
            return bad(HPA_E_INVALID_TABLE, "call site %u: cs_node must be a CALL node of the caller", e);
    }
    return HPA_OK;
}

static hpa_status load_binary(hpa_handle* h, const hpa_structure* s, Binary* B) {
    const uint64_t R = s->n_ranges;
    const uint32_t M = s->n_nodes, F = s->n_funcs, E = s->n_calls;
    std::vector<uint32_t> depth;
    uint32_t max_depth = 0;
    char msg[256] = {0};
    const hpa_status vst = check_structure(s, depth, max_depth, msg, sizeof msg);
    if (vst) return h->fail(vst, "%s", msg);
    const uint64_t base = s->range_lo[0];
    const uint64_t span = s->range_hi[R - 1] - base;
    if (M >= DIR_SEARCH) return h->fail(HPA_E_INVALID_TABLE, "n_nodes must be < 2^31");
    B->n_nodes = M; B->n_funcs = F; B->n_calls = E; B->n_ranges = R; B->max_depth = max_depth;
    // attribution tables: the ranges as entries {lo, node} of offsets from the
    // segment base with each gap between two ranges as an entry of node M
    // (UNKNOWN) and a last entry at the span; and a bucket directory of at
    // most DIR_PER_ENTRY buckets per entry (at least DIR_MIN_ENTRIES, at most
    // DIR_MAX_ENTRIES) of 2^dshift bytes each.  A directory entry answers
    // directly when its bucket lies inside one table entry (that entry's
    // node), otherwise it holds DIR_SEARCH | the entry holding the bucket start.
    std::vector<uint2> ent;
    ent.reserve(R + R / 4 + 2);
    for (uint64_t i = 0; i < R; ++i) {
        ent.push_back(make_uint2((uint32_t)(s->range_lo[i] - base), s->range_node[i]));
        if (i + 1 < R && s->range_hi[i] < s->range_lo[i + 1]) ent.push_back(make_uint2((uint32_t)(s->range_hi[i] - base), M));
    }
    ent.push_back(make_uint2((uint32_t)span, M));
    const uint64_t n_ent = ent.size();
    const uint64_t dir_cap = std::min<uint64_t>(DIR_MAX_ENTRIES, std::max<uint64_t>(DIR_PER_ENTRY * n_ent, DIR_MIN_ENTRIES));
    uint32_t dshift = 4;
    while (dshift < 31 && (span >> dshift) + 1 > dir_cap) ++dshift;
    const uint64_t n_dir = (span >> dshift) + 1;
    std::vector<uint32_t> dir(n_dir + 1);
    {
        uint64_t j = 0;
        for (uint64_t b = 0; b <= n_dir; ++b) {
            const uint64_t start = b << dshift, end = start + (1ull << dshift);
            if (start >= span) { dir[b] = M; continue; }
            while (j + 1 < n_ent && ent[j + 1].x <= start) ++j;
            dir[b] = (ent[j + 1].x >= end) ? ent[j].y : (DIR_SEARCH | (uint32_t)j);
        }
    }
    hpa_status st;
    uint2* d_ent; uint32_t* d_dir;
    if ((st = upload(h, B, ent, &d_ent)) || (st = upload(h, B, dir, &d_dir))) return st;
    B->dev.pc_base = base;
    B->dev.span = span;
    B->dev.dshift = dshift;
    B->dev.n_dir = (uint32_t)n_dir;
    B->dev.n_ent = (uint32_t)n_ent;
    B->dev.n_nodes = M;
    B->dev.dir = d_dir;
    B->dev.ent = d_ent;
    // host copies kept for the other analyses
    B->node_parent.assign(s->node_parent, s->node_parent + M);
    B->node_kind.assign(s->node_kind, s->node_kind + M);
    B->node_func.assign(s->node_func, s->node_func + M);
    B->node_depth = depth;
    if (E) {
        B->cs_caller.assign(s->cs_caller, s->cs_caller + E);
        B->cs_callee.assign(s->cs_callee, s->cs_callee + E);
        B->cs_node.assign(s->cs_node, s->cs_node + E);
    }
    return build_callgraph(h, B);
}

extern "C" hpa_status hpa_binary_info_get(hpa_handle* h, uint32_t id, hpa_binary_info* info, uint32_t* cnode_of_func) {
    if (!h) return HPA_E_INVALID_ARG;
    Binary* B = h->binary(id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", id);
    if (info) {
        info->n_nodes = B->n_nodes; info->n_funcs = B->n_funcs; info->n_calls = B->n_calls;
        info->n_cnodes = B->n_cnodes; info->n_scc = B->n_scc; info->cdag_levels = B->cdag_levels;
        info->n_ranges = B->n_ranges;
        info->max_depth = B->max_depth;
        info->reserved = 0;
    }
    if (cnode_of_func) std::copy(B->cnode_of_func.begin(), B->cnode_of_func.end(), cnode_of_func);
    return HPA_OK;
}

// ------------------------------------------------------------------ aggregation calls
// Scratch layout of one aggregation over N records in G groups (n_buf buffers).
hpa_status hpa_handle::carve_work(AggWork& w, uint64_t N, uint64_t G, uint32_t n, uint32_t cap, uint32_t sb,
                                  uint32_t sbits, bool has_cnt, bool val64, uint64_t staged, uint64_t cnt_words,
                                  uint64_t seg_words, uint64_t cnt2_words) {
    const uint64_t N2 = std::max(N, staged);   // the second record buffer also stages samples in tile order
    const uint64_t L_max = G + 6 * (N / cap + 1) + n + 8;   // items + sub-bins of big groups
    w.G = (uint32_t)G; w.n_buf = n; w.cap = cap; w.q = cap / 2; w.sb = sb; w.sbits = sbits;
    w.span_log = std::min<uint32_t>(10, 32 - sbits);
    // scatter cursors padded to 2^cur_shift words; by default only while the
    // padded cursors take at most 2 MB (beyond that they crowd L2 instead)
    w.cur_shift = opt.cursor_pad ? std::min<uint32_t>(opt.cursor_pad - 1, 6) : (G <= 65536 ? 3 : 0);
    if (((G + 1) << w.cur_shift) > (64ull << 20)) w.cur_shift = 0;
    w.sort_mode = std::min<uint32_t>(opt.leaf_ranking, 3);
    w.L_max = (uint32_t)L_max; w.has_cnt = has_cnt || val64; w.val64 = val64;
    w.n_rec = N;
    auto layout = [&](Carve& c) {
        w.grp_hist = c.take<uint32_t>(G + 1);
        w.grp_cursor = c.take<uint32_t>((G + 1) << w.cur_shift);
        w.item_id = c.take<uint32_t>(G + 1);
        w.item_grp0 = c.take<uint32_t>(G + 1);
        w.item_nleaf = c.take<uint32_t>(G + 1);
        w.leaf_start = c.take<uint32_t>(L_max);
        w.leaf_end = c.take<uint32_t>(L_max);
        w.leaf_grp0 = c.take<uint32_t>(L_max);
        w.leaf_info = c.take<uint32_t>(L_max);
        w.leaf_d = c.take<uint32_t>(L_max + 1);
        w.leaf_look = c.take<unsigned long long>(L_max);
        w.leaf_ticket = c.take<uint32_t>(1);
        w.buf_first_leaf = c.take<uint32_t>(n + 1);
        w.buf_bad = c.take<unsigned long long>(n);
        const bool pair = has_cnt && !val64;
        w.rec_sub = pair ? nullptr : c.take<uint32_t>(N + 1);
        w.rec_cnt = nullptr;
        w.rec2_sub = pair ? nullptr : c.take<uint32_t>(N2 + 1);
        w.rec2_cnt = nullptr;
        w.rec_pair = pair ? c.take<uint2>(N + 1) : nullptr;
        w.rec2_pair = pair ? c.take<uint2>(N2 + 1) : nullptr;
        w.rec_v64 = val64 ? c.take<uint64_t>(N + 1) : nullptr;
        w.rec2_v64 = val64 ? c.take<uint64_t>(N + 1) : nullptr;
        w.tmp_key = c.take<uint32_t>(N + 1);
        w.tmp_val = c.take<uint64_t>(N + 1);
        w.part_cnt = cnt_words ? c.take<uint32_t>(cnt_words) : nullptr;
        w.seg_chunk = seg_words ? c.take<uint32_t>(seg_words) : nullptr;
        w.cnt2 = cnt2_words ? c.take<uint32_t>(cnt2_words) : nullptr;
        w.rec2_dig = seg_words ? c.take<uint8_t>(N + 16) : nullptr;
        w.scan_tmp = c.take<uint32_t>(scan_tmp_words(
            std::max<uint64_t>(std::max<uint64_t>(G, L_max), std::max(std::max(cnt_words, seg_words), cnt2_words))));
    };
    Carve probe{nullptr};
    layout(probe);
    hpa_status st = ensure_scratch(probe.off + 256);
    if (st) return st;
    Carve real{(char*)scratch};
    layout(real);
    last_carve = real.off;
    w.bins = d_bins;
    w.status = d_status;
    return HPA_OK;
}

// Calls whose groups (contexts summed over the buffers) exceed SUB_GROUPS run
// as consecutive sub-batches of whole buffers, one pipeline after another on
// the same scratch, so that the per-group arrays of a sub-batch stay in L2.
constexpr uint64_t SUB_GROUPS = 1ull << 20;

hpa_status hpa_handle::aggregate(uint32_t n, const uint32_t* binary_ids, const hpa_samples* in, hpa_profile* outs,
                                 bool use_graph) {
    if (n == 0) return HPA_OK;
    uint64_t N = 0, G = 0;
    uint32_t max_stall = 1;
    bool has_cnt = false;
    for (uint32_t b = 0; b < n; ++b) {
        const hpa_samples& s = in[b];
        Binary* B = binary(binary_ids[b]);
        if (!B) return fail(HPA_E_INVALID_ARG, "buffer %u: no binary %u", b, binary_ids[b]);
        if (s.n_ctx == 0) return fail(HPA_E_INVALID_ARG, "buffer %u: n_ctx must be >= 1", b);
        if (s.n_stall == 0 || s.n_stall > HPA_MAX_STALL)
            return fail(HPA_E_INVALID_ARG, "buffer %u: n_stall must be in [1, %u]", b, HPA_MAX_STALL);
        if (s.n && (!s.pc || !s.ctx || !s.stall)) return fail(HPA_E_INVALID_ARG, "buffer %u: null sample array", b);
        hpa_profile& o = outs[b];
        if (!o.n_keys || (o.capacity && (!o.key_ctx || !o.key_node || !o.key_stall || !o.val)))
            return fail(HPA_E_INVALID_ARG, "buffer %u: output arrays missing", b);
        N += s.n;
        G += s.n_ctx;
        max_stall = std::max(max_stall, s.n_stall);
        has_cnt |= s.count != nullptr;
    }
    if (N >= 0xFFFFFFF0ull) return fail(HPA_E_INVALID_ARG, "too many samples in one call (%llu)", (unsigned long long)N);
    if (G >= 0xFFFFFFF0ull) return fail(HPA_E_INVALID_ARG, "too many contexts in one call");
    const uint32_t sb = ceil_log2_u64(max_stall);
    if (opt.leaf_capacity && opt.leaf_capacity != LEAF_CAP_SMALL && opt.leaf_capacity != LEAF_CAP_LARGE)
        return fail(HPA_E_INVALID_ARG, "leaf_capacity must be 0, %u or %u", LEAF_CAP_SMALL, LEAF_CAP_LARGE);

    // sub-batches and their configurations
    struct Sub {
        uint32_t b0 = 0, b1 = 0, sbits = 0, cap = 0, ctx_max = 0;
        uint64_t N = 0, G = 0, tiles = 0, part_len = 0, n_parts = 0, n_cnt = 0, n_seg = 0, n_cnt2 = 0;
        uint32_t max_nodes = 0, mode = 0, shift = 0, nbin_max = 0;
    };
    std::vector<Sub> subs;
    for (uint32_t b = 0; b < n; ++b) {
        if (subs.empty() || (subs.back().G + in[b].n_ctx > SUB_GROUPS && subs.back().b1 > subs.back().b0)) {
            subs.emplace_back();
            subs.back().b0 = subs.back().b1 = b;
        }
        Sub& u = subs.back();
        u.b1 = b + 1;
        u.N += in[b].n;
        u.G += in[b].n_ctx;
        u.tiles += (in[b].n + TILE - 1) / TILE;
        u.max_nodes = std::max(u.max_nodes, binary(binary_ids[b])->n_nodes);
        u.ctx_max = std::max(u.ctx_max, in[b].n_ctx);
    }
    uint64_t N_max = 0, G_max = 0, staged_max = 0, cnt_words_max = 0, seg_words_max = 0, cnt2_words_max = 0;
    uint32_t n_max = 0, sbits_max = 0, cap_min = LEAF_CAP_LARGE;
    const uint64_t target_parts = (uint64_t)sms * 8;
    for (Sub& u : subs) {
        const uint32_t nb = ceil_log2_u64((uint64_t)u.max_nodes + 1);
        if (nb + sb > 32) return fail(HPA_E_INVALID_ARG, "(n_nodes + 1) * 2^stall_bits exceeds 2^32");
        u.sbits = nb + sb;
        u.cap = opt.leaf_capacity ? opt.leaf_capacity
                                  : ((u.G && u.N / u.G >= LEAF_CAP_SMALL / 2) ? LEAF_CAP_LARGE : LEAF_CAP_SMALL);
        // partition paths (no global atomics): bins = contexts when every
        // buffer has at most PART_CTX_MAX of them (mode 1), buckets of
        // 2^shift contexts and a second pass up to PART2_CTX_MAX (mode 2),
        // else per-context cursors (mode 0); parts of part_len samples,
        // about 8 per SM over the sub-batch
        u.part_len = std::max<uint64_t>(TILE, (u.N + target_parts - 1) / target_parts + TILE - 1) / TILE * TILE;
        if (opt.grouping != 1) u.mode = u.ctx_max <= PART_CTX_MAX ? 1 : (u.ctx_max <= PART2_CTX_MAX ? 2 : 0);
        u.shift = u.mode == 2 ? ceil_log2_u64(u.ctx_max) - 8 : 0;
        for (uint32_t b = u.b0; b < u.b1; ++b) {
            const uint64_t pb = (in[b].n + u.part_len - 1) / u.part_len;
            const uint32_t nbin = (in[b].n_ctx + (1u << u.shift) - 1) >> u.shift;
            u.n_parts += pb;
            u.n_cnt += pb * nbin;
            u.n_seg += nbin;
            u.nbin_max = std::max(u.nbin_max, nbin);
        }
        if (u.n_cnt > PART_CNT_MAX) u.mode = 0;
        if (u.mode == 2) u.n_cnt2 = (u.N / PART2_LEN + u.n_seg + 1) << u.shift;
        N_max = std::max(N_max, u.N);
        G_max = std::max(G_max, u.G);
        n_max = std::max(n_max, u.b1 - u.b0);
        sbits_max = std::max(sbits_max, u.sbits);
        cap_min = std::min(cap_min, u.cap);
        staged_max = std::max(staged_max, u.mode ? 0 : u.tiles * TILE);
        cnt_words_max = std::max(cnt_words_max, u.mode ? u.n_cnt + 1 : 0);
        seg_words_max = std::max(seg_words_max, u.mode == 2 ? u.n_seg + 2 : 0);
        cnt2_words_max = std::max(cnt2_words_max, u.mode == 2 ? u.n_cnt2 + 1 : 0);
    }
    AggWork w0{};
    hpa_status st = carve_work(w0, N_max, G_max, n_max, cap_min, sb, sbits_max, has_cnt, false, staged_max,
                               cnt_words_max, seg_words_max, cnt2_words_max);
    if (st) return st;

    // descriptors: every buffer's BufDev, then per sub-batch its prefix arrays
    // exact size of the layout below (every take is 256-byte aligned)
    Carve probe{nullptr};
    probe.take<BufDev>(n);
    for (const Sub& u : subs) {
        probe.take<uint64_t>(u.b1 - u.b0 + 1);
        probe.take<uint32_t>(u.b1 - u.b0 + 1);
        probe.take<uint64_t>(u.b1 - u.b0 + 1);
        probe.take<uint32_t>(u.b1 - u.b0 + 1);
    }
    const size_t desc_bytes = probe.off + 256;
    if ((st = ensure_staging(desc_bytes, use_graph && !timing))) return st;
    Carve hs{(char*)staging};
    BufDev* hb = hs.take<BufDev>(n);
    char* ds = (char*)d_staging;
    auto dev_of = [&](const void* p) { return ds + ((const char*)p - (const char*)staging); };
    std::vector<AggWork> ws;
    for (const Sub& u : subs) {
        const uint32_t nk = u.b1 - u.b0;
        uint64_t* htile = hs.take<uint64_t>(nk + 1);
        uint32_t* hgrp = hs.take<uint32_t>(nk + 1);
        uint64_t* hpart = hs.take<uint64_t>(nk + 1);
        uint32_t* hseg = hs.take<uint32_t>(nk + 1);
        uint64_t tb = 0, pbase = 0, cbase = 0;
        uint32_t gb = 0, sgb = 0;
        for (uint32_t b = u.b0; b < u.b1; ++b) {
            const uint32_t k = b - u.b0;
            const hpa_samples& s = in[b];
            hpa_profile& o = outs[b];
            BufDev d{};
            d.pc = s.pc; d.ctx = s.ctx; d.stall = s.stall; d.count = s.count; d.n = s.n;
            d.tile_base = tb; d.n_ctx = s.n_ctx; d.n_stall = s.n_stall; d.grp_base = gb; d.bin = binary_ids[b];
            d.part_base = pbase; d.cnt_base = cbase; d.seg_base = sgb;
            d.total = o.total; d.unknown = o.unknown;
            d.key_ctx = o.key_ctx; d.key_node = o.key_node; d.key_stall = o.key_stall; d.val = o.val;
            d.n_keys = o.n_keys; d.capacity = o.capacity;
            hb[b] = d;
            htile[k] = tb;
            hgrp[k] = gb;
            hpart[k] = pbase;
            hseg[k] = sgb;
            const uint64_t pb = (s.n + u.part_len - 1) / u.part_len;
            const uint32_t nbin = (s.n_ctx + (1u << u.shift) - 1) >> u.shift;
            pbase += pb;
            cbase += pb * nbin;
            sgb += nbin;
            tb += (s.n + TILE - 1) / TILE;
            gb += s.n_ctx;
            o.n_ctx = s.n_ctx;
            o.n_stall = s.n_stall;
            o.n_nodes = binary(binary_ids[b])->n_nodes;
        }
        htile[nk] = tb;
        hgrp[nk] = gb;
        hpart[nk] = pbase;
        hseg[nk] = sgb;
        AggWork w = w0;
        w.G = (uint32_t)u.G;
        w.n_buf = nk;
        w.cap = u.cap;
        w.q = u.cap / 2;
        w.sbits = u.sbits;
        w.span_log = std::min<uint32_t>(10, 32 - u.sbits);
        w.n_tiles = u.tiles;
        w.emit_totals = 1;
        w.timeout_iters = opt.timeout_iters;
        w.small_leaves = opt.small_leaves == 2 || (opt.small_leaves == 0 && u.N < 64 * u.G);
        w.leaf_hash = opt.leaf_hash;
        w.emit_separate = opt.leaf_emit == 0 ? 1u : 0u;
        if (u.mode) {
            w.part_mode = u.mode;
            w.part_ctx_max = u.nbin_max;
            w.part_shift = u.shift;
            w.part_len = u.part_len;
            w.n_parts = u.n_parts;
            w.n_cnt = u.n_cnt;
            w.n_seg = (uint32_t)u.n_seg;
            w.n_cnt2 = u.n_cnt2;
        }
        w.bufs = (const BufDev*)dev_of(hb + u.b0);
        w.buf_tile = (const uint64_t*)dev_of(htile);
        w.buf_grp = (const uint32_t*)dev_of(hgrp);
        w.buf_part = (const uint64_t*)dev_of(hpart);
        w.buf_seg = (const uint32_t*)dev_of(hseg);
        ws.push_back(w);
    }
    const size_t used = hs.off;
    if (used > desc_bytes) return fail(HPA_E_INTERNAL, "descriptor layout overflows its staging area");
    if (use_graph && !timing) return launch_graph(ws, used, n, in);
    if ((st = upload_staging(used))) return st;
    // (each sub-batch's first kernel zeroes its buffers' totals)
    for (size_t k = 0; k < ws.size(); ++k)
        run_aggregate(ws[k], stream, sms, &launches, timing ? phase_events(k == 0) : nullptr);
    return cuda(cudaGetLastError(), "aggregation launch");
}

// One CUDA graph per batch shape: the descriptor upload (from the pinned
// staging area, rewritten before every replay) and every kernel of the
// pipeline (the first of which zeroes the totals).  User pointers reach the kernels only
// through the uploaded descriptors, so a replay serves new buffers of the
// same shape.
static uint64_t mix64(uint64_t h, uint64_t v) {
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return h;
}

hpa_status hpa_handle::launch_graph(const std::vector<AggWork>& ws, size_t staged_bytes, uint32_t n,
                                    const hpa_samples* in) {
    uint64_t key = mix64(0, ws.size());
    for (const AggWork& w : ws) {
        key = mix64(key, w.G); key = mix64(key, w.n_buf); key = mix64(key, w.n_tiles); key = mix64(key, w.cap);
        key = mix64(key, w.sb); key = mix64(key, w.sbits); key = mix64(key, w.L_max); key = mix64(key, w.has_cnt);
        key = mix64(key, w.cur_shift); key = mix64(key, (uint64_t)(uintptr_t)w.grp_hist);
        key = mix64(key, w.part_mode); key = mix64(key, w.part_len); key = mix64(key, w.n_parts);
        key = mix64(key, w.part_shift);
        key = mix64(key, w.sort_mode); key = mix64(key, w.small_leaves); key = mix64(key, w.leaf_hash);
    }
    key = mix64(key, staged_bytes);
    for (uint32_t b = 0; b < n; ++b) key = mix64(mix64(key, in[b].n), in[b].n_ctx);
    CachedGraph* g = nullptr;
    for (auto& c : graphs)
        if (c.key == key && c.epoch == scratch_epoch) g = &c;
    hpa_status st;
    if (!g) {
        if (!capture_stream && cudaStreamCreateWithFlags(&capture_stream, cudaStreamNonBlocking) != cudaSuccess)
            return cuda(cudaGetLastError(), "capture stream");
        cudaGraph_t graph = nullptr;
        uint64_t k0 = launches;
        if ((st = cuda(cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeRelaxed), "begin capture"))) return st;
        cudaMemcpyAsync(d_staging, staging, staged_bytes, cudaMemcpyHostToDevice, capture_stream);
        for (const AggWork& w : ws) run_aggregate(w, capture_stream, sms, &launches, nullptr);
        cudaError_t e = cudaStreamEndCapture(capture_stream, &graph);
        if ((st = cuda(e, "end capture"))) return st;
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if ((st = cuda(e, "graph instantiate"))) return st;
        if (graphs.size() >= 16) {
            cudaGraphExecDestroy(graphs.front().exec);
            graphs.erase(graphs.begin());
        }
        graphs.push_back(CachedGraph{key, scratch_epoch, launches - k0, exec});
        launches = k0;
        g = &graphs.back();
    }
    if ((st = cuda(cudaGraphLaunch(g->exec, stream), "graph launch"))) return st;
    launches += g->kernels;
    ++graph_replays;
    StagingSlot& sl = stage_slots[staging_slot];
    st = cuda(cudaEventRecord(sl.ev, stream), "cudaEventRecord");
    sl.live = true;
    return st;
}

// A call with the shape of the call before it (binary, samples, contexts,
// stall reasons, counts or not) replays a captured CUDA graph of the whole
// pipeline (cached per shape, as for batches): repeated calls on buffers of
// one size then pay neither the host's launches nor their gaps.  A call of a
// new shape runs kernel by kernel, so sizes that change from call to call
// never pay for a capture.
extern "C" hpa_status hpa_attribute_samples(hpa_handle* h, uint32_t binary_id, const hpa_samples* in, hpa_profile* out) {
    hpa::Trace trace_("hpa.attribute_samples");
    if (!h || !in || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    uint64_t shape = mix64(mix64(mix64(0x5EEDull, binary_id), in->n), in->n_ctx);
    shape = mix64(mix64(shape, in->n_stall), in->count ? 1u : 0u);
    const bool repeat = shape == h->last_plain_shape && !h->capturing();
    h->last_plain_shape = shape;
    return h->aggregate(1, &binary_id, in, out, repeat);
}

// every buffer of the call in one captured CUDA graph (cached per batch shape)
extern "C" hpa_status hpa_attribute_batch(hpa_handle* h, uint32_t n, const uint32_t* ids, const hpa_samples* in,
                                          hpa_profile* outs) {
    hpa::Trace trace_("hpa.attribute_batch");
    if (!h || (n && (!ids || !in || !outs))) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    return h->aggregate(n, ids, in, outs, true);
}

extern "C" hpa_status hpa_reserve(hpa_handle* h, uint64_t max_samples, uint64_t max_groups) {
    if (!h) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    const uint64_t N = max_samples, G = max_groups;
    const uint64_t L = G + 6 * (N / LEAF_CAP_SMALL + 1) + 300;
    const uint64_t C = std::min<uint64_t>(PART_CNT_MAX, G * ((uint64_t)h->sms * 8 + 2));   // part counters
    size_t bytes = (G + 1) * 4 * 12 + L * 4 * 5 + (N + TILE + 1) * (4 * 6 + 8) + 256 * 40 + (C + 1) * 4 +
                   scan_tmp_words(std::max(std::max(G, L), C)) * 4 + N + (64ull << 20);   // two-level partition
    return h->ensure_scratch(bytes + (1 << 20));
}

// Host <-> device copies in chunks of 64 MB, round-robin over the copy
// streams, ordered after the work already on the handle's stream and joined
// back into it: several copy engines move one call's arrays at once.
hpa_status hpa_handle::copies(const Copy* c, int n, cudaMemcpyKind kind) {
    if (!copy_fork) {
        if (cudaEventCreateWithFlags(&copy_fork, cudaEventDisableTiming) != cudaSuccess)
            return cuda(cudaGetLastError(), "copy event");
        for (int i = 0; i < N_COPY_STREAMS; ++i)
            if (cudaStreamCreateWithFlags(&copy_streams[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&copy_join[i], cudaEventDisableTiming) != cudaSuccess)
                return cuda(cudaGetLastError(), "copy streams");
    }
    hpa_status st;
    if ((st = cuda(cudaEventRecord(copy_fork, stream), "cudaEventRecord"))) return st;
    for (int i = 0; i < N_COPY_STREAMS; ++i)
        if ((st = cuda(cudaStreamWaitEvent(copy_streams[i], copy_fork, 0), "cudaStreamWaitEvent"))) return st;
    constexpr size_t CHUNK = 64ull << 20;
    int k = 0;
    for (int j = 0; j < n; ++j)
        for (size_t off = 0; off < c[j].bytes; off += CHUNK, ++k) {
            const size_t b = std::min(CHUNK, c[j].bytes - off);
            if ((st = cuda(cudaMemcpyAsync((char*)c[j].dst + off, (const char*)c[j].src + off, b, kind,
                                           copy_streams[k % N_COPY_STREAMS]), "cudaMemcpyAsync")))
                return st;
        }
    for (int i = 0; i < N_COPY_STREAMS; ++i) {
        if ((st = cuda(cudaEventRecord(copy_join[i], copy_streams[i]), "cudaEventRecord"))) return st;
        if ((st = cuda(cudaStreamWaitEvent(stream, copy_join[i], 0), "cudaStreamWaitEvent"))) return st;
    }
    return HPA_OK;
}

extern "C" hpa_status hpa_attribute_samples_host(hpa_handle* h, uint32_t binary_id, const hpa_samples* in,
                                                 hpa_profile* out) {
    hpa::Trace trace_("hpa.attribute_samples_host");
    if (!h || !in || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    const uint64_t n = in->n;
    const bool cnt = in->count != nullptr;
    // device copies of the inputs and outputs, kept by the handle
    const size_t out_cap = out->capacity;
    auto layout = [&](Carve& c, hpa_samples& di, hpa_profile& d) {
        di = *in;
        di.pc = c.take<uint64_t>(n);
        di.ctx = c.take<uint32_t>(n);
        di.stall = c.take<uint8_t>(n);
        di.count = cnt ? c.take<uint32_t>(n) : nullptr;
        d = *out;
        d.key_ctx = c.take<uint32_t>(out_cap);
        d.key_node = c.take<uint32_t>(out_cap);
        d.key_stall = c.take<uint8_t>(out_cap);
        d.val = c.take<uint64_t>(out_cap);
        d.n_keys = c.take<uint64_t>(1);
        d.total = out->total ? c.take<uint64_t>(HPA_MAX_STALL) : nullptr;
        d.unknown = out->unknown ? c.take<uint64_t>(HPA_MAX_STALL) : nullptr;
    };
    hpa_samples di;
    hpa_profile d;
    Carve probe{nullptr};
    layout(probe, di, d);
    const size_t need = probe.off + 256;
    hpa_status st;
    if (need > h->host_io_cap) {
        if ((st = h->cuda(cudaStreamSynchronize(h->stream), "sync"))) return st;
        if (h->host_io) cudaFree(h->host_io);
        h->host_io = nullptr;
        h->host_io_cap = 0;
        if (cudaMalloc(&h->host_io, need) != cudaSuccess) {
            cudaGetLastError();
            return h->fail(HPA_E_OOM, "host-call buffers of %zu bytes", need);
        }
        h->host_io_cap = need;
    }
    Carve c{(char*)h->host_io};
    layout(c, di, d);
    uint64_t* pc = (uint64_t*)di.pc;
    uint32_t* ctx = (uint32_t*)di.ctx;
    uint8_t* stall = (uint8_t*)di.stall;
    uint32_t* count = (uint32_t*)di.count;
    cudaStream_t s = h->stream;
    const hpa_handle::Copy cin[4] = {{pc, in->pc, n * 8}, {ctx, in->ctx, n * 4}, {stall, in->stall, n},
                                     {count, in->count, cnt ? n * 4 : 0}};
    if ((st = h->copies(cin, 4, cudaMemcpyHostToDevice))) return st;
    if ((st = h->aggregate(1, &binary_id, &di, &d))) return st;
    uint64_t K = 0;
    if ((st = h->cuda(cudaMemcpyAsync(&K, d.n_keys, 8, cudaMemcpyDeviceToHost, s), "D2H n_keys")) ||
        (st = h->cuda(cudaStreamSynchronize(s), "sync")))
        return st;
    const uint64_t k = std::min<uint64_t>(K, out_cap);
    if (k) {
        const hpa_handle::Copy cout[4] = {{out->key_ctx, d.key_ctx, k * 4}, {out->key_node, d.key_node, k * 4},
                                          {out->key_stall, d.key_stall, k}, {out->val, d.val, k * 8}};
        if ((st = h->copies(cout, 4, cudaMemcpyDeviceToHost))) return st;
    }
    if (out->total) cudaMemcpyAsync(out->total, d.total, 8 * in->n_stall, cudaMemcpyDeviceToHost, s);
    if (out->unknown) cudaMemcpyAsync(out->unknown, d.unknown, 8 * in->n_stall, cudaMemcpyDeviceToHost, s);
    *out->n_keys = K;
    out->n_ctx = d.n_ctx;
    out->n_stall = d.n_stall;
    out->n_nodes = d.n_nodes;
    return hpa_sync(h, nullptr);
}

namespace hpa {

// polls with a sleep between reads; records a timeout instead of spinning on
__global__ void k_wait_flag(const uint32_t* flag, uint32_t value, uint32_t limit, DevStatus* st) {
    const volatile uint32_t* f = flag;
    for (uint32_t it = 0; it < limit; ++it) {
        if (*f == value) return;
        __nanosleep(1000);
    }
    raise_status(st, 7 /* HPA_E_TIMEOUT */, 0);
}

}  // namespace hpa

extern "C" hpa_status hpa_wait_flag(hpa_handle* h, const uint32_t* flag, uint32_t value) {
    if (!h || !flag) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    hpa::k_wait_flag<<<1, 1, 0, h->stream>>>(flag, value, h->opt.timeout_iters, h->d_status);
    h->launches += 1;
    return h->cuda(cudaGetLastError(), "wait launch");
}
