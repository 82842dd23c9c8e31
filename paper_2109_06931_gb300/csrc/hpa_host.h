// Host-side state of libhpa: the handle and loaded binaries.
#pragma once

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "hpa.h"
#include "hpa_internal.h"

namespace hpa {

// An NVTX range around a library call (named "hpa.<call>"), so that traces
// taken with Nsight tools show the library's calls over its kernels; without
// a tool attached the calls are no-ops.
struct Trace {
    explicit Trace(const char* name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace&) = delete;
    Trace& operator=(const Trace&) = delete;
};

// Device tables of a binary's static call graph (Section 6.3 steps 1 and 3),
// shared by every context.
struct DevCallGraph {
    uint32_t F, E, V, n_levels, M;
    const uint32_t* node_func;   // [M]
    const uint32_t* node_cs;     // [M] call site of a CALL node, else 0xFFFFFFFF
    const uint32_t* cs_caller;   // [E]
    const uint32_t* cs_callee;   // [E]
    const uint32_t* cnode_of_func;  // [F]
    const uint32_t* fin_off;     // [F+1] in-edges of each function (original graph)
    const uint32_t* fin_edge;    // [E]
    const uint32_t* cin_off;     // [V+1] external in-edges of each condensed node
    const uint32_t* cin_edge;
    const uint32_t* cout_off;    // [V+1] external out-edges of each condensed node
    const uint32_t* cout_edge;
    const uint32_t* cout_head;   // condensed callee of each cout_edge entry
    const uint32_t* level_off;   // [n_levels+1] condensed nodes by height (sinks first)
    const uint32_t* level_node;
    const uint8_t* edge_intra;   // [E] 1 if the edge lies inside one SCC
    const uint8_t* cnode_live;   // [V] 0 for rows of functions inside a non-trivial SCC
    const uint32_t* cs_head;     // [E] condensed node of each call site's callee
    const uint32_t* level_of;    // [V] level (height) of each live condensed node
};

struct Binary {
    DevBinary dev{};
    DevCallGraph cg{};
    std::vector<void*> dev_allocs;
    uint32_t n_nodes = 0, n_funcs = 0, n_calls = 0, max_depth = 0;
    uint64_t n_ranges = 0;
    std::vector<uint32_t> node_parent, node_func, node_depth;
    std::vector<uint8_t> node_kind;
    std::vector<uint32_t> cs_caller, cs_callee, cs_node;
    uint32_t n_cnodes = 0, n_scc = 0, cdag_levels = 0;
    std::vector<uint32_t> cnode_of_func;
    const uint32_t* d_node_parent = nullptr;   // structure tree on the device
    const uint32_t* d_node_depth = nullptr;
    ~Binary();
};

// Bump allocator over a scratch arena (base null: only measures the size).
struct Carve {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
};

struct CachedGraph {
    uint64_t key = 0;
    uint64_t epoch = 0;
    uint64_t kernels = 0;       // kernels one replay launches
    cudaGraphExec_t exec = nullptr;
};

}  // namespace hpa

struct hpa_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    hpa_options opt{};
    std::string err;
    int sms = 0;
    hpa::DevStatus* d_status = nullptr;
    std::vector<hpa::Binary*> bins;
    hpa::DevBinary* d_bins = nullptr;
    size_t d_bins_cap = 0;
    void* scratch = nullptr;
    size_t scratch_cap = 0;
    uint64_t scratch_epoch = 0;
    // Descriptor staging: pinned host buffers and their device copies.  Slot 0
    // serves graph calls (a captured graph copies from the buffer it was
    // captured with); the other calls rotate over the remaining slots, so that
    // a call waits only for the upload of the call N_STAGING - 1 before it,
    // not for the previous call's (which may sit behind work still queued).
    // staging / d_staging / staging_cap name the slot ensure_staging chose.
    static constexpr int N_STAGING = 8;
    struct StagingSlot {
        void* host = nullptr;
        void* dev = nullptr;
        size_t cap = 0;
        cudaEvent_t ev = nullptr;
        bool live = false;
    };
    StagingSlot stage_slots[N_STAGING];
    int staging_slot = 0, staging_next = 1;
    void* staging = nullptr;      // pinned host descriptors of the current slot
    void* d_staging = nullptr;
    size_t staging_cap = 0;
    uint64_t launches = 0;
    std::vector<hpa::CachedGraph> graphs;
    void* host_io = nullptr;
    size_t host_io_cap = 0;
    void* pinned_io = nullptr;
    size_t last_carve = 0;        // scratch bytes used by the last carve_work
    cudaStream_t capture_stream = nullptr;
    // copies between host and device spread over several streams (copy engines)
    static constexpr int N_COPY_STREAMS = 4;
    cudaStream_t copy_streams[N_COPY_STREAMS] = {};
    cudaEvent_t copy_fork = nullptr, copy_join[N_COPY_STREAMS] = {};
    struct Copy { void* dst; const void* src; size_t bytes; };
    hpa_status copies(const Copy* c, int n, cudaMemcpyKind kind);
    uint64_t graph_replays = 0;
    uint64_t last_plain_shape = 0;   // shape of the previous hpa_attribute_samples call
    void* cct_scratch = nullptr;
    size_t cct_cap = 0;
    void* aux_scratch = nullptr;  // intermediate keys of analyses built on the aggregation
    size_t aux_cap = 0;
    // phase timing
    bool timing = false;
    std::vector<std::vector<cudaEvent_t>> ev_pool, ev_pending;
    std::vector<bool> ev_counts;   // per pending event set: starts a new call
    double phase_ms[hpa::N_PHASES] = {0};
    uint64_t phase_calls = 0;
    cudaEvent_t* phase_events(bool new_call = true);
    void collect_phase_times();

    ~hpa_handle();
    hpa_status fail(hpa_status st, const char* fmt, ...);
    hpa_status cuda(cudaError_t e, const char* what);
    bool capturing() const;
    hpa_status ensure_scratch(size_t bytes);
    hpa_status ensure_staging(size_t bytes, bool for_graph = false);
    hpa_status upload_staging(size_t bytes);
    hpa::Binary* binary(uint32_t id);
    hpa_status refresh_bin_table();
    hpa_status aggregate(uint32_t n, const uint32_t* binary_ids, const hpa_samples* in, hpa_profile* outs,
                         bool use_graph = false);
    hpa_status launch_graph(const std::vector<hpa::AggWork>& ws, size_t staged_bytes, uint32_t n,
                            const hpa_samples* in);
    hpa_status carve_work(hpa::AggWork& w, uint64_t N, uint64_t G, uint32_t n_buf, uint32_t cap, uint32_t sb,
                          uint32_t sbits, bool has_cnt, bool val64, uint64_t staged = 0,
                          uint64_t cnt_words = 0,    // part counters incl. the scan total (0: none)
                          uint64_t seg_words = 0,    // bucket segments + 2 (two-level partition; 0: none)
                          uint64_t cnt2_words = 0);  // second-pass counters incl. the scan total
    // descriptors of single-output pipelines (expansion, union) in the staging area
    hpa_status stage_single_output(hpa::AggWork& w, uint32_t bin, uint32_t n_ctx, const hpa_profile& out);
};

namespace hpa {
hpa_status build_callgraph(hpa_handle* h, Binary* B);

// copy a host vector into a device allocation owned by binary B
template <typename T>
inline hpa_status upload(hpa_handle* h, Binary* B, const std::vector<T>& v, T** out) {
    *out = nullptr;
    if (v.empty()) return HPA_OK;
    void* p = nullptr;
    if (cudaMalloc(&p, v.size() * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return h->fail(HPA_E_OOM, "structure table of %zu bytes", v.size() * sizeof(T));
    }
    B->dev_allocs.push_back(p);
    *out = (T*)p;
    return h->cuda(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "structure upload");
}
}
