// hpa_attribute_samples_noalloc: the attribution + aggregation call for
// callers that must not allocate device memory during the call.
//
// Who cannot allocate: a measurement tool running inside the application it
// observes, where the application's caching allocator holds the device memory
// (an allocation by the tool would change the footprint under measurement and
// may fail outright), and a serving loop sharing the GPU with other work,
// where cudaFree synchronises the whole device.  This entry point takes its
// scratch from one fixed array declared at file scope in device memory and
// calls no cudaMalloc, cudaFree or other allocating routine.  The kernels are
// the same ones hpa_attribute_samples launches.
//
// The array is NOALLOC_SCRATCH_BYTES (48 MiB) on every GPU that loads this
// library, for as long as the process lives.  All calls on one device share
// it and it keeps the last call's contents: two calls that overlap on the GPU
// (on different streams or handles without synchronisation between them)
// race and corrupt each other's results.  Each call clears the parts that
// must start at zero.

#include <algorithm>
#include <mutex>

#include "hpa_host.h"

namespace hpa {

constexpr size_t NOALLOC_SCRATCH_BYTES = 48ull << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// device address of g_noalloc_scratch per device, looked up once per device
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256];
static bool g_noalloc_ready[256];

static hpa_status noalloc_address(hpa_handle* h, void** out) {
    if (h->device < 0 || h->device >= 256) return h->fail(HPA_E_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ready[h->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return h->cuda(e, "cudaGetSymbolAddress(static scratch)");
        g_noalloc_ptr[h->device] = p;
        g_noalloc_ready[h->device] = true;
    }
    *out = g_noalloc_ptr[h->device];
    return HPA_OK;
}

// descriptors of the single buffer, written on the device from kernel arguments
__global__ void k_noalloc_descriptors(BufDev d, uint64_t tiles, uint32_t groups, BufDev* bufs, uint64_t* tile,
                                      uint32_t* grp) {
    bufs[0] = d;
    tile[0] = 0;
    tile[1] = tiles;
    grp[0] = 0;
    grp[1] = groups;
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_attribute_samples_noalloc(hpa_handle* h, uint32_t binary_id, const hpa_samples* in,
                                                    hpa_profile* out) {
    hpa::Trace trace_("hpa.attribute_samples_noalloc");
    if (!h || !in || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = h->binary(binary_id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", binary_id);
    const hpa_samples& s = *in;
    if (s.n_ctx == 0) return h->fail(HPA_E_INVALID_ARG, "n_ctx must be >= 1");
    if (s.n_stall == 0 || s.n_stall > HPA_MAX_STALL)
        return h->fail(HPA_E_INVALID_ARG, "n_stall must be in [1, %u]", HPA_MAX_STALL);
    if (s.n && (!s.pc || !s.ctx || !s.stall)) return h->fail(HPA_E_INVALID_ARG, "null sample array");
    if (!out->n_keys || (out->capacity && (!out->key_ctx || !out->key_node || !out->key_stall || !out->val)))
        return h->fail(HPA_E_INVALID_ARG, "output arrays missing");
    const uint64_t N = s.n, G = s.n_ctx;
    const bool has_cnt = s.count != nullptr;
    const uint32_t sb = ceil_log2_u64(s.n_stall);
    const uint32_t nb = ceil_log2_u64((uint64_t)B->n_nodes + 1);
    if (nb + sb > 32) return h->fail(HPA_E_INVALID_ARG, "(n_nodes + 1) * 2^stall_bits exceeds 2^32");
    if (h->opt.leaf_capacity && h->opt.leaf_capacity != LEAF_CAP_SMALL && h->opt.leaf_capacity != LEAF_CAP_LARGE)
        return h->fail(HPA_E_INVALID_ARG, "leaf_capacity must be 0, %u or %u", LEAF_CAP_SMALL, LEAF_CAP_LARGE);
    const uint32_t cap = h->opt.leaf_capacity ? h->opt.leaf_capacity
                                              : ((N / G >= LEAF_CAP_SMALL / 2) ? LEAF_CAP_LARGE : LEAF_CAP_SMALL);
    const uint64_t L_max = G + 6 * (N / cap + 1) + 9;

    AggWork w{};
    w.G = (uint32_t)G; w.n_buf = 1; w.cap = cap; w.q = cap / 2; w.sb = sb; w.sbits = nb + sb;
    w.span_log = std::min<uint32_t>(10, 32 - w.sbits);
    w.cur_shift = 0;
    w.L_max = (uint32_t)L_max; w.has_cnt = has_cnt; w.val64 = false;
    w.emit_totals = 1;
    w.timeout_iters = h->opt.timeout_iters;
    w.sort_mode = std::min<uint32_t>(h->opt.leaf_ranking, 3);
    w.leaf_hash = h->opt.leaf_hash;
    w.emit_separate = h->opt.leaf_emit == 0 ? 1u : 0u;
    w.small_leaves = h->opt.small_leaves == 2 || (h->opt.small_leaves == 0 && N < 64 * G);
    w.n_tiles = (N + TILE - 1) / TILE;
    BufDev* d_buf = nullptr;
    uint64_t* d_tile = nullptr;
    uint32_t* d_grp = nullptr;
    auto layout = [&](Carve& c) {
        d_buf = c.take<BufDev>(1);
        d_tile = c.take<uint64_t>(2);
        d_grp = c.take<uint32_t>(2);
        w.grp_hist = c.take<uint32_t>(G + 1);
        w.grp_cursor = c.take<uint32_t>(G + 1);
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
        w.buf_first_leaf = c.take<uint32_t>(2);
        w.buf_bad = c.take<unsigned long long>(1);
        w.rec_sub = has_cnt ? nullptr : c.take<uint32_t>(N + 1);
        w.rec2_sub = has_cnt ? nullptr : c.take<uint32_t>(w.n_tiles * TILE + 1);
        w.rec_pair = has_cnt ? c.take<uint2>(N + 1) : nullptr;
        w.rec2_pair = has_cnt ? c.take<uint2>(w.n_tiles * TILE + 1) : nullptr;
        w.tmp_key = c.take<uint32_t>(N + 1);
        w.tmp_val = c.take<uint64_t>(N + 1);
        w.scan_tmp = c.take<uint32_t>(scan_tmp_words(std::max<uint64_t>(G, L_max)));
    };
    Carve probe{nullptr};
    layout(probe);
    if (probe.off > NOALLOC_SCRATCH_BYTES)
        return h->fail(HPA_E_INVALID_ARG,
                       "this call needs %zu bytes of scratch; the static scratch of hpa_attribute_samples_noalloc "
                       "holds %zu (use hpa_attribute_samples, or fewer samples / contexts per call)",
                       probe.off, NOALLOC_SCRATCH_BYTES);
    void* base = nullptr;
    hpa_status st = noalloc_address(h, &base);
    if (st) return st;
    Carve real{(char*)base};
    layout(real);
    w.bufs = d_buf;
    w.buf_tile = d_tile;
    w.buf_grp = d_grp;
    w.bins = h->d_bins;
    w.status = h->d_status;
    w.n_rec = N;
    BufDev d{};
    d.pc = s.pc; d.ctx = s.ctx; d.stall = s.stall; d.count = s.count; d.n = s.n;
    d.tile_base = 0; d.n_ctx = s.n_ctx; d.n_stall = s.n_stall; d.grp_base = 0; d.bin = binary_id;
    d.total = out->total; d.unknown = out->unknown;
    d.key_ctx = out->key_ctx; d.key_node = out->key_node; d.key_stall = out->key_stall; d.val = out->val;
    d.n_keys = out->n_keys; d.capacity = out->capacity;
    cudaStream_t stream = h->stream;
    k_noalloc_descriptors<<<1, 1, 0, stream>>>(d, w.n_tiles, (uint32_t)G, d_buf, d_tile, d_grp);
    h->launches += 1;
    out->n_ctx = s.n_ctx;
    out->n_stall = s.n_stall;
    out->n_nodes = B->n_nodes;
    run_aggregate(w, stream, h->sms, &h->launches, nullptr);
    return h->cuda(cudaGetLastError(), "aggregation launch (static scratch)");
}
