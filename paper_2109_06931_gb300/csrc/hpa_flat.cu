// hpa_flat_profile: the flat view of a profile (Section 7: besides the
// calling-context (top-down) view, costs are presented by static program
// structure alone).  Every key's value is added into a dense accumulator
// indexed by (node, stall) -- UNKNOWN coded as node n_nodes -- and the
// nonzero entries are compacted in index order, which is (node, stall)
// order.  Exact: 64-bit integer sums.

#include "hpa_host.h"

namespace hpa {

constexpr int FLAT_CHUNK = 4096;           // accumulator entries per compaction block
constexpr uint64_t FLAT_MAX = 1ull << 28;  // accumulator entries (2 GiB)

struct FlatArgs {
    const uint32_t* ctx;
    const uint32_t* node;
    const uint8_t* stall;
    const uint64_t* val;
    const uint64_t* n_keys;
    uint64_t cap;
    uint32_t M, n_ctx, n_stall, sb;
    unsigned long long* acc;     // [(M + 1) << sb]
    uint64_t n_acc;
    uint32_t* chunk;             // [chunks + 1] nonzero entries per chunk -> exclusive scan
    uint64_t n_chunk;
    // output
    uint32_t* key_ctx;
    uint32_t* key_node;
    uint8_t* key_stall;
    uint64_t* out_val;
    uint64_t* out_n;
    uint64_t out_cap;
    uint64_t* total;
    uint64_t* unknown;
    DevStatus* status;
};

__global__ void k_flat_accum(FlatArgs a) {
    const uint64_t K = min(*a.n_keys, a.cap);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < K; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t n = a.node[i], r = a.stall[i];
        if (a.ctx[i] >= a.n_ctx || r >= a.n_stall || (n != UNKNOWN && n >= a.M)) {
            atomicAdd(&a.status->bad, 1ull);
            raise_status(a.status, 3 /* HPA_E_INVALID_SAMPLE */, 0);
            continue;
        }
        const uint64_t idx = ((uint64_t)(n == UNKNOWN ? a.M : n) << a.sb) | r;
        atomicAdd(&a.acc[idx], (unsigned long long)a.val[i]);
    }
}

__global__ void __launch_bounds__(256) k_flat_count(FlatArgs a) {
    __shared__ uint32_t sw[33];
    for (uint64_t c = blockIdx.x; c < a.n_chunk; c += gridDim.x) {
        const uint64_t e0 = c * FLAT_CHUNK;
        uint32_t nz = 0;
        for (uint64_t e = e0 + threadIdx.x; e < min(e0 + FLAT_CHUNK, a.n_acc); e += 256) nz += a.acc[e] != 0;
        uint32_t tot;
        block_exclusive_scan<uint32_t, 256>(nz, sw, &tot);
        if (threadIdx.x == 0) a.chunk[c] = tot;
    }
}

__global__ void __launch_bounds__(256) k_flat_emit(FlatArgs a) {
    __shared__ uint32_t sw[33];
    __shared__ unsigned long long tot_s[HPA_MAX_STALL_DEV], unk_s[HPA_MAX_STALL_DEV];
    if (threadIdx.x < HPA_MAX_STALL_DEV) { tot_s[threadIdx.x] = 0; unk_s[threadIdx.x] = 0; }
    __syncthreads();
    const uint32_t smask = (1u << a.sb) - 1;
    for (uint64_t c = blockIdx.x; c < a.n_chunk; c += gridDim.x) {
        const uint64_t e0 = c * FLAT_CHUNK, e1 = min(e0 + FLAT_CHUNK, a.n_acc);
        uint32_t base = a.chunk[c];
        // entries in order: 16 consecutive entries per thread, a block scan places them
        constexpr int EPT = FLAT_CHUNK / 256;
        const uint64_t t0 = e0 + (uint64_t)threadIdx.x * EPT;
        unsigned long long v[EPT];
        uint32_t nz = 0;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            v[k] = (t0 + k < e1) ? a.acc[t0 + k] : 0ull;
            nz += v[k] != 0;
        }
        uint32_t tot;
        uint32_t pos = base + block_exclusive_scan<uint32_t, 256>(nz, sw, &tot);
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            if (!v[k]) continue;
            const uint64_t idx = t0 + k;
            const uint32_t node = (uint32_t)(idx >> a.sb), stall = (uint32_t)idx & smask;
            atomicAdd(&tot_s[stall], v[k]);
            if (node == a.M) atomicAdd(&unk_s[stall], v[k]);
            if (pos < a.out_cap) {
                a.key_ctx[pos] = 0;
                a.key_node[pos] = node == a.M ? UNKNOWN : node;
                a.key_stall[pos] = (uint8_t)stall;
                a.out_val[pos] = v[k];
            }
            ++pos;
        }
    }
    __syncthreads();
    if (threadIdx.x < a.n_stall) {
        if (a.total && tot_s[threadIdx.x]) atomicAdd((unsigned long long*)&a.total[threadIdx.x], tot_s[threadIdx.x]);
        if (a.unknown && unk_s[threadIdx.x]) atomicAdd((unsigned long long*)&a.unknown[threadIdx.x], unk_s[threadIdx.x]);
    }
}

__global__ void k_flat_finish(FlatArgs a) {
    const uint64_t K = a.chunk[a.n_chunk];
    *a.out_n = K;
    if (K > a.out_cap) raise_status(a.status, 4 /* HPA_E_CAPACITY */, 0);
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_flat_profile(hpa_handle* h, uint32_t binary_id, const hpa_profile* p, hpa_profile* out) {
    hpa::Trace trace_("hpa.flat_profile");
    if (!h || !p || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = h->binary(binary_id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", binary_id);
    if (!p->n_keys || (p->capacity && (!p->key_ctx || !p->key_node || !p->key_stall || !p->val)))
        return h->fail(HPA_E_INVALID_ARG, "input profile arrays missing");
    if (p->n_stall == 0 || p->n_stall > HPA_MAX_STALL || p->n_ctx == 0)
        return h->fail(HPA_E_INVALID_ARG, "input profile has no n_ctx / n_stall (produce it with hpa_attribute_samples)");
    if (!out->n_keys || (out->capacity && (!out->key_ctx || !out->key_node || !out->key_stall || !out->val)))
        return h->fail(HPA_E_INVALID_ARG, "output arrays missing");
    const uint32_t sb = ceil_log2_u64(p->n_stall);
    const uint64_t n_acc = ((uint64_t)B->n_nodes + 1) << sb;
    if (n_acc > FLAT_MAX)
        return h->fail(HPA_E_INVALID_ARG, "(n_nodes + 1) * 2^stall_bits = %llu exceeds %llu accumulator entries",
                       (unsigned long long)n_acc, (unsigned long long)FLAT_MAX);
    const uint64_t n_chunk = (n_acc + FLAT_CHUNK - 1) / FLAT_CHUNK;
    FlatArgs a{};
    auto layout = [&](Carve& c) {
        a.acc = c.take<unsigned long long>(n_acc);
        a.chunk = c.take<uint32_t>(n_chunk + 1);
        a.n_acc = n_acc;
        a.n_chunk = n_chunk;
    };
    Carve probe{nullptr};
    layout(probe);
    const size_t need = probe.off + scan_tmp_words(n_chunk) * 4 + 512;
    hpa_status st = h->ensure_scratch(need);
    if (st) return st;
    Carve c{(char*)h->scratch};
    layout(c);
    uint32_t* scan_tmp = c.take<uint32_t>(scan_tmp_words(n_chunk));
    a.ctx = p->key_ctx; a.node = p->key_node; a.stall = p->key_stall; a.val = p->val;
    a.n_keys = p->n_keys; a.cap = p->capacity;
    a.M = B->n_nodes; a.n_ctx = p->n_ctx; a.n_stall = p->n_stall; a.sb = sb;
    a.key_ctx = out->key_ctx; a.key_node = out->key_node; a.key_stall = out->key_stall; a.out_val = out->val;
    a.out_n = out->n_keys; a.out_cap = out->capacity; a.total = out->total; a.unknown = out->unknown;
    a.status = h->d_status;
    cudaStream_t s = h->stream;
    cudaMemsetAsync(a.acc, 0, n_acc * 8, s);
    if (out->total) cudaMemsetAsync(out->total, 0, 8 * p->n_stall, s);
    if (out->unknown) cudaMemsetAsync(out->unknown, 0, 8 * p->n_stall, s);
    const int blocks = h->sms * 8;
    k_flat_accum<<<blocks, 256, 0, s>>>(a);
    k_flat_count<<<blocks, 256, 0, s>>>(a);
    scan_u32(a.chunk, a.chunk, n_chunk, scan_tmp, s, &h->launches);
    k_flat_emit<<<blocks, 256, 0, s>>>(a);
    k_flat_finish<<<1, 1, 0, s>>>(a);
    h->launches += 4;
    out->n_ctx = 1;
    out->n_stall = p->n_stall;
    out->n_nodes = B->n_nodes;
    return h->cuda(cudaGetLastError(), "flat profile launch");
}
