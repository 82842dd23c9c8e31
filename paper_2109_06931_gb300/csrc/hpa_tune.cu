// hpa_tune: picks the aggregation configuration by timing the candidates on
// the caller's own buffer.  The configurations differ only in speed: leaf
// capacity (shared-memory leaves of 4096 records, two CTAs per SM, or 10240
// records, one CTA per SM), grouping of records by context (per-part counters
// with shared-memory cursors, or per-context cursor atomics) and aggregation
// inside a leaf (radix sort of the records, or a shared-memory hash table
// and a sort of the distinct keys) and the equal-digit search of the leaf
// radix sort (__match_any_sync, or alternating with ballots).

#include "hpa_host.h"

using namespace hpa;

extern "C" hpa_status hpa_tune(hpa_handle* h, uint32_t binary_id, const hpa_samples* in, hpa_profile* out,
                               uint32_t reps, hpa_options* best, float* ms) {
    hpa::Trace trace_("hpa.tune");
    if (!h || !in || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    if (reps == 0) reps = 2;
    const hpa_options base = h->opt;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return h->cuda(cudaGetLastError(), "cudaEventCreate");
    }
    static const uint32_t caps[2] = {LEAF_CAP_SMALL, LEAF_CAP_LARGE};
    hpa_status st = HPA_OK;
    float best_ms = 0.f;
    hpa_options chosen = base;
    int k = 0;
    for (int c = 0; c < 2 && !st; ++c)
        for (uint32_t g = 0; g < 2 && !st; ++g)
            for (uint32_t hsh = 0; hsh <= 1 && !st; ++hsh)
                for (uint32_t r = 1; r <= 3 && !st; r += 2, ++k) {     // __match_any_sync, alternating
                hpa_options o = base;
                o.leaf_capacity = caps[c];
                o.grouping = g;
                o.leaf_hash = hsh;
                o.leaf_ranking = r;
                h->opt = o;
                if ((st = h->aggregate(1, &binary_id, in, out))) break;          // untimed
                cudaEventRecord(e0, h->stream);
                for (uint32_t i = 0; i < reps && !st; ++i) st = h->aggregate(1, &binary_id, in, out);
                cudaEventRecord(e1, h->stream);
                if (st) break;
                if ((st = h->cuda(cudaEventSynchronize(e1), "cudaEventSynchronize"))) break;
                if ((st = hpa_sync(h, nullptr))) break;
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                t /= (float)reps;
                if (ms) ms[k] = t;
                if (k == 0 || t < best_ms) {
                    best_ms = t;
                    chosen = o;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->opt = st ? base : chosen;
    if (!st && best) *best = chosen;
    return st;
}
