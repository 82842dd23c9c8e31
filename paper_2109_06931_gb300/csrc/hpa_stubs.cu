// Entry points whose kernels live in later translation units.
#include "hpa_host.h"
extern "C" hpa_status hpa_attribute_batch(hpa_handle* h, uint32_t n, const uint32_t* ids, const hpa_samples* in, hpa_profile* outs) {
    if (!h || (n && (!ids || !in || !outs))) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    return h->aggregate(n, ids, in, outs, true);
}
