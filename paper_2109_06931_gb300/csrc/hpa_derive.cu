// Derived metrics across profiles (Section 4.5: sum, min, mean, max,
// standard deviation and coefficient of variation over thread profiles) and
// the warp issue rate W = (S - S_stall) / S per context (Section 7).
//
// The keys of all P profiles are partitioned by context and sorted per leaf
// with the shared plan / partition stages; a run of equal keys holds at most
// one value per profile.  Per key: present count, sum, exact sum of squares
// (128-bit), min and max; absent profiles count as 0:
//   mean = sum / P, var = (P * sumsq - sum^2) / P^2 (exact integer
//   numerator, FP32 from there), std = sqrt(var), cov = std / mean.

#include <algorithm>

#include "hpa_host.h"
#include "hpa_warpagg.cuh"

namespace hpa {

struct ProfDesc {
    const uint32_t* ctx;
    const uint32_t* node;
    const uint8_t* stall;
    const uint64_t* val;
    const uint64_t* n_keys;
    uint64_t cap;
    uint64_t base;     // first flattened index
};

struct StatOut {
    uint64_t* mn;
    uint64_t* mx;
    float* mean;
    float* sd;
    float* cov;
};

struct DeriveArgs {
    const ProfDesc* prof;
    const uint64_t* prof_base;   // [P + 1]
    uint32_t P;
    uint64_t total;              // sum of capacities
    uint32_t M;                  // UNKNOWN coded as node M
    uint32_t n_ctx;              // union contexts (groups)
    uint32_t sb;
    StatOut tmp;                 // per run (at the leaf's record offsets)
};

__device__ __forceinline__ bool fetch(const DeriveArgs& A, uint64_t i, uint32_t& c, uint32_t& sub, uint64_t& v,
                                      uint32_t sb) {
    const uint32_t p = upper_index<uint64_t>(A.prof_base, A.P, i);
    const ProfDesc& d = A.prof[p];
    const uint64_t j = i - d.base;
    if (j >= min(*d.n_keys, d.cap)) return false;
    c = d.ctx[j];
    const uint32_t n = d.node[j];
    const uint32_t node = n == UNKNOWN ? A.M : n;
    sub = (node << sb) | d.stall[j];
    v = d.val[j];
    return c < A.n_ctx && (n == UNKNOWN || n < A.M);
}

// Both passes walk the flattened keys warp by warp (the loop is uniform in
// a warp) and count with warp-aggregated atomics: the profiles are sorted by
// context, so the lanes of a warp mostly share one.
__global__ void k_union_hist(AggWork w, DeriveArgs A) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); i0 < A.total; i0 += stride) {
        const uint64_t i = i0 + (threadIdx.x & 31u);
        uint32_t c = 0, sub;
        uint64_t v;
        bool ok = false;
        if (i < A.total) {
            ok = fetch(A, i, c, sub, v, w.sb);
            if (!ok) {
                const uint32_t p = upper_index<uint64_t>(A.prof_base, A.P, i);
                if (i - A.prof[p].base < min(*A.prof[p].n_keys, A.prof[p].cap)) atomicAdd(&w.buf_bad[0], 1ull);
            }
        }
        warp_agg_inc(ok ? &w.grp_hist[c] : nullptr);
    }
}

__global__ void k_union_scatter(AggWork w, DeriveArgs A) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); i0 < A.total; i0 += stride) {
        const uint64_t i = i0 + (threadIdx.x & 31u);
        uint32_t c = 0, sub = 0;
        uint64_t v = 0;
        const bool ok = i < A.total && fetch(A, i, c, sub, v, w.sb);
        const uint32_t slot = warp_agg_inc(ok ? &w.grp_cursor[(size_t)c << w.cur_shift] : nullptr);
        if (!ok) continue;
        w.rec_sub[slot] = sub;
        w.rec_v64[slot] = v;
    }
}

// Statistics of one key from its exact integer sums.  The variance's
// numerator P * sumsq - sum^2 is exact (128-bit); the divisions and the
// square root are FP32, the precision of the outputs (a few ulp of error).
__device__ __forceinline__ void key_stats(uint32_t P, uint32_t cnt, unsigned long long sum, unsigned long long sql,
                                          unsigned long long sqh, unsigned long long mn, unsigned long long mx,
                                          const StatOut& o, size_t at) {
    const unsigned __int128 sq = ((unsigned __int128)sqh << 64) | sql;
    const unsigned __int128 num = (unsigned __int128)P * sq - (unsigned __int128)sum * sum;
    const float numf = __fmaf_rn(__ull2float_rn((unsigned long long)(num >> 64)), 18446744073709551616.0f,
                                 __ull2float_rn((unsigned long long)num));
    const float pf = (float)P;
    const float var = numf / (pf * pf);
    const float sd = sqrtf(var);
    const float mean = __ull2float_rn(sum) / pf;
    o.mn[at] = cnt < P ? 0ull : mn;
    o.mx[at] = mx;
    o.mean[at] = mean;
    o.sd[at] = sd;
    o.cov[at] = sd / mean;
}

constexpr int DS_THREADS = 512;
constexpr int DS_CAP = LEAF_CAP_SMALL;
constexpr int DS_WIN = 1024;    // keys per dense window of the oversized path

// Leaf of the union: the records' keys are sorted with their index within
// the leaf in the upper 32 bits of each element (9-bit digits), and the
// values are gathered by index afterwards, run by run.
template <int THREADS, int CAP>
__global__ void __launch_bounds__(THREADS, 2) k_leaf_stats(AggWork w, DeriveArgs A) {
    using Sort = PackedRadix<THREADS, CAP, uint64_t>;
    constexpr int EPT = (CAP + THREADS - 1) / THREADS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename Sort::Smem& S = *reinterpret_cast<typename Sort::Smem*>(smem_raw);
    __shared__ uint32_t sw[33];
    __shared__ uint32_t gb[1025];
    __shared__ unsigned long long red[2];
    const uint32_t n_leaves = w.item_nleaf[w.G];
    const uint32_t* seg = w.grp_hist;
    for (uint32_t l = blockIdx.x; l < n_leaves; l += gridDim.x) {
        const uint32_t start = w.leaf_start[l], end = w.leaf_end[l], info = w.leaf_info[l];
        const uint32_t n = end - start;
        const uint32_t* src_sub = (info & 1u) ? w.rec2_sub : w.rec_sub;
        const uint64_t* src_val = (info & 1u) ? w.rec2_v64 : w.rec_v64;
        if (n == 0) {
            if (threadIdx.x == 0) w.leaf_d[l] = 0;
            continue;
        }
        if (n <= (uint32_t)CAP) {
            const uint32_t g0 = w.leaf_grp0[l];
            uint32_t ng = 1;
            if (!(info & 1u)) {
                uint32_t lo = g0, hi = min(w.G, g0 + 1024u);
                while (hi - lo > 1) {
                    const uint32_t m = (lo + hi) >> 1;
                    if (seg[m] < end) lo = m; else hi = m;
                }
                ng = lo - g0 + 1;
            }
            const uint32_t gbits = ng > 1 ? ceil_log2_u64(ng) : 0;
            if (ng > 1) {
                for (uint32_t j = threadIdx.x; j <= ng; j += THREADS) gb[j] = seg[g0 + j] - start;
                __syncthreads();
            }
            for (uint32_t i = threadIdx.x; i < n; i += THREADS)
                S.el[0][i] = (uint64_t)src_sub[start + i] | ((uint64_t)i << 32);
            __syncthreads();
            if (ng > 1) {
                for (uint32_t j = threadIdx.x; j < ng; j += THREADS) {
                    const uint32_t a = gb[j], e = min(gb[j + 1], n);
                    for (uint32_t i = a; i < e; ++i) S.el[0][i] |= (uint64_t)(j << w.sbits);
                }
                __syncthreads();
            }
            const int cur = Sort::sort(S, (int)n, (int)(w.sbits + gbits), 0, w.status);
            const uint64_t* el = S.el[cur];
            const int c0 = threadIdx.x * EPT, c1 = min((int)n, c0 + EPT);
            uint32_t heads = 0;
            for (int i = c0; i < c1; ++i) heads += (i == 0) || ((uint32_t)el[i] != (uint32_t)el[i - 1]);
            uint32_t n_runs;
            uint32_t run = block_exclusive_scan<uint32_t, THREADS>(heads, sw, &n_runs);
            for (int i = c0; i < c1; ++i) {
                const uint32_t k = (uint32_t)el[i];
                if (!(i == 0 || k != (uint32_t)el[i - 1])) continue;
                uint32_t cnt = 0;
                unsigned long long sum = 0, sql = 0, sqh = 0, mn = ~0ull, mx = 0;
                for (int j = i; j < (int)n && (uint32_t)el[j] == k; ++j) {
                    const unsigned long long x = src_val[start + (uint32_t)(el[j] >> 32)];
                    ++cnt;
                    sum += x;
                    const unsigned long long lo2 = x * x, hi2 = __umul64hi(x, x);
                    sql += lo2;
                    sqh += hi2 + (sql < lo2);
                    mn = min(mn, x);
                    mx = max(mx, x);
                }
                const size_t at = (size_t)start + run;
                w.tmp_key[at] = k;
                w.tmp_val[at] = sum;
                key_stats(A.P, cnt, sum, sql, sqh, mn, mx, A.tmp, at);
                ++run;
            }
            if (threadIdx.x == 0) w.leaf_d[l] = n_runs;
            __syncthreads();
        } else {
            // oversized sub-bin (one group): dense per-key accumulators, window by window
            uint32_t* cntw = reinterpret_cast<uint32_t*>(smem_raw);
            unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem_raw + DS_WIN * 4);
            unsigned long long *sumw = acc, *sqlw = acc + DS_WIN, *sqhw = acc + 2 * DS_WIN,
                               *mnw = acc + 3 * DS_WIN, *mxw = acc + 4 * DS_WIN;
            uint32_t kmn = 0xFFFFFFFFu, kmx = 0;
            for (uint32_t i = start + threadIdx.x; i < end; i += THREADS) {
                const uint32_t k = src_sub[i];
                kmn = min(kmn, k); kmx = max(kmx, k);
            }
            for (int o = 16; o > 0; o >>= 1) {
                kmn = min(kmn, __shfl_xor_sync(0xffffffffu, kmn, o));
                kmx = max(kmx, __shfl_xor_sync(0xffffffffu, kmx, o));
            }
            if (threadIdx.x == 0) { red[0] = 0xFFFFFFFFull; red[1] = 0; }
            __syncthreads();
            if (lane_id() == 0) { atomicMin(&red[0], (unsigned long long)kmn); atomicMax(&red[1], (unsigned long long)kmx); }
            __syncthreads();
            const uint32_t k0 = (uint32_t)red[0], k1 = (uint32_t)red[1];
            __syncthreads();
            uint32_t out = 0;
            constexpr int DEPT = DS_WIN / THREADS;
            for (uint64_t wlo = k0; wlo <= k1; wlo += DS_WIN) {
                for (int j = threadIdx.x; j < DS_WIN; j += THREADS) {
                    cntw[j] = 0; sumw[j] = 0; sqlw[j] = 0; sqhw[j] = 0; mnw[j] = ~0ull; mxw[j] = 0;
                }
                __syncthreads();
                for (uint32_t i = start + threadIdx.x; i < end; i += THREADS) {
                    const uint32_t k = src_sub[i];
                    if (k < wlo || (uint64_t)k >= wlo + DS_WIN) continue;
                    const uint32_t j = k - (uint32_t)wlo;
                    const unsigned long long x = src_val[i];
                    atomicAdd(&cntw[j], 1u);
                    atomicAdd(&sumw[j], x);
                    const unsigned long long lo2 = x * x, hi2 = __umul64hi(x, x);
                    const unsigned long long old = atomicAdd(&sqlw[j], lo2);
                    const unsigned long long carry = (old + lo2 < old) ? 1ull : 0ull;
                    if (hi2 + carry) atomicAdd(&sqhw[j], hi2 + carry);
                    atomicMin(&mnw[j], x);
                    atomicMax(&mxw[j], x);
                }
                __syncthreads();
                const int b0 = threadIdx.x * DEPT;
                uint32_t nz = 0;
                for (int j = 0; j < DEPT; ++j) nz += cntw[b0 + j] != 0;
                uint32_t tot;
                uint32_t pos = block_exclusive_scan<uint32_t, THREADS>(nz, sw, &tot);
                for (int j = 0; j < DEPT; ++j) {
                    const int q = b0 + j;
                    if (!cntw[q]) continue;
                    const size_t at = (size_t)start + out + pos;
                    w.tmp_key[at] = (uint32_t)(wlo + q);
                    w.tmp_val[at] = sumw[q];
                    key_stats(A.P, cntw[q], sumw[q], sqlw[q], sqhw[q], mnw[q], mxw[q], A.tmp, at);
                    ++pos;
                }
                out += tot;
                __syncthreads();
            }
            if (threadIdx.x == 0) w.leaf_d[l] = out;
            __syncthreads();
        }
    }
}

struct DerivedOut {
    uint32_t* key_ctx;
    uint32_t* key_node;
    uint8_t* key_stall;
    uint64_t* sum;
    uint64_t* mn;
    uint64_t* mx;
    float* mean;
    float* sd;
    float* cov;
    uint64_t capacity;
    uint32_t n_ctx;
    uint32_t S;
    uint32_t issued;
    unsigned long long* per_ctx_stall;   // scratch [n_ctx][S]
    uint64_t* S_all;
    uint64_t* S_issued;
    float* W;
    float* frac;
};

__global__ void __launch_bounds__(256) k_emit_stats(AggWork w, DeriveArgs A, DerivedOut o) {
    const uint32_t n_leaves = w.item_nleaf[w.G];
    const uint32_t* leaf_out = w.leaf_d;
    const uint32_t smask = (w.sbits >= 32) ? 0xFFFFFFFFu : ((1u << w.sbits) - 1);
    const uint32_t stmask = (1u << w.sb) - 1;
    for (uint32_t l = blockIdx.x; l < n_leaves; l += gridDim.x) {
        const uint32_t d = leaf_out[l + 1] - leaf_out[l];
        if (d == 0 || w.buf_bad[0]) continue;
        const uint32_t start = w.leaf_start[l], g0 = w.leaf_grp0[l];
        for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
            const uint64_t pos = (uint64_t)leaf_out[l] + i;
            const size_t at = (size_t)start + i;
            const uint32_t k = w.tmp_key[at];
            const uint32_t sub = k & smask;
            const uint32_t c = g0 + ((w.sbits >= 32) ? 0u : (k >> w.sbits));
            const uint32_t node = sub >> w.sb, r = sub & stmask;
            const uint64_t sum = w.tmp_val[at];
            if (c < o.n_ctx && r < o.S) atomicAdd(&o.per_ctx_stall[(size_t)c * o.S + r], (unsigned long long)sum);
            if (pos >= o.capacity) continue;
            o.key_ctx[pos] = c;
            o.key_node[pos] = node == A.M ? UNKNOWN : node;
            o.key_stall[pos] = (uint8_t)r;
            o.sum[pos] = sum;
            o.mn[pos] = A.tmp.mn[at];
            o.mx[pos] = A.tmp.mx[at];
            o.mean[pos] = A.tmp.mean[at];
            o.sd[pos] = A.tmp.sd[at];
            o.cov[pos] = A.tmp.cov[at];
        }
    }
}

// W = (S - S_stall) / S = S_issued / S and the share of each stall reason
__global__ void k_issue_rate(DerivedOut o) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < o.n_ctx; c += gridDim.x * blockDim.x) {
        unsigned long long s = 0, si = 0;
        for (uint32_t r = 0; r < o.S; ++r) {
            const unsigned long long x = o.per_ctx_stall[(size_t)c * o.S + r];
            s += x;
            if (r < 32 && ((o.issued >> r) & 1u)) si += x;
        }
        if (o.S_all) o.S_all[c] = s;
        if (o.S_issued) o.S_issued[c] = si;
        const float nanf_ = __int_as_float(0x7fc00000);
        if (o.W) o.W[c] = s ? (float)((double)si / (double)s) : nanf_;
        if (o.frac)
            for (uint32_t r = 0; r < o.S; ++r)
                o.frac[(size_t)c * o.S + r] = s ? (float)((double)o.per_ctx_stall[(size_t)c * o.S + r] / (double)s) : nanf_;
    }
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_derive_metrics(hpa_handle* h, const hpa_profile* const* ps, uint32_t P, hpa_derived* out) {
    hpa::Trace trace_("hpa.derive_metrics");
    if (!h || !out || (P && !ps)) return HPA_E_INVALID_ARG;
    if (P == 0) return h->fail(HPA_E_INVALID_ARG, "no profiles");
    cudaSetDevice(h->device);
    uint64_t N = 0;
    uint32_t G = 0, S = 0, M = 0;
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
    if (!out->n_keys || (out->capacity && (!out->key_ctx || !out->key_node || !out->key_stall || !out->sum ||
                                           !out->min || !out->max || !out->mean || !out->std || !out->cov)))
        return h->fail(HPA_E_INVALID_ARG, "derived output arrays missing");
    if (out->n_ctx < G) return h->fail(HPA_E_INVALID_ARG, "out->n_ctx (%u) is smaller than the profiles' contexts (%u)", out->n_ctx, G);
    if (N >= 0xFFFFFFF0ull) return h->fail(HPA_E_INVALID_ARG, "too many keys");
    const uint32_t sb = ceil_log2_u64(S);
    const uint32_t nb = ceil_log2_u64((uint64_t)M + 1);
    if (nb + sb > 32) return h->fail(HPA_E_INVALID_ARG, "(n_nodes + 1) * 2^stall_bits exceeds 2^32");
    AggWork w{};
    hpa_status st = h->carve_work(w, N, G, 1, DS_CAP, sb, nb + sb, true, true);
    if (st) return st;
    // extra scratch: per-run statistics and per-(ctx, stall) sums, after the work arrays
    Carve probe{nullptr};
    probe.off = h->last_carve;
    DeriveArgs A{};
    auto layout = [&](Carve& c) {
        A.tmp.mn = c.take<uint64_t>(N + 1);
        A.tmp.mx = c.take<uint64_t>(N + 1);
        A.tmp.mean = c.take<float>(N + 1);
        A.tmp.sd = c.take<float>(N + 1);
        A.tmp.cov = c.take<float>(N + 1);
        return c.take<unsigned long long>((size_t)out->n_ctx * S);
    };
    layout(probe);
    if (probe.off > h->scratch_cap) {
        if ((st = h->ensure_scratch(probe.off + 256))) return st;
        if ((st = h->carve_work(w, N, G, 1, DS_CAP, sb, nb + sb, true, true))) return st;
    }
    Carve real{(char*)h->scratch};
    real.off = h->last_carve;
    unsigned long long* pcs = layout(real);
    // descriptors: profiles, their flattened bases, and the single output
    if ((st = h->ensure_staging(P * sizeof(ProfDesc) + (P + 1) * 8 + sizeof(BufDev) + 4096))) return st;
    Carve hs{(char*)h->staging};
    ProfDesc* hp = hs.take<ProfDesc>(P);
    uint64_t* hbase = hs.take<uint64_t>(P + 1);
    BufDev* hb = hs.take<BufDev>(1);
    uint64_t* htile = hs.take<uint64_t>(2);
    uint32_t* hgrp = hs.take<uint32_t>(2);
    uint64_t base = 0;
    for (uint32_t p = 0; p < P; ++p) {
        const hpa_profile* q = ps[p];
        hp[p] = ProfDesc{q->key_ctx, q->key_node, q->key_stall, q->val, q->n_keys, q->capacity, base};
        hbase[p] = base;
        base += q->capacity;
    }
    hbase[P] = base;
    BufDev d{};
    d.n_ctx = G; d.n_stall = S; d.n_keys = out->n_keys; d.capacity = out->capacity;
    *hb = d;
    htile[0] = htile[1] = 0;
    hgrp[0] = 0; hgrp[1] = G;
    if ((st = h->upload_staging(hs.off))) return st;
    char* ds = (char*)h->d_staging;
    auto dev = [&](void* hostp) { return ds + ((char*)hostp - (char*)h->staging); };
    A.prof = (const ProfDesc*)dev(hp);
    A.prof_base = (const uint64_t*)dev(hbase);
    A.P = P; A.total = N; A.M = M; A.n_ctx = G; A.sb = sb;
    w.bufs = (const BufDev*)dev(hb);
    w.buf_tile = (const uint64_t*)dev(htile);
    w.buf_grp = (const uint32_t*)dev(hgrp);
    w.n_tiles = 0;
    DerivedOut o{out->key_ctx, out->key_node, out->key_stall, out->sum, out->min, out->max, out->mean, out->std,
                 out->cov, out->capacity, out->n_ctx, S, h->opt.issued_mask, pcs, out->S, out->S_issued, out->W, out->frac};
    cudaStream_t s = h->stream;
    const int sms = h->sms;
    clear_work(w, s);
    cudaMemsetAsync(pcs, 0, (size_t)out->n_ctx * S * 8, s);
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((N + 255) / 256, (uint64_t)sms * 8));
    k_union_hist<<<blocks, 256, 0, s>>>(w, A);
    run_plan(w, s, sms, &h->launches, false);
    k_union_scatter<<<blocks, 256, 0, s>>>(w, A);
    launch_big_partition(w, s, sms, &h->launches);
    using Sort = PackedRadix<DS_THREADS, DS_CAP, uint64_t>;
    const size_t smem = std::max(sizeof(typename Sort::Smem), (size_t)DS_WIN * 44);
    set_smem_limit((const void*)k_leaf_stats<DS_THREADS, DS_CAP>, (int)smem);
    k_leaf_stats<DS_THREADS, DS_CAP><<<sms * 2, DS_THREADS, smem, s>>>(w, A);
    scan_u32(w.leaf_d, w.leaf_d, w.L_max, w.scan_tmp, s, &h->launches);
    k_emit_stats<<<sms * 8, 256, 0, s>>>(w, A, o);
    launch_finalize(w, s, &h->launches);
    k_issue_rate<<<(out->n_ctx + 255) / 256, 256, 0, s>>>(o);
    h->launches += 5;
    return h->cuda(cudaGetLastError(), "derive launch");
}
