// GPU calling context trees of every launch context of a profile (Section
// 6.3, steps 1-4) as sparse rows: per context, the condensed nodes whose
// inclusive cost is not zero and the call sites whose share is not zero --
// the part of the call graph above the context's sampled functions.
//
// Contexts are taken in order from a counter, several CTAs per SM, one
// context per CTA at a time; every step walks the context's own part of the
// graph, never the whole graph:
//  step 1  the context's keys give the exclusive cost of each condensed node
//          (exact 64-bit sums per stall reason, rows zeroed through a list of
//          the nodes with samples) and the measured weight of each call site
//          (samples at its call instruction, all stall reasons; reset through
//          a list of the touched call sites);
//  step 2  functions with samples and no measured incoming weight get weight
//          1 on every incoming call site, repeated through their callers that
//          have no measured incoming weight (a breadth-first queue);
//  step 3  static condensation (Tarjan at load); a condensed node with cost or
//          a member in the step-2 closure whose incoming weight is still zero
//          gets the same rule on the condensed graph (FIXUP2);
//  rows    a bitmap marks the call sites of nonzero weight; the nodes of
//          nonzero inclusive cost are those reachable upward from the nodes
//          with samples through such call sites (a breadth-first search that
//          also fixes each node's incoming weight W, each call site's ratio
//          w / W and its row bit); rows in id order come from the bitmaps'
//          popcounts, their offsets from a look-back over the contexts;
//  step 4  level by level (nodes bucketed by level with a counting sort), one
//          thread per (node, stall column):
//          incl(v) = excl(v) + sum_e r(e) * incl(head(e)),
//          accumulated in double-float arithmetic (error-free products and
//          sums of float pairs) from the float rows of the heads, which are the
//          output rows themselves; each stored value is rounded once to float.
// Contexts without keys have no rows and cost a counter step.

#include <algorithm>

#include "hpa_host.h"

namespace hpa {

// one context per SM at a time, its level-synchronous steps (a barrier and a
// chain of dependent loads per level) spread over 1,024 threads (on 2,000
// contexts of 10^4 keys: 1,024 x 1 took 39.0 ms, 512 x 2 40.6 ms, 256 x 4
// 45.4 ms, 128 x 8 72.9 ms)
constexpr int GALL_THREADS = 1024;
constexpr int GALL_PER_SM = 1;
constexpr size_t GALL_SMEM_MAX = 48 * 1024;   // bitmaps in shared memory up to this size, else in the slot

// per-node / per-function flags of one context (u32 words, atomicOr)
enum : uint32_t {
    GF_HAS = 1,      // function: samples (S(f) > 0)
    GF_MEAS = 2,     // function: a measured incoming call-site weight
    GF_Z = 4,        // function: in the step-2 closure
    GC_NEED = 8,     // condensed node: cost or a member in the step-2 closure
    GC_Z2 = 16,      // condensed node: in the FIXUP2 closure
    GC_EXCL = 32     // condensed node: exclusive cost (keys with a value)
};

struct GallSlot {
    uint32_t* flags;             // [V]
    unsigned long long* wmeas;   // [E] measured call-site weights (reset through `touched`)
    uint32_t* touched;           // [E]
    unsigned long long* excl;    // [V][S] rows of GC_EXCL nodes
    float* ratio;                // [E] r(e) of the context's call-site rows
    uint32_t* q_has;             // [F] functions with samples
    uint32_t* q_z;               // [F] step-2 closure (breadth-first queue)
    uint32_t* q_need;            // [V] nodes with cost or a member in the closure
    uint32_t* q_z2;              // [V] FIXUP2 closure
    uint32_t* q_excl;            // [V] nodes with samples
    uint32_t* q_clos;            // [V] nodes of nonzero inclusive cost (breadth-first queue)
    uint32_t* cl_node;           // [V] the same in level order
    uint32_t* cl_row;            // [V] their rows
    uint32_t* ce_off;            // [V + 1] active out-edges of cl_node[k]
    float* ce_ratio;             // [E]
    uint32_t* ce_hrow;           // [E]
    uint32_t* bits;              // bitmaps when they do not fit shared memory
};

struct GallArgs {
    DevCallGraph g;
    const uint32_t* key_ctx;
    const uint32_t* key_node;
    const uint8_t* key_stall;
    const uint64_t* key_val;
    const uint64_t* n_keys;
    uint64_t key_cap;
    uint32_t n_ctx, S, M;            // contexts, stall reasons, S + 1
    const uint64_t* ctx_start;       // [n_ctx + 1] first key of each context
    hpa_gpucct_all out;
    unsigned long long* look_n;      // [n_ctx] look-back words (node rows)
    unsigned long long* look_e;      // [n_ctx] look-back words (call-site rows)
    uint32_t* ticket;
    char* slots;
    size_t slot_bytes;
    uint32_t smem_bits;              // bitmaps in dynamic shared memory (else in the slot)
    uint32_t timeout_iters;
    DevStatus* status;
};

// bitmaps of one context: call sites of nonzero weight, call-site rows,
// nodes of nonzero inclusive cost, the prefix of the node bitmap's popcounts,
// and the per-level counters of the sweep lists
struct GallBits {
    uint32_t *wpos, *erow, *clos, *npre, *lev;
    uint32_t we, wv;                 // words per call-site / node bitmap
};

__host__ __device__ inline size_t gall_bits_words(const DevCallGraph& g) {
    const size_t we = ((size_t)g.E + 31) / 32 + 1, wv = ((size_t)g.V + 31) / 32 + 1;
    return 2 * we + 2 * wv + g.n_levels + 2;
}

__device__ inline GallBits gall_bits(const DevCallGraph& g, uint32_t* base) {
    GallBits b;
    b.we = (g.E + 31) / 32 + 1;
    b.wv = (g.V + 31) / 32 + 1;
    b.wpos = base;
    b.erow = b.wpos + b.we;
    b.clos = b.erow + b.we;
    b.npre = b.clos + b.wv;
    b.lev = b.npre + b.wv;
    return b;
}

__host__ __device__ inline size_t gall_layout(const DevCallGraph& g, uint32_t S, char* base, GallSlot* s) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~size_t(255);
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    GallSlot t;
    t.flags = (uint32_t*)take((size_t)g.V * 4);
    t.wmeas = (unsigned long long*)take((size_t)g.E * 8 + 8);
    t.touched = (uint32_t*)take((size_t)g.E * 4 + 4);
    t.excl = (unsigned long long*)take((size_t)g.V * S * 8);
    t.ratio = (float*)take((size_t)g.E * 4 + 4);
    t.q_has = (uint32_t*)take((size_t)g.F * 4 + 4);
    t.q_z = (uint32_t*)take((size_t)g.F * 4 + 4);
    t.q_need = (uint32_t*)take((size_t)g.V * 4 + 4);
    t.q_z2 = (uint32_t*)take((size_t)g.V * 4 + 4);
    t.q_excl = (uint32_t*)take((size_t)g.V * 4 + 4);
    t.q_clos = (uint32_t*)take((size_t)g.V * 4 + 4);
    t.cl_node = (uint32_t*)take((size_t)g.V * 4 + 4);
    t.cl_row = (uint32_t*)take((size_t)g.V * 4 + 4);
    t.ce_off = (uint32_t*)take((size_t)g.V * 4 + 8);
    t.ce_ratio = (float*)take((size_t)g.E * 4 + 4);
    t.ce_hrow = (uint32_t*)take((size_t)g.E * 4 + 4);
    t.bits = (uint32_t*)take(gall_bits_words(g) * 4);
    if (s) *s = t;
    return (off + 255) & ~size_t(255);
}

// first key of every context (keys sorted by context): each key that starts a
// context fills the starts of the contexts since the previous key's
__global__ void k_ctx_bounds(const uint32_t* key_ctx, const uint64_t* n_keys, uint64_t key_cap, uint32_t n_ctx,
                             uint64_t* start) {
    const uint64_t K = min(*n_keys, key_cap);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= K; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = i < K ? min(key_ctx[i], n_ctx) : n_ctx;
        const uint32_t p = i == 0 ? 0u : min(key_ctx[i - 1], n_ctx) + 1u;
        for (uint32_t x = p; x <= c; ++x) start[x] = i;
    }
}

// look-back over contexts: publish this context's row count, add up the
// counts before it until a published inclusive prefix (context 0 publishes
// one at once); bounded waits
constexpr unsigned long long GL_AGG = 1ull << 62, GL_INCL = 1ull << 63, GL_VAL = (1ull << 62) - 1;

__device__ unsigned long long ctx_lookback(unsigned long long* look, uint32_t c, unsigned long long cnt,
                                           uint32_t limit, DevStatus* st) {
    if (c == 0) {
        st_release_u64(&look[0], GL_INCL | cnt);
        return 0;
    }
    st_release_u64(&look[c], GL_AGG | cnt);
    unsigned long long prefix = 0;
    uint32_t j = c - 1, polls = 0;
    for (;;) {
        const unsigned long long s = ld_acquire_u64(&look[j]);
        if (s & GL_INCL) { prefix += s & GL_VAL; break; }
        if (s & GL_AGG) {
            prefix += s & GL_VAL;
            if (j == 0) break;
            --j;
            continue;
        }
        if (++polls > limit) {
            raise_status(st, 7 /* HPA_E_TIMEOUT */, 12);
            break;
        }
        __nanosleep(32);
    }
    st_release_u64(&look[c], GL_INCL | (prefix + cnt));
    return prefix;
}

// double-float accumulation: hi + lo carries the exact sum of products of
// floats until the final rounding (error-free product by fmaf, error-free
// sum by the two-sum of floats); the _rn intrinsics keep the compiler from
// contracting the steps
__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float pe = fmaf(x, y, -p);
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    const float l = __fadd_rn(lo, __fadd_rn(e, pe));
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
}

__device__ __forceinline__ void df_from_u64(unsigned long long x, float& hi, float& lo) {
    hi = __ull2float_rn(x);
    const long long r = (long long)(x - (unsigned long long)hi);
    lo = __ll2float_rn(r);
}

__device__ __forceinline__ bool bit_get(const uint32_t* b, uint32_t i) { return (b[i >> 5] >> (i & 31)) & 1u; }
// sets bit i; true if it was already set
__device__ __forceinline__ bool bit_set(uint32_t* b, uint32_t i) {
    const uint32_t m = 1u << (i & 31);
    return (atomicOr(&b[i >> 5], m) & m) != 0;
}
// row of node v: nodes of nonzero inclusive cost before it in id order
__device__ __forceinline__ uint32_t node_rank(const GallBits& B, uint32_t v) {
    return B.npre[v >> 5] + __popc(B.clos[v >> 5] & ((1u << (v & 31)) - 1u));
}

// zero incoming weight before FIXUP2 (measured weights and the step-2 closure)
__device__ __forceinline__ bool w_zero_step2(const DevCallGraph& g, const GallSlot& T, uint32_t v) {
    if (v < g.F) return !(T.flags[v] & (GF_MEAS | GF_Z));
    for (uint32_t j = g.cin_off[v]; j < g.cin_off[v + 1]; ++j) {
        const uint32_t e = g.cin_edge[j];
        if (T.wmeas[e] || (T.flags[g.cs_callee[e]] & GF_Z)) return false;
    }
    return true;
}

// weight of external call site e after steps 2 and 3
__device__ __forceinline__ unsigned long long w2_of(const GallSlot& T, const GallBits& B, uint32_t e) {
    const unsigned long long w = T.wmeas[e];
    return w ? w : (bit_get(B.wpos, e) ? 1ull : 0ull);
}

// Block-wide exclusive prefix sums of cnt(i) over the items [0, n), in id
// order (each thread a contiguous chunk): put(i, sum of cnt over the items
// before i).  Returns the total.
template <typename CNT, typename PUT>
__device__ uint32_t block_prefix_sum(uint32_t n, CNT cnt, PUT put, uint32_t* sw) {
    const uint32_t per = (n + GALL_THREADS - 1) / GALL_THREADS;
    const uint32_t a = min(n, threadIdx.x * per), b = min(n, a + per);
    uint32_t c = 0;
    for (uint32_t i = a; i < b; ++i) c += cnt(i);
    uint32_t tot;
    uint32_t r = block_exclusive_scan<uint32_t, GALL_THREADS>(c, sw, &tot);
    for (uint32_t i = a; i < b; ++i) {
        put(i, r);
        r += cnt(i);
    }
    return tot;
}

// Level-synchronous breadth-first processing of a queue: q[0, *s_n) holds the
// first level (set before the call); visit(x, push) may append with push(y).
template <typename VISIT>
__device__ void block_bfs(uint32_t* q, uint32_t* s_n, uint32_t cap, DevStatus* st, VISIT visit) {
    uint32_t lo = 0;
    for (;;) {
        __syncthreads();
        const uint32_t hi = *s_n;
        __syncthreads();                       // every thread has read *s_n before anyone pushes
        if (hi == lo) break;
        for (uint32_t k = lo + threadIdx.x; k < hi; k += GALL_THREADS)
            visit(q[k], [&](uint32_t y) {
                const uint32_t at = atomicAdd(s_n, 1u);
                if (in_bounds(st, at, cap, 116)) q[at] = y;             // site 116: breadth-first queue
            });
        lo = hi;
    }
}

__global__ void __launch_bounds__(GALL_THREADS, GALL_PER_SM) k_gpucct_all(GallArgs A) {
    const DevCallGraph& g = A.g;
    extern __shared__ __align__(16) uint32_t gsm[];
    __shared__ uint32_t sw[33];
    __shared__ uint32_t s_c, s_ntouch, s_nhas, s_nz, s_nneed, s_nz2, s_nexcl, s_nclos;
    __shared__ unsigned long long s_nbase, s_ebase;
    GallSlot T;
    gall_layout(g, A.S, A.slots + (size_t)blockIdx.x * A.slot_bytes, &T);
    const GallBits B = gall_bits(g, A.smem_bits ? gsm : T.bits);
    const uint32_t tid = threadIdx.x;
    const uint32_t S = A.S, M = A.M;
    const uint32_t limit = A.timeout_iters ? A.timeout_iters : (1u << 22);
    const hpa_gpucct_all& O = A.out;
    // every slot starts with no touched call site
    for (uint32_t e = tid; e < g.E; e += GALL_THREADS) T.wmeas[e] = 0;
    __syncthreads();
    for (;;) {
        if (tid == 0) s_c = atomicAdd(A.ticket, 1u);
        __syncthreads();
        const uint32_t c = s_c;
        if (c >= A.n_ctx) break;
        const uint64_t k0 = A.ctx_start[c], k1 = A.ctx_start[c + 1];
        uint32_t n_rows = 0, n_edges = 0;
        if (k1 > k0) {
            // ---- step 1
            for (uint32_t v = tid; v < g.V; v += GALL_THREADS) T.flags[v] = 0;
            for (uint32_t i = tid; i < 2 * B.we + B.wv; i += GALL_THREADS) B.wpos[i] = 0;   // wpos, erow, clos
            if (tid == 0) { s_ntouch = 0; s_nhas = 0; s_nz = 0; s_nneed = 0; s_nz2 = 0; s_nexcl = 0; s_nclos = 0; }
            __syncthreads();
            for (uint64_t i = k0 + tid; i < k1; i += GALL_THREADS) {
                const uint32_t n = A.key_node[i];
                if (n == UNKNOWN) continue;
                const uint32_t r = A.key_stall[i];
                if (n >= g.M || r >= S) { raise_status(A.status, 1 /* HPA_E_INVALID_ARG */, 13); continue; }
                const unsigned long long v = A.key_val[i];
                if (!v) continue;
                const uint32_t f = g.node_func[n];
                if (!(atomicOr(&T.flags[f], GF_HAS) & GF_HAS)) T.q_has[atomicAdd(&s_nhas, 1u)] = f;
                const uint32_t cv = g.cnode_of_func[f];
                if (!(atomicOr(&T.flags[cv], GC_EXCL) & GC_EXCL)) T.q_excl[atomicAdd(&s_nexcl, 1u)] = cv;
                const uint32_t e = g.node_cs[n];
                if (e != UNKNOWN && atomicAdd(&T.wmeas[e], v) == 0ull) T.touched[atomicAdd(&s_ntouch, 1u)] = e;
            }
            __syncthreads();
            const uint32_t ntouch = s_ntouch, nhas = s_nhas, nexcl = s_nexcl;
            for (uint32_t k = tid; k < nexcl; k += GALL_THREADS)
                for (uint32_t r = 0; r < S; ++r) T.excl[(size_t)T.q_excl[k] * S + r] = 0;
            for (uint32_t t = tid; t < ntouch; t += GALL_THREADS) {
                const uint32_t e = T.touched[t];
                atomicOr(&T.flags[g.cs_callee[e]], GF_MEAS);
                if (!g.edge_intra[e]) bit_set(B.wpos, e);
            }
            __syncthreads();
            for (uint64_t i = k0 + tid; i < k1; i += GALL_THREADS) {
                const uint32_t n = A.key_node[i];
                const uint32_t r = A.key_stall[i];
                if (n == UNKNOWN || n >= g.M || r >= S) continue;
                atomicAdd(&T.excl[(size_t)g.cnode_of_func[g.node_func[n]] * S + r], (unsigned long long)A.key_val[i]);
            }
            // ---- step 2: zero-weight fix-up, closure through callers
            for (uint32_t k = tid; k < nhas; k += GALL_THREADS) {
                const uint32_t f = T.q_has[k];
                if (!(T.flags[f] & GF_MEAS) && g.fin_off[f + 1] > g.fin_off[f] &&
                    !(atomicOr(&T.flags[f], GF_Z) & GF_Z))
                    T.q_z[atomicAdd(&s_nz, 1u)] = f;
            }
            block_bfs(T.q_z, &s_nz, g.F, A.status, [&](uint32_t f, auto push) {
                for (uint32_t j = g.fin_off[f]; j < g.fin_off[f + 1]; ++j) {
                    const uint32_t e = g.fin_edge[j];
                    if (!g.edge_intra[e]) bit_set(B.wpos, e);           // weight 1 (FIXUP)
                    const uint32_t h = g.cs_caller[e];
                    if (g.fin_off[h + 1] > g.fin_off[h] && !(T.flags[h] & GF_MEAS) &&
                        !(atomicOr(&T.flags[h], GF_Z) & GF_Z))
                        push(h);
                }
            });
            // ---- step 3: FIXUP2 on the condensed graph
            const uint32_t nz = s_nz;
            for (uint32_t k = tid; k < nhas + nz; k += GALL_THREADS) {
                const uint32_t cv = g.cnode_of_func[k < nhas ? T.q_has[k] : T.q_z[k - nhas]];
                if (!(atomicOr(&T.flags[cv], GC_NEED) & GC_NEED)) T.q_need[atomicAdd(&s_nneed, 1u)] = cv;
            }
            __syncthreads();
            const uint32_t nneed = s_nneed;
            for (uint32_t k = tid; k < nneed; k += GALL_THREADS) {
                const uint32_t v = T.q_need[k];
                if (g.cin_off[v + 1] > g.cin_off[v] && w_zero_step2(g, T, v) && !(atomicOr(&T.flags[v], GC_Z2) & GC_Z2))
                    T.q_z2[atomicAdd(&s_nz2, 1u)] = v;
            }
            block_bfs(T.q_z2, &s_nz2, g.V, A.status, [&](uint32_t v, auto push) {
                for (uint32_t j = g.cin_off[v]; j < g.cin_off[v + 1]; ++j) {
                    const uint32_t e = g.cin_edge[j];
                    bit_set(B.wpos, e);                                  // weight 1 (FIXUP2)
                    const uint32_t u = g.cnode_of_func[g.cs_caller[e]];
                    if (g.cin_off[u + 1] > g.cin_off[u] && !(T.flags[u] & GC_Z2) && w_zero_step2(g, T, u) &&
                        !(atomicOr(&T.flags[u], GC_Z2) & GC_Z2))
                        push(u);
                }
            });
            // ---- nodes of nonzero inclusive cost: upward from the nodes with
            // samples through call sites of nonzero weight; on the way each
            // node's incoming weight, its call sites' ratios and row bits
            for (uint32_t k = tid; k < nexcl; k += GALL_THREADS) {
                const uint32_t v = T.q_excl[k];
                bit_set(B.clos, v);
                T.q_clos[k] = v;
            }
            if (tid == 0) s_nclos = nexcl;
            block_bfs(T.q_clos, &s_nclos, g.V, A.status, [&](uint32_t v, auto push) {
                unsigned long long W = 0;
                for (uint32_t j = g.cin_off[v]; j < g.cin_off[v + 1]; ++j) W += w2_of(T, B, g.cin_edge[j]);
                if (!W) return;
                const float Wf = __ull2float_rn(W);
                for (uint32_t j = g.cin_off[v]; j < g.cin_off[v + 1]; ++j) {
                    const uint32_t e = g.cin_edge[j];
                    const unsigned long long w = w2_of(T, B, e);
                    if (!w) continue;
                    T.ratio[e] = __fdiv_rn(__ull2float_rn(w), Wf);   // correctly rounded below 2^24
                    bit_set(B.erow, e);
                    const uint32_t u = g.cnode_of_func[g.cs_caller[e]];
                    if (!bit_set(B.clos, u)) push(u);
                }
            });
            // ---- row counts and the node rows' popcount prefix
            n_rows = block_prefix_sum(B.wv, [&](uint32_t i) -> uint32_t { return __popc(B.clos[i]); },
                                      [&](uint32_t i, uint32_t r) { B.npre[i] = r; }, sw);
            uint32_t ne = 0;
            for (uint32_t i = tid; i < B.we; i += GALL_THREADS) ne += __popc(B.erow[i]);
            uint32_t tot;
            block_exclusive_scan<uint32_t, GALL_THREADS>(ne, sw, &tot);
            n_edges = tot;
        }
        // ---- offsets of this context's rows
        if (tid == 0) {
            s_nbase = ctx_lookback(A.look_n, c, n_rows, limit, A.status);
            s_ebase = ctx_lookback(A.look_e, c, n_edges, limit, A.status);
        }
        __syncthreads();
        const unsigned long long nb = s_nbase, eb = s_ebase;
        if (tid == 0) {
            if (O.node_off) O.node_off[c] = nb;
            if (O.edge_off) O.edge_off[c] = eb;
            if (c == A.n_ctx - 1) {
                if (O.node_off) O.node_off[A.n_ctx] = nb + n_rows;
                if (O.edge_off) O.edge_off[A.n_ctx] = eb + n_edges;
                O.counts[0] = nb + n_rows;
                O.counts[1] = eb + n_edges;
                if ((O.cap_nodes || O.cap_edges) && (nb + n_rows > O.cap_nodes || eb + n_edges > O.cap_edges))
                    raise_status(A.status, 4 /* HPA_E_CAPACITY */, 0);
            }
        }
        const bool fits = k1 > k0 && nb + n_rows <= O.cap_nodes && eb + n_edges <= O.cap_edges;
        if (fits) {
            // ---- node rows (bitmap order = id order)
            for (uint32_t i = tid; i < B.wv; i += GALL_THREADS) {
                uint32_t m = B.clos[i], r = B.npre[i];
                while (m) {
                    const uint32_t b = __ffs(m) - 1;
                    m &= m - 1;
                    O.node_id[nb + r++] = i * 32 + b;
                }
            }
            // ---- call-site rows in id order
            block_prefix_sum(B.we, [&](uint32_t i) -> uint32_t { return __popc(B.erow[i]); },
                             [&](uint32_t i, uint32_t r) {
                                 uint32_t m = B.erow[i];
                                 while (m) {
                                     const uint32_t b = __ffs(m) - 1;
                                     m &= m - 1;
                                     const uint32_t e = i * 32 + b, f = g.cs_callee[e], h = g.cs_head[e];
                                     // site 114: call-site row
                                     if (!in_bounds(A.status, eb + r, O.cap_edges, 114)) break;
                                     O.edge_id[eb + r] = e;
                                     O.ratio[eb + r] = T.ratio[e];
                                     uint8_t fl = 0;
                                     if (T.flags[f] & GF_Z) fl |= HPA_EDGE_FIXUP;
                                     if (T.flags[h] & GC_Z2) fl |= HPA_EDGE_FIXUP2;
                                     O.flags[eb + r] = fl;
                                     ++r;
                                 }
                             },
                             sw);
            // ---- sweep lists: the nodes bucketed by level, their active out-edges
            for (uint32_t l = tid; l <= g.n_levels; l += GALL_THREADS) B.lev[l] = 0;
            __syncthreads();
            const uint32_t ncl = n_rows;
            for (uint32_t k = tid; k < ncl; k += GALL_THREADS) atomicAdd(&B.lev[g.level_of[T.q_clos[k]]], 1u);
            __syncthreads();
            if (tid == 0) {
                uint32_t run = 0;
                for (uint32_t l = 0; l <= g.n_levels; ++l) { const uint32_t x = B.lev[l]; B.lev[l] = run; run += x; }
            }
            __syncthreads();
            for (uint32_t k = tid; k < ncl; k += GALL_THREADS) {
                const uint32_t v = T.q_clos[k];
                const uint32_t p = atomicAdd(&B.lev[g.level_of[v]], 1u);
                if (!in_bounds(A.status, p, ncl, 113)) continue;               // site 113: sweep list
                T.cl_node[p] = v;
                T.cl_row[p] = node_rank(B, v);
            }
            __syncthreads();
            // (B.lev[l] now holds the end of level l, which is where level l + 1 starts)
            const uint32_t n_ce = block_prefix_sum(
                ncl,
                [&](uint32_t k) -> uint32_t {
                    const uint32_t v = T.cl_node[k];
                    uint32_t a = 0;
                    for (uint32_t j = g.cout_off[v]; j < g.cout_off[v + 1]; ++j) a += bit_get(B.erow, g.cout_edge[j]);
                    return a;
                },
                [&](uint32_t k, uint32_t r) { T.ce_off[k] = r; }, sw);
            if (tid == 0) T.ce_off[ncl] = n_ce;
            __syncthreads();
            for (uint32_t k = tid; k < ncl; k += GALL_THREADS) {
                const uint32_t v = T.cl_node[k];
                uint32_t o = T.ce_off[k];
                for (uint32_t j = g.cout_off[v]; j < g.cout_off[v + 1]; ++j) {
                    const uint32_t e = g.cout_edge[j];
                    if (bit_get(B.erow, e)) {
                        T.ce_ratio[o] = T.ratio[e];
                        T.ce_hrow[o] = node_rank(B, g.cout_head[j]);
                        ++o;
                    }
                }
            }
            __syncthreads();
            // ---- step 4: level by level, one thread per (node, stall column)
            float* incl = O.incl + (size_t)nb * M;
            for (uint32_t lev = 0; lev < g.n_levels; ++lev) {
                const uint32_t c0 = lev ? B.lev[lev - 1] : 0u, nk = B.lev[lev] - c0;
                for (uint32_t it = tid; it < nk * M; it += GALL_THREADS) {
                    const uint32_t k = c0 + it / M, r = it % M;
                    const uint32_t v = T.cl_node[k];
                    const uint32_t e0 = T.ce_off[k], e1 = T.ce_off[k + 1];
                    float hi = 0.0f, lo = 0.0f;
                    if (T.flags[v] & GC_EXCL) {
                        unsigned long long x = 0;
                        if (r < S) x = T.excl[(size_t)v * S + r];
                        else for (uint32_t q = 0; q < S; ++q) x += T.excl[(size_t)v * S + q];
                        df_from_u64(x, hi, lo);
                    }
                    for (uint32_t j = e0; j < e1; j += 4) {
                        float q[4], x[4];
                        uint32_t hr[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (j + u < e1) { q[u] = T.ce_ratio[j + u]; hr[u] = T.ce_hrow[j + u]; }
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (j + u < e1) x[u] = incl[(size_t)hr[u] * M + r];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (j + u < e1) df_add_prod(hi, lo, q[u], x[u]);
                    }
                    if (in_bounds(A.status, T.cl_row[k], ncl, 115))          // site 115: node row
                        incl[(size_t)T.cl_row[k] * M + r] = __fadd_rn(hi, lo);
                }
                __syncthreads();
            }
            // ---- shares: a(e) = r(e) * incl(head(e)), if requested
            if (O.a) {
                for (uint64_t it = tid; it < (uint64_t)n_edges * M; it += GALL_THREADS) {
                    const uint32_t row = (uint32_t)(it / M), r = (uint32_t)(it % M);
                    const uint32_t e = O.edge_id[eb + row];
                    O.a[(eb + row) * M + r] = __fmul_rn(T.ratio[e], incl[(size_t)node_rank(B, g.cs_head[e]) * M + r]);
                }
            }
        }
        // ---- the next context starts with no measured call-site weight
        if (k1 > k0) {
            __syncthreads();
            for (uint32_t t = tid; t < s_ntouch; t += GALL_THREADS) T.wmeas[T.touched[t]] = 0;
        }
        __syncthreads();
    }
}

}  // namespace hpa

using namespace hpa;

extern "C" hpa_status hpa_apportion_all(hpa_handle* h, uint32_t binary_id, const hpa_profile* p, hpa_gpucct_all* out) {
    hpa::Trace trace_("hpa.apportion_all");
    if (!h || !p || !out) return HPA_E_INVALID_ARG;
    cudaSetDevice(h->device);
    Binary* B = h->binary(binary_id);
    if (!B) return h->fail(HPA_E_INVALID_ARG, "no binary %u", binary_id);
    if (!p->n_keys || (p->capacity && (!p->key_ctx || !p->key_node || !p->key_stall || !p->val)))
        return h->fail(HPA_E_INVALID_ARG, "profile arrays missing");
    if (p->n_stall == 0 || p->n_stall > HPA_MAX_STALL || p->n_ctx == 0)
        return h->fail(HPA_E_INVALID_ARG, "profile has no n_ctx / n_stall (produce it with hpa_attribute_samples)");
    if (!out->counts) return h->fail(HPA_E_INVALID_ARG, "counts array missing");
    if (out->cap_nodes && (!out->node_id || !out->incl))
        return h->fail(HPA_E_INVALID_ARG, "node row arrays missing");
    if (out->cap_edges && (!out->edge_id || !out->ratio || !out->flags))
        return h->fail(HPA_E_INVALID_ARG, "edge row arrays missing");
    const DevCallGraph& g = B->cg;
    if (g.F == 0) return h->fail(HPA_E_INVALID_ARG, "binary has no functions");
    GallArgs A{};
    A.g = g;
    A.key_ctx = p->key_ctx; A.key_node = p->key_node; A.key_stall = p->key_stall; A.key_val = p->val;
    A.n_keys = p->n_keys; A.key_cap = p->capacity;
    A.n_ctx = p->n_ctx; A.S = p->n_stall; A.M = p->n_stall + 1;
    A.out = *out;
    A.timeout_iters = h->opt.timeout_iters;
    A.status = h->d_status;
    A.slot_bytes = gall_layout(g, A.S, nullptr, nullptr);
    const size_t bits_bytes = gall_bits_words(g) * 4;
    A.smem_bits = bits_bytes <= GALL_SMEM_MAX ? 1u : 0u;
    const uint32_t grid = std::max<uint32_t>(1, std::min<uint32_t>(p->n_ctx, (uint32_t)h->sms * GALL_PER_SM));
    // scratch: per-CTA slots, then context starts, look-back words and the ticket
    Carve probe{nullptr};
    probe.take<char>(A.slot_bytes * grid);
    probe.take<uint64_t>((size_t)p->n_ctx + 1);
    probe.take<unsigned long long>(p->n_ctx);
    probe.take<unsigned long long>(p->n_ctx);
    probe.take<uint32_t>(1);
    hpa_status st = h->ensure_scratch(probe.off + 256);
    if (st) return st;
    Carve c{(char*)h->scratch};
    A.slots = c.take<char>(A.slot_bytes * grid);
    uint64_t* start = c.take<uint64_t>((size_t)p->n_ctx + 1);
    A.ctx_start = start;
    A.look_n = c.take<unsigned long long>(p->n_ctx);
    A.look_e = c.take<unsigned long long>(p->n_ctx);
    A.ticket = c.take<uint32_t>(1);
    cudaStream_t s = h->stream;
    cudaMemsetAsync(A.look_n, 0, sizeof(unsigned long long) * p->n_ctx, s);
    cudaMemsetAsync(A.look_e, 0, sizeof(unsigned long long) * p->n_ctx, s);
    cudaMemsetAsync(A.ticket, 0, sizeof(uint32_t), s);
    const int bb = (int)std::max<uint64_t>(1, std::min<uint64_t>((p->capacity + 256) / 256, (uint64_t)h->sms * 8));
    k_ctx_bounds<<<bb, 256, 0, s>>>(p->key_ctx, p->n_keys, p->capacity, p->n_ctx, start);
    const size_t dsm = A.smem_bits ? bits_bytes : 0;
    if (dsm) set_smem_limit((const void*)k_gpucct_all, (int)dsm);
    k_gpucct_all<<<grid, GALL_THREADS, dsm, s>>>(A);
    h->launches += 2;
    return h->cuda(cudaGetLastError(), "apportion (every context) launch");
}
