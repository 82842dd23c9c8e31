// GPU calling context trees of every launch context of a profile (Section
// 6.3, steps 1-4) as sparse rows: per context, the condensed nodes whose
// inclusive cost is not zero and the call sites whose share is not zero --
// the part of the call graph above the context's sampled functions.
//
// One CTA per context at a time, contexts taken in order from a counter:
//  step 1  the context's keys give the exclusive cost of each condensed node
//          (exact 64-bit sums per stall reason) and the measured weight of
//          each call site (samples at its call instruction, all stall
//          reasons); a per-CTA list of the touched call sites resets them;
//  step 2  functions with samples and no measured incoming weight get weight
//          1 on every incoming call site, repeated through their callers that
//          have no measured incoming weight (frontier-parallel closure);
//  step 3  static condensation (Tarjan at load); a condensed node with cost or
//          a member in the step-2 closure whose incoming weight is still zero
//          gets the same rule on the condensed graph (FIXUP2);
//  rows    a condensed node has a nonzero inclusive cost iff it has cost
//          itself or an outgoing call site of nonzero weight into a node with
//          nonzero inclusive cost (found level by level, sinks first); the
//          rows of the context are those nodes and those call sites, in id
//          order; a look-back over the contexts gives their offsets;
//  step 4  level by level, one thread per (node, stall column):
//          incl(v) = excl(v) + sum_e r(e) * incl(head(e)), r(e) = w(e) / W(head),
//          accumulated in double-float arithmetic (error-free products and
//          sums of float pairs) from the float rows of the heads, which are the
//          output rows themselves; each stored value is rounded once to float.
// Contexts without keys have no rows and cost a counter step.

#include <algorithm>

#include "hpa_host.h"

namespace hpa {

// several contexts per SM, so that one context's level-synchronous steps (a
// barrier and a chain of dependent loads per level) overlap another's work
constexpr int GALL_THREADS = 256;
constexpr int GALL_PER_SM = 4;

// per-node / per-function flags of one context (u32 words, atomicOr)
enum : uint32_t {
    GF_HAS = 1,      // function: samples (S(f) > 0)
    GF_MEAS = 2,     // function: a measured incoming call-site weight
    GF_Z = 4,        // function: in the step-2 closure
    GC_NEED = 8,     // condensed node: cost or a member in the step-2 closure
    GC_Z2 = 16,      // condensed node: in the FIXUP2 closure
    GC_EXCL = 32,    // condensed node: exclusive cost (keys with a value)
    GC_CLOS = 64     // condensed node: nonzero inclusive cost
};

struct GallSlot {
    uint32_t* flags;             // [V]
    uint32_t* rowmap;            // [V] row of a node within its context
    unsigned long long* wmeas;   // [E] measured call-site weights (reset through `touched`)
    uint32_t* touched;           // [E]
    unsigned long long* excl;    // [V][S] rows of GC_EXCL nodes
    unsigned long long* Wc;      // [V] incoming weight of GC_CLOS nodes
    float* ratio;                // [E] r(e) of the context's edge rows
    uint8_t* wpos;               // [E] w(e) > 0 after steps 2 and 3, by call site
    uint8_t* wpos_c;             // [E] the same in cout order
    uint32_t* front[2];          // [max(F, V)]
    // the step-4 sweep's lists: nodes with nonzero inclusive cost in level
    // order, each with its active out-edges (ratio, row of the head)
    uint32_t* cl_node;           // [V]
    uint32_t* cl_off;            // [n_levels + 1]
    uint32_t* ce_off;            // [V + 1]
    float* ce_ratio;             // [E]
    uint32_t* ce_hrow;           // [E]
    uint32_t* pos_pre;           // [V + 1] prefix counts over level positions
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
    unsigned long long* look_e;      // [n_ctx] look-back words (edge rows)
    uint32_t* ticket;
    char* slots;
    size_t slot_bytes;
    uint32_t timeout_iters;
    DevStatus* status;
};

__host__ __device__ inline size_t gall_layout(const DevCallGraph& g, uint32_t S, char* base, GallSlot* s) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~size_t(255);
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const size_t FV = g.F > g.V ? g.F : g.V;
    GallSlot t;
    t.flags = (uint32_t*)take((size_t)g.V * 4);
    t.rowmap = (uint32_t*)take((size_t)g.V * 4);
    t.wmeas = (unsigned long long*)take((size_t)g.E * 8 + 8);
    t.touched = (uint32_t*)take((size_t)g.E * 4 + 4);
    t.excl = (unsigned long long*)take((size_t)g.V * S * 8);
    t.Wc = (unsigned long long*)take((size_t)g.V * 8);
    t.ratio = (float*)take((size_t)g.E * 4 + 4);
    t.wpos = (uint8_t*)take((size_t)g.E + 4);
    t.wpos_c = (uint8_t*)take((size_t)g.E + 4);
    t.front[0] = (uint32_t*)take(FV * 4);
    t.front[1] = (uint32_t*)take(FV * 4);
    t.cl_node = (uint32_t*)take((size_t)g.V * 4 + 4);
    t.cl_off = (uint32_t*)take((size_t)g.n_levels * 4 + 8);
    t.ce_off = (uint32_t*)take((size_t)g.V * 4 + 8);
    t.ce_ratio = (float*)take((size_t)g.E * 4 + 4);
    t.ce_hrow = (uint32_t*)take((size_t)g.E * 4 + 4);
    t.pos_pre = (uint32_t*)take((size_t)g.V * 4 + 8);
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

// the look-back of the fused leaves, over contexts: publish this context's
// row count, add up the counts before it until a published inclusive prefix
// (context 0 publishes one at once); bounded waits
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

// weight of call site e after steps 2 and 3 (external edges only)
__device__ __forceinline__ unsigned long long w2_of(const DevCallGraph& g, const GallSlot& T, uint32_t e) {
    const unsigned long long w = T.wmeas[e];
    if (w) return w;
    const uint32_t f = g.cs_callee[e];
    if (T.flags[f] & GF_Z) return 1ull;
    return (T.flags[g.cnode_of_func[f]] & GC_Z2) ? 1ull : 0ull;
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

// Block-wide exclusive prefix counts of pred over the items [0, n), in id
// order: each thread takes a contiguous chunk; put(i, prefix) for every item
// (all = true) or only for the items satisfying pred.  Returns the count.
template <bool ALL, typename P, typename PUT>
__device__ uint32_t block_prefix(uint32_t n, P pred, PUT put, uint32_t* sw) {
    const uint32_t per = (n + GALL_THREADS - 1) / GALL_THREADS;
    const uint32_t a = min(n, threadIdx.x * per), b = min(n, a + per);
    uint32_t c = 0;
    for (uint32_t i = a; i < b; ++i) c += pred(i) ? 1u : 0u;
    uint32_t tot;
    uint32_t r = block_exclusive_scan<uint32_t, GALL_THREADS>(c, sw, &tot);
    for (uint32_t i = a; i < b; ++i) {
        const bool p = pred(i);
        if (ALL || p) put(i, r);
        r += p ? 1u : 0u;
    }
    return tot;
}

// Block-wide exclusive prefix sums of cnt(i) over the items [0, n), in id
// order: put(i, sum of cnt over the items before i).  Returns the total.
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

__global__ void __launch_bounds__(GALL_THREADS, GALL_PER_SM) k_gpucct_all(GallArgs A) {
    const DevCallGraph& g = A.g;
    __shared__ uint32_t sw[33];
    __shared__ uint32_t s_c, s_cnt[2], s_ntouch;
    __shared__ unsigned long long s_nbase, s_ebase;
    GallSlot T;
    gall_layout(g, A.S, A.slots + (size_t)blockIdx.x * A.slot_bytes, &T);
    const uint32_t tid = threadIdx.x;
    const uint32_t S = A.S, M = A.M;
    const uint32_t limit = A.timeout_iters ? A.timeout_iters : (1u << 22);
    const hpa_gpucct_all& O = A.out;
    const uint32_t n_pos = g.level_off[g.n_levels];     // live condensed nodes, in level order
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
            if (tid == 0) s_ntouch = 0;
            __syncthreads();
            for (uint64_t i = k0 + tid; i < k1; i += GALL_THREADS) {
                const uint32_t n = A.key_node[i];
                if (n == UNKNOWN) continue;
                const uint32_t r = A.key_stall[i];
                if (n >= g.M || r >= S) { raise_status(A.status, 1 /* HPA_E_INVALID_ARG */, 13); continue; }
                const unsigned long long v = A.key_val[i];
                if (!v) continue;
                const uint32_t f = g.node_func[n];
                atomicOr(&T.flags[f], GF_HAS);
                atomicOr(&T.flags[g.cnode_of_func[f]], GC_EXCL);
                const uint32_t e = g.node_cs[n];
                if (e != UNKNOWN && atomicAdd(&T.wmeas[e], v) == 0ull) T.touched[atomicAdd(&s_ntouch, 1u)] = e;
            }
            __syncthreads();
            const uint32_t ntouch = s_ntouch;
            for (uint32_t v = tid; v < g.V; v += GALL_THREADS)
                if (T.flags[v] & GC_EXCL)
                    for (uint32_t r = 0; r < S; ++r) T.excl[(size_t)v * S + r] = 0;
            for (uint32_t t = tid; t < ntouch; t += GALL_THREADS) atomicOr(&T.flags[g.cs_callee[T.touched[t]]], GF_MEAS);
            __syncthreads();
            for (uint64_t i = k0 + tid; i < k1; i += GALL_THREADS) {
                const uint32_t n = A.key_node[i];
                const uint32_t r = A.key_stall[i];
                if (n == UNKNOWN || n >= g.M || r >= S) continue;
                atomicAdd(&T.excl[(size_t)g.cnode_of_func[g.node_func[n]] * S + r], (unsigned long long)A.key_val[i]);
            }
            // ---- step 2: zero-weight fix-up, closure through callers
            if (tid == 0) s_cnt[0] = 0;
            __syncthreads();
            for (uint32_t f = tid; f < g.F; f += GALL_THREADS) {
                const uint32_t fl = T.flags[f];
                if ((fl & GF_HAS) && !(fl & GF_MEAS) && g.fin_off[f + 1] > g.fin_off[f]) {
                    atomicOr(&T.flags[f], GF_Z);
                    T.front[0][atomicAdd(&s_cnt[0], 1u)] = f;
                }
            }
            __syncthreads();
            int cur = 0;
            for (;;) {
                const uint32_t cnt = s_cnt[cur];
                if (cnt == 0) break;
                if (tid == 0) s_cnt[cur ^ 1] = 0;
                __syncthreads();
                for (uint32_t k = tid; k < cnt; k += GALL_THREADS) {
                    const uint32_t f = T.front[cur][k];
                    for (uint32_t j = g.fin_off[f]; j < g.fin_off[f + 1]; ++j) {
                        const uint32_t h = g.cs_caller[g.fin_edge[j]];
                        if (g.fin_off[h + 1] > g.fin_off[h] && !(T.flags[h] & GF_MEAS) &&
                            !(atomicOr(&T.flags[h], GF_Z) & GF_Z))
                            T.front[cur ^ 1][atomicAdd(&s_cnt[cur ^ 1], 1u)] = h;
                    }
                }
                __syncthreads();
                cur ^= 1;
            }
            // ---- step 3: FIXUP2 on the condensed graph
            for (uint32_t f = tid; f < g.F; f += GALL_THREADS)
                if (T.flags[f] & (GF_HAS | GF_Z)) atomicOr(&T.flags[g.cnode_of_func[f]], GC_NEED);
            if (tid == 0) s_cnt[0] = 0;
            __syncthreads();
            for (uint32_t v = tid; v < g.V; v += GALL_THREADS)
                if (g.cnode_live[v] && (T.flags[v] & GC_NEED) && g.cin_off[v + 1] > g.cin_off[v] &&
                    w_zero_step2(g, T, v)) {
                    atomicOr(&T.flags[v], GC_Z2);
                    T.front[0][atomicAdd(&s_cnt[0], 1u)] = v;
                }
            __syncthreads();
            cur = 0;
            for (;;) {
                const uint32_t cnt = s_cnt[cur];
                if (cnt == 0) break;
                if (tid == 0) s_cnt[cur ^ 1] = 0;
                __syncthreads();
                for (uint32_t k = tid; k < cnt; k += GALL_THREADS) {
                    const uint32_t v = T.front[cur][k];
                    for (uint32_t j = g.cin_off[v]; j < g.cin_off[v + 1]; ++j) {
                        const uint32_t u = g.cnode_of_func[g.cs_caller[g.cin_edge[j]]];
                        if (g.cin_off[u + 1] > g.cin_off[u] && !(T.flags[u] & GC_Z2) && w_zero_step2(g, T, u) &&
                            !(atomicOr(&T.flags[u], GC_Z2) & GC_Z2))
                            T.front[cur ^ 1][atomicAdd(&s_cnt[cur ^ 1], 1u)] = u;
                    }
                }
                __syncthreads();
                cur ^= 1;
            }
            // ---- call sites of nonzero weight (by id and in cout order)
            for (uint32_t e = tid; e < g.E; e += GALL_THREADS)
                T.wpos[e] = (!g.edge_intra[e] && w2_of(g, T, e)) ? 1 : 0;
            __syncthreads();
            for (uint32_t j = tid; j < g.cout_off[g.V]; j += GALL_THREADS) T.wpos_c[j] = T.wpos[g.cout_edge[j]];
            __syncthreads();
            // ---- nodes with nonzero inclusive cost, level by level (sinks first)
            for (uint32_t lev = 0; lev < g.n_levels; ++lev) {
                for (uint32_t k = g.level_off[lev] + tid; k < g.level_off[lev + 1]; k += GALL_THREADS) {
                    const uint32_t v = g.level_node[k];
                    bool clos = (T.flags[v] & GC_EXCL) != 0;
                    for (uint32_t j = g.cout_off[v]; !clos && j < g.cout_off[v + 1]; ++j)
                        clos = T.wpos_c[j] && (T.flags[g.cout_head[j]] & GC_CLOS);
                    if (clos) atomicOr(&T.flags[v], GC_CLOS);
                }
                __syncthreads();
            }
            // ---- rows: nodes and call sites in id order, incoming weights
            auto node_row = [&](uint32_t v) { return g.cnode_live[v] && (T.flags[v] & GC_CLOS); };
            n_rows = block_prefix<false>(g.V, node_row, [&](uint32_t v, uint32_t r) { T.rowmap[v] = r; }, sw);
            auto edge_row = [&](uint32_t e) {
                return T.wpos[e] && (T.flags[g.cnode_of_func[g.cs_callee[e]]] & GC_CLOS);
            };
            n_edges = block_prefix<false>(g.E, edge_row, [](uint32_t, uint32_t) {}, sw);
            for (uint32_t v = tid; v < g.V; v += GALL_THREADS)
                if (node_row(v)) {
                    unsigned long long W = 0;
                    for (uint32_t j = g.cin_off[v]; j < g.cin_off[v + 1]; ++j) W += w2_of(g, T, g.cin_edge[j]);
                    T.Wc[v] = W;
                }
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
            // ---- node and edge rows
            for (uint32_t v = tid; v < g.V; v += GALL_THREADS)
                if (g.cnode_live[v] && (T.flags[v] & GC_CLOS)) O.node_id[nb + T.rowmap[v]] = v;
            auto edge_row = [&](uint32_t e) {
                return T.wpos[e] && (T.flags[g.cnode_of_func[g.cs_callee[e]]] & GC_CLOS);
            };
            block_prefix<false>(g.E, edge_row,
                                [&](uint32_t e, uint32_t r) {
                                    const uint32_t f = g.cs_callee[e], h = g.cnode_of_func[f];
                                    const unsigned long long w = w2_of(g, T, e), W = T.Wc[h];
                                    const float q = __fdiv_rn(__ull2float_rn(w), __ull2float_rn(W));
                                    T.ratio[e] = q;
                                    O.edge_id[eb + r] = e;
                                    O.ratio[eb + r] = q;
                                    uint8_t fl = 0;
                                    if (T.flags[f] & GF_Z) fl |= HPA_EDGE_FIXUP;
                                    if (T.flags[h] & GC_Z2) fl |= HPA_EDGE_FIXUP2;
                                    O.flags[eb + r] = fl;
                                },
                                sw);
            // ---- sweep lists: nonzero nodes in level order, their active out-edges
            const uint32_t n_cl = block_prefix<true>(
                n_pos, [&](uint32_t k) { return (T.flags[g.level_node[k]] & GC_CLOS) != 0; },
                [&](uint32_t k, uint32_t r) {
                    T.pos_pre[k] = r;
                    const uint32_t v = g.level_node[k];
                    if (T.flags[v] & GC_CLOS) T.cl_node[r] = v;
                },
                sw);
            if (tid == 0) T.pos_pre[n_pos] = n_cl;
            __syncthreads();
            for (uint32_t lev = tid; lev <= g.n_levels; lev += GALL_THREADS) T.cl_off[lev] = T.pos_pre[g.level_off[lev]];
            const uint32_t n_ce = block_prefix_sum(
                n_cl,
                [&](uint32_t k) -> uint32_t {
                    const uint32_t v = T.cl_node[k];
                    uint32_t a = 0;
                    for (uint32_t j = g.cout_off[v]; j < g.cout_off[v + 1]; ++j)
                        a += (T.wpos_c[j] && (T.flags[g.cout_head[j]] & GC_CLOS)) ? 1u : 0u;
                    return a;
                },
                [&](uint32_t k, uint32_t r) { T.ce_off[k] = r; }, sw);
            if (tid == 0) T.ce_off[n_cl] = n_ce;
            __syncthreads();
            for (uint32_t k = tid; k < n_cl; k += GALL_THREADS) {
                const uint32_t v = T.cl_node[k];
                uint32_t o = T.ce_off[k];
                for (uint32_t j = g.cout_off[v]; j < g.cout_off[v + 1]; ++j) {
                    const uint32_t hd = g.cout_head[j];
                    if (T.wpos_c[j] && (T.flags[hd] & GC_CLOS)) {
                        T.ce_ratio[o] = T.ratio[g.cout_edge[j]];
                        T.ce_hrow[o] = T.rowmap[hd];
                        ++o;
                    }
                }
            }
            __syncthreads();
            // ---- step 4: level by level, one thread per (node, stall column)
            float* incl = O.incl + (size_t)nb * M;
            for (uint32_t lev = 0; lev < g.n_levels; ++lev) {
                const uint32_t c0 = T.cl_off[lev], nk = T.cl_off[lev + 1] - c0;
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
                    incl[(size_t)T.rowmap[v] * M + r] = __fadd_rn(hi, lo);
                }
                __syncthreads();
            }
            // ---- shares: a(e) = r(e) * incl(head(e)), if requested
            if (O.a) {
                for (uint64_t it = tid; it < (uint64_t)n_edges * M; it += GALL_THREADS) {
                    const uint32_t row = (uint32_t)(it / M), r = (uint32_t)(it % M);
                    const uint32_t e = O.edge_id[eb + row];
                    const uint32_t hd = g.cnode_of_func[g.cs_callee[e]];
                    O.a[(eb + row) * M + r] = __fmul_rn(T.ratio[e], incl[(size_t)T.rowmap[hd] * M + r]);
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
    k_gpucct_all<<<grid, GALL_THREADS, 0, s>>>(A);
    h->launches += 2;
    return h->cuda(cudaGetLastError(), "apportion (every context) launch");
}
