// CPU oracle for GPU PC-sample analysis (arXiv 2109.06931).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
// statement of what the CUDA library computes.  Only the test suite, the
// smoke check and the benchmark's CPU-baseline leg may load it; the library
// never calls it and shares no code, header or table with it.
//
// Every function follows one passage of the paper, cited beside it:
//   Section 4.2   a PC sample = (instruction address, stall reason, count);
//                 it becomes a GPU-instruction node under the kernel's context.
//   Section 4.5   a raw metric is the sum of all measured values of a kind
//                 in a context; post-mortem derived metrics are sum, min,
//                 mean, max, std. deviation and coefficient of variation;
//                 a per-invocation quantity is the ratio of two summed raw
//                 metrics.
//   Section 5     instructions map to lines, loops, inlined code, functions.
//   Section 6.1   statistic generation propagates values up the calling
//                 context tree (inclusive metrics).
//   Section 6.3   GPU calling context tree, steps 1-4 (call-graph weights,
//                 zero-weight fix-up, SCC collapse, gprof-style splitting).
//   Section 7     warp issue rate W = (S - S_stall) / S, per context and per
//                 (context, function).
// Readings of points the paper leaves open are stated where they are used.
//
// Floating point is double precision throughout; counts are exact uint64.
// Parity status: every entry point is pinned by tests against brute force,
// closed forms or hand-computed cases (no "parity unpinned" function).

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <tuple>
#include <vector>
#include <algorithm>

namespace {

const uint32_t UNKNOWN = 0xFFFFFFFFu;   // attribution of a PC in no range
const uint32_t NO_PARENT = 0xFFFFFFFFu;

const int OK = 0, INVALID_ARG = 1, INVALID_TABLE = 2, INVALID_SAMPLE = 3;

typedef std::tuple<uint32_t, uint32_t, uint32_t> Key;   // (ctx, node, stall)

// A sorted key -> value list handed back to the caller.
struct KeyList {
    std::vector<uint32_t> ctx, node, stall;
    std::vector<uint64_t> val;
    std::vector<uint64_t> total, unknown;   // per stall reason (attribution only)
    int status = OK;
    uint64_t bad = 0;
};

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// O1 + O2: attribution (Section 4.2, Section 5) and raw-metric aggregation
// (Section 4.5).
//
// O1: for each sample, the range is the last one with lo <= pc (ranges are
//     sorted by lo and disjoint); the sample belongs to that range's node if
//     pc < hi (half-open ranges), else to UNKNOWN.
// O2: raw metric of key (ctx, node, stall) = sum of the counts of its samples;
//     a missing count array means every record counts 1; keys whose sum is 0
//     are omitted.  Any record with ctx >= n_ctx or stall >= n_stall fails the
//     whole call (status INVALID_SAMPLE, number of bad records in `bad`).
void* orc_attribute(uint64_t n_ranges, const uint64_t* range_lo, const uint64_t* range_hi,
                    const uint32_t* range_node, uint64_t n, const uint64_t* pc,
                    const uint32_t* ctx, const uint8_t* stall, const uint32_t* count,
                    uint32_t n_ctx, uint32_t n_stall) {
    KeyList* out = new KeyList();
    out->total.assign(n_stall, 0);
    out->unknown.assign(n_stall, 0);
    for (uint64_t i = 0; i < n; ++i)
        if (ctx[i] >= n_ctx || stall[i] >= n_stall) out->bad++;
    if (out->bad) { out->status = INVALID_SAMPLE; return out; }

    std::map<Key, uint64_t> agg;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t* it = std::upper_bound(range_lo, range_lo + n_ranges, pc[i]);
        uint32_t node = UNKNOWN;
        if (it != range_lo) {
            uint64_t j = (uint64_t)(it - range_lo) - 1;
            if (pc[i] < range_hi[j]) node = range_node[j];
        }
        uint64_t c = count ? count[i] : 1;
        agg[Key(ctx[i], node, stall[i])] += c;
        out->total[stall[i]] += c;
        if (node == UNKNOWN) out->unknown[stall[i]] += c;
    }
    for (auto& kv : agg) {
        if (kv.second == 0) continue;
        out->ctx.push_back(std::get<0>(kv.first));
        out->node.push_back(std::get<1>(kv.first));
        out->stall.push_back(std::get<2>(kv.first));
        out->val.push_back(kv.second);
    }
    return out;
}

// ---------------------------------------------------------------------------
// O4(a): inclusive metrics over the program-structure tree inside each
// context (Section 6.1, statistic generation: values propagate up the tree).
// Every key's value is added to its node and to every ancestor of that node
// up to the function node (node_parent == NO_PARENT).  UNKNOWN has no
// ancestors and keeps its own value.  Output sorted by (ctx, node, stall).
void* orc_inclusive_structure(uint32_t n_nodes, const uint32_t* node_parent, uint64_t k,
                              const uint32_t* kctx, const uint32_t* knode,
                              const uint8_t* kstall, const uint64_t* kval) {
    KeyList* out = new KeyList();
    std::map<Key, uint64_t> agg;
    for (uint64_t i = 0; i < k; ++i) {
        uint32_t n = knode[i];
        if (n == UNKNOWN) { agg[Key(kctx[i], n, kstall[i])] += kval[i]; continue; }
        if (n >= n_nodes) { out->status = INVALID_ARG; return out; }
        uint32_t steps = 0;
        while (n != NO_PARENT) {
            agg[Key(kctx[i], n, kstall[i])] += kval[i];
            n = node_parent[n];
            if (++steps > n_nodes) { out->status = INVALID_ARG; return out; }
        }
    }
    for (auto& kv : agg) {
        out->ctx.push_back(std::get<0>(kv.first));
        out->node.push_back(std::get<1>(kv.first));
        out->stall.push_back(std::get<2>(kv.first));
        out->val.push_back(kv.second);
    }
    return out;
}

// Flat view (Section 7: costs by static structure regardless of calling
// context): the values of all keys summed per (node, stall), every context
// pooled into context 0; per-stall totals and UNKNOWN totals of the result.
void* orc_flat(uint32_t n_stall, uint64_t k, const uint32_t* knode, const uint8_t* kstall, const uint64_t* kval) {
    KeyList* out = new KeyList();
    std::map<std::pair<uint32_t, uint32_t>, uint64_t> agg;
    for (uint64_t i = 0; i < k; ++i) {
        if (kstall[i] >= n_stall) { out->status = INVALID_ARG; return out; }
        agg[std::make_pair(knode[i], (uint32_t)kstall[i])] += kval[i];
    }
    out->total.assign(n_stall, 0);
    out->unknown.assign(n_stall, 0);
    for (auto& kv : agg) {
        if (!kv.second) continue;                  // a key whose values sum to 0 is omitted
        out->ctx.push_back(0);
        out->node.push_back(kv.first.first);
        out->stall.push_back(kv.first.second);
        out->val.push_back(kv.second);
        out->total[kv.first.second] += kv.second;
        if (kv.first.first == UNKNOWN) out->unknown[kv.first.second] += kv.second;
    }
    return out;
}

// O4(b): inclusive metrics over the host calling-context tree (Section 6.1).
// Launch context c is CCT node c.  host[h][r] = sum of the values of all keys
// (UNKNOWN included) whose context lies in the subtree of h: each key's value
// is added to its context and to every ancestor.  `host` is n_cct x n_stall.
int orc_inclusive_cct(uint32_t n_cct, const uint32_t* cct_parent, uint32_t n_stall, uint64_t k,
                      const uint32_t* kctx, const uint8_t* kstall, const uint64_t* kval,
                      uint64_t* host) {
    std::memset(host, 0, sizeof(uint64_t) * (size_t)n_cct * n_stall);
    for (uint64_t i = 0; i < k; ++i) {
        uint32_t h = kctx[i];
        if (h >= n_cct || kstall[i] >= n_stall) return INVALID_ARG;
        uint32_t steps = 0;
        while (h != NO_PARENT) {
            host[(size_t)h * n_stall + kstall[i]] += kval[i];
            h = cct_parent[h];
            if (++steps > n_cct) return INVALID_ARG;
        }
    }
    return OK;
}

// ---------------------------------------------------------------------------
// O5: derived metrics across P profiles (Section 4.5) and warp issue rate
// (Section 7).
//
// For every key in the union of the P profiles, x_p is the profile's value or
// 0 where the key is absent: sum, min, max, mean = sum / P, population std
// sqrt(sum (x_p - mean)^2 / P) by two passes, CoV = std / mean.
// Per context, over the sum of all profiles: S = all samples, S_issued = the
// samples whose stall reason is in issued_mask (not stalled),
// W = (S - S_stall) / S = S_issued / S (NaN when S = 0), and the fraction of
// S in each stall reason (NaN when S = 0).
struct Derived {
    std::vector<uint32_t> ctx, node, stall;
    std::vector<uint64_t> sum;
    std::vector<double> mn, mx, mean, sd, cov;
    std::vector<uint64_t> S, S_issued;
    std::vector<double> W, frac;
};

void* orc_derive(uint32_t P, const uint64_t* nkeys, const uint32_t* const* kctx,
                 const uint32_t* const* knode, const uint8_t* const* kstall,
                 const uint64_t* const* kval, uint32_t n_ctx, uint32_t n_stall,
                 uint32_t issued_mask) {
    Derived* d = new Derived();
    std::map<Key, std::vector<uint64_t>> u;
    for (uint32_t p = 0; p < P; ++p)
        for (uint64_t i = 0; i < nkeys[p]; ++i) {
            auto& v = u[Key(kctx[p][i], knode[p][i], kstall[p][i])];
            if (v.empty()) v.assign(P, 0);
            v[p] += kval[p][i];
        }
    d->S.assign(n_ctx, 0);
    d->S_issued.assign(n_ctx, 0);
    for (auto& kv : u) {
        const std::vector<uint64_t>& x = kv.second;
        uint64_t s = 0, lo = x[0], hi = x[0];
        for (uint32_t p = 0; p < P; ++p) { s += x[p]; lo = std::min(lo, x[p]); hi = std::max(hi, x[p]); }
        double mean = (double)s / P;
        double ss = 0;
        for (uint32_t p = 0; p < P; ++p) { double e = (double)x[p] - mean; ss += e * e; }
        double sd = std::sqrt(ss / P);
        d->ctx.push_back(std::get<0>(kv.first));
        d->node.push_back(std::get<1>(kv.first));
        d->stall.push_back(std::get<2>(kv.first));
        d->sum.push_back(s);
        d->mn.push_back((double)lo);
        d->mx.push_back((double)hi);
        d->mean.push_back(mean);
        d->sd.push_back(sd);
        d->cov.push_back(sd / mean);
        uint32_t c = std::get<0>(kv.first), r = std::get<2>(kv.first);
        if (c < n_ctx) {
            d->S[c] += s;
            if (r < 32 && ((issued_mask >> r) & 1u)) d->S_issued[c] += s;
        }
    }
    d->W.assign(n_ctx, NAN);
    d->frac.assign((size_t)n_ctx * n_stall, NAN);
    std::vector<uint64_t> per((size_t)n_ctx * n_stall, 0);
    for (auto& kv : u) {
        uint32_t c = std::get<0>(kv.first), r = std::get<2>(kv.first);
        if (c < n_ctx && r < n_stall) {
            uint64_t s = 0;
            for (uint64_t v : kv.second) s += v;
            per[(size_t)c * n_stall + r] += s;
        }
    }
    for (uint32_t c = 0; c < n_ctx; ++c) {
        if (d->S[c] == 0) continue;
        d->W[c] = (double)d->S_issued[c] / (double)d->S[c];
        for (uint32_t r = 0; r < n_stall; ++r)
            d->frac[(size_t)c * n_stall + r] = (double)per[(size_t)c * n_stall + r] / (double)d->S[c];
    }
    return d;
}

// O5 per function: warp issue rate and stall shares per (launch context,
// function) (Section 7 reads W per kernel and per function).  A key counts
// toward (its context, the function of its node); UNKNOWN keys belong to no
// function and are left out.  S = all counts of the pair, S_issued = those
// whose stall reason is in issued_mask, W = S_issued / S, frac[r] = the share
// of S in stall reason r.  One row per pair with S > 0, ascending by
// (context, function).
struct IssueRows {
    std::vector<uint32_t> ctx, func;
    std::vector<uint64_t> S, S_issued;
    std::vector<double> W, frac;
    int status = OK;
};

void* orc_issue_by_function(uint32_t n_nodes, const uint32_t* node_func, uint32_t n_stall, uint32_t issued_mask,
                            uint64_t k, const uint32_t* kctx, const uint32_t* knode, const uint8_t* kstall,
                            const uint64_t* kval) {
    IssueRows* o = new IssueRows();
    std::map<std::pair<uint32_t, uint32_t>, std::vector<uint64_t>> per;   // (ctx, func) -> count per stall
    for (uint64_t i = 0; i < k; ++i) {
        if (knode[i] == UNKNOWN) continue;
        if (knode[i] >= n_nodes || kstall[i] >= n_stall) { o->status = INVALID_ARG; return o; }
        std::vector<uint64_t>& v = per[std::make_pair(kctx[i], node_func[knode[i]])];
        if (v.empty()) v.assign(n_stall, 0);
        v[kstall[i]] += kval[i];
    }
    for (auto& kv : per) {
        uint64_t S = 0, issued = 0;
        for (uint32_t r = 0; r < n_stall; ++r) {
            S += kv.second[r];
            if (r < 32 && ((issued_mask >> r) & 1u)) issued += kv.second[r];
        }
        if (S == 0) continue;
        o->ctx.push_back(kv.first.first);
        o->func.push_back(kv.first.second);
        o->S.push_back(S);
        o->S_issued.push_back(issued);
        o->W.push_back((double)issued / (double)S);
        for (uint32_t r = 0; r < n_stall; ++r) o->frac.push_back((double)kv.second[r] / (double)S);
    }
    return o;
}

// O5 ratio of raw metrics (Section 4.5: a quantity known once per kernel
// invocation, such as its registers, is recovered from two raw metrics that
// are summed over threads and ranks like any other -- the quantity summed
// over invocations and the number of invocations -- by dividing the sums).
// Profiles 0 .. P_num - 1 are the numerator group, the next P_den the
// denominator group.  Per key (context, node, stall) of the union of both
// groups: num = the sum of the numerator group's values (0 where absent),
// den = the same over the denominator group, ratio = num / den (NaN when
// den = 0).  One row per key, ascending.
struct RatioRows {
    std::vector<uint32_t> ctx, node, stall;
    std::vector<uint64_t> num, den;
    std::vector<double> ratio;
};

void* orc_ratio(uint32_t P_num, uint32_t P_den, const uint64_t* nkeys, const uint32_t* const* kctx,
                const uint32_t* const* knode, const uint8_t* const* kstall, const uint64_t* const* kval) {
    RatioRows* o = new RatioRows();
    std::map<Key, std::pair<uint64_t, uint64_t>> u;   // key -> (numerator sum, denominator sum)
    for (uint32_t p = 0; p < P_num + P_den; ++p)
        for (uint64_t i = 0; i < nkeys[p]; ++i) {
            std::pair<uint64_t, uint64_t>& v = u[Key(kctx[p][i], knode[p][i], kstall[p][i])];
            if (p < P_num) v.first += kval[p][i];
            else v.second += kval[p][i];
        }
    for (auto& kv : u) {
        o->ctx.push_back(std::get<0>(kv.first));
        o->node.push_back(std::get<1>(kv.first));
        o->stall.push_back(std::get<2>(kv.first));
        o->num.push_back(kv.second.first);
        o->den.push_back(kv.second.second);
        o->ratio.push_back(kv.second.second == 0 ? NAN : (double)kv.second.first / (double)kv.second.second);
    }
    return o;
}

// ---------------------------------------------------------------------------
// O3: approximate GPU calling context tree (Section 6.3, steps 1-4), per
// launch context c.
//
// Step 1: static call graph from the call sites (one edge per call
//   instruction).  w(e) = samples at e's call instruction (node cs_node[e]),
//   summed over stall reasons, in context c.  excl(f)[r] = samples of c in
//   nodes of f (UNKNOWN excluded); S(f) = sum_r excl(f)[r], which includes
//   f's own call instructions.
// Step 2 ("a function has samples and none of its incoming edges has a
//   non-zero weight ... repeat through callers"): Z0 = {f : S(f) > 0,
//   indeg(f) >= 1, every measured w(in(f)) = 0}; a caller g of a member of Z
//   joins Z when indeg(g) >= 1 and every measured w(in(g)) = 0.  Every edge
//   into a member of Z gets weight 1 (flag FIXUP).  Roots (indeg 0) stop it.
// Step 3: Tarjan's SCCs; a non-trivial SCC (>= 2 members or a self-call) is
//   one condensed node whose exclusive cost is the sum of its members'; its
//   internal edges are dropped (flag INTRA_SCC, a = 0).  Reading for a
//   condensed node left with zero incoming weight although it has cost or
//   holds a member of Z (step 2 precedes step 3 and cannot see this): apply
//   the step-2 rule again on the condensed graph (flag FIXUP2).
// Step 4 (gprof assumption): r(e) = w(e) / W(head), W(v) = incoming weight of
//   v (r = 0 when W = 0); bottom-up over the condensed DAG
//   incl(v) = excl(v) + sum_{e out of v} r(e) incl(head(e)), and
//   a(e) = r(e) incl(head(e)).  Cost that cannot be passed up stays at roots.
//
// Output layout, per requested context (dense): condensed node ids are
// f for a function in a trivial SCC and F + k for the k-th non-trivial SCC
// (SCCs ordered by smallest member); incl[V][n_stall + 1] (last column is the
// total over stall reasons), a[E][n_stall + 1], flags[E].  Rows of functions
// that belong to a non-trivial SCC stay zero.
struct GpuCct {
    uint32_t V = 0;
    std::vector<uint32_t> cnode_of_func;
    std::vector<double> incl, a;
    std::vector<uint8_t> flags;
    int status = OK;
};

enum { F_FIXUP = 1, F_FIXUP2 = 2, F_INTRA = 4 };

// Tarjan's strongly connected components, iterative form of the published
// recursive algorithm (Tarjan 1972).  Returns comp[f] and the components in
// the order Tarjan completes them (every component after all components it
// reaches: reverse topological order of the condensed graph).
static void tarjan(uint32_t F, const std::vector<std::vector<uint32_t>>& succ,
                   std::vector<uint32_t>& comp, std::vector<std::vector<uint32_t>>& comps) {
    std::vector<int64_t> index(F, -1), low(F, 0);
    std::vector<char> on(F, 0);
    std::vector<uint32_t> st;
    comp.assign(F, 0);
    comps.clear();
    int64_t next = 0;
    std::vector<std::pair<uint32_t, size_t>> call;   // (vertex, next successor position)
    for (uint32_t s = 0; s < F; ++s) {
        if (index[s] >= 0) continue;
        call.push_back({s, 0});
        index[s] = low[s] = next++; st.push_back(s); on[s] = 1;
        while (!call.empty()) {
            uint32_t v = call.back().first;
            size_t& pos = call.back().second;
            if (pos < succ[v].size()) {
                uint32_t w = succ[v][pos++];
                if (index[w] < 0) {
                    index[w] = low[w] = next++; st.push_back(w); on[w] = 1;
                    call.push_back({w, 0});
                } else if (on[w]) {
                    low[v] = std::min(low[v], index[w]);
                }
            } else {
                if (low[v] == index[v]) {
                    std::vector<uint32_t> c;
                    uint32_t w;
                    do { w = st.back(); st.pop_back(); on[w] = 0; comp[w] = (uint32_t)comps.size(); c.push_back(w); } while (w != v);
                    comps.push_back(c);
                }
                call.pop_back();
                if (!call.empty()) { uint32_t u = call.back().first; low[u] = std::min(low[u], low[v]); }
            }
        }
    }
}

void* orc_apportion(uint32_t n_nodes, const uint32_t* node_func, uint32_t F, uint32_t E,
                    const uint32_t* cs_caller, const uint32_t* cs_callee, const uint32_t* cs_node,
                    uint32_t n_stall, uint64_t k, const uint32_t* kctx, const uint32_t* knode,
                    const uint8_t* kstall, const uint64_t* kval,
                    uint32_t n_req, const uint32_t* req_ctx) {
    GpuCct* g = new GpuCct();
    const uint32_t M = n_stall + 1;
    // static graph, step 1 / step 3 parts that do not depend on the context
    std::vector<std::vector<uint32_t>> succ(F), in_edges(F);
    std::vector<int64_t> call_of_node(n_nodes, -1);
    for (uint32_t e = 0; e < E; ++e) {
        if (cs_caller[e] >= F || cs_callee[e] >= F || cs_node[e] >= n_nodes) { g->status = INVALID_ARG; return g; }
        succ[cs_caller[e]].push_back(cs_callee[e]);
        in_edges[cs_callee[e]].push_back(e);
        call_of_node[cs_node[e]] = e;
    }
    std::vector<uint32_t> comp;
    std::vector<std::vector<uint32_t>> comps;
    tarjan(F, succ, comp, comps);
    const uint32_t C = (uint32_t)comps.size();
    std::vector<char> nontrivial(C, 0);
    for (uint32_t c = 0; c < C; ++c) if (comps[c].size() >= 2) nontrivial[c] = 1;
    for (uint32_t e = 0; e < E; ++e) if (cs_caller[e] == cs_callee[e]) nontrivial[comp[cs_caller[e]]] = 1;
    // canonical condensed ids
    std::vector<std::pair<uint32_t, uint32_t>> nt;   // (smallest member, comp)
    for (uint32_t c = 0; c < C; ++c)
        if (nontrivial[c]) nt.push_back({*std::min_element(comps[c].begin(), comps[c].end()), c});
    std::sort(nt.begin(), nt.end());
    std::vector<uint32_t> cid(C);
    for (uint32_t c = 0; c < C; ++c) if (!nontrivial[c]) cid[c] = comps[c][0];
    for (uint32_t i = 0; i < nt.size(); ++i) cid[nt[i].second] = F + i;
    g->V = F + (uint32_t)nt.size();
    g->cnode_of_func.resize(F);
    for (uint32_t f = 0; f < F; ++f) g->cnode_of_func[f] = cid[comp[f]];

    g->incl.assign((size_t)n_req * g->V * M, 0.0);
    g->a.assign((size_t)n_req * E * M, 0.0);
    g->flags.assign((size_t)n_req * E, 0);

    for (uint32_t q = 0; q < n_req; ++q) {
        const uint32_t c = req_ctx[q];
        // step 1: exclusive costs and measured call weights in context c
        std::vector<std::vector<double>> excl(F, std::vector<double>(n_stall, 0.0));
        std::vector<uint64_t> S(F, 0), w(E, 0);
        for (uint64_t i = 0; i < k; ++i) {
            if (kctx[i] != c || knode[i] == UNKNOWN) continue;
            if (knode[i] >= n_nodes || kstall[i] >= n_stall) { g->status = INVALID_ARG; return g; }
            uint32_t f = node_func[knode[i]];
            excl[f][kstall[i]] += (double)kval[i];
            S[f] += kval[i];
            if (call_of_node[knode[i]] >= 0) w[call_of_node[knode[i]]] += kval[i];
        }
        std::vector<char> measured_in(F, 0);
        for (uint32_t f = 0; f < F; ++f)
            for (uint32_t e : in_edges[f]) if (w[e] > 0) measured_in[f] = 1;
        // step 2: zero-weight fix-up, closure through callers
        std::vector<double> wt(E);
        for (uint32_t e = 0; e < E; ++e) wt[e] = (double)w[e];
        std::vector<uint8_t> fl(E, 0);
        std::vector<char> inZ(F, 0);
        std::vector<uint32_t> work;
        for (uint32_t f = 0; f < F; ++f)
            if (S[f] > 0 && !in_edges[f].empty() && !measured_in[f]) { inZ[f] = 1; work.push_back(f); }
        while (!work.empty()) {
            uint32_t f = work.back(); work.pop_back();
            for (uint32_t e : in_edges[f]) {
                wt[e] = 1.0; fl[e] |= F_FIXUP;
                uint32_t h = cs_caller[e];
                if (!inZ[h] && !in_edges[h].empty() && !measured_in[h]) { inZ[h] = 1; work.push_back(h); }
            }
        }
        // step 3: condensation
        std::vector<std::vector<double>> cex(C, std::vector<double>(n_stall, 0.0));
        std::vector<char> cneed(C, 0);
        for (uint32_t f = 0; f < F; ++f) {
            for (uint32_t r = 0; r < n_stall; ++r) cex[comp[f]][r] += excl[f][r];
            if (S[f] > 0 || inZ[f]) cneed[comp[f]] = 1;
        }
        std::vector<std::vector<uint32_t>> cin(C), cout_(C);
        for (uint32_t e = 0; e < E; ++e) {
            uint32_t a = comp[cs_caller[e]], b = comp[cs_callee[e]];
            if (a == b) { fl[e] |= F_INTRA; wt[e] = 0.0; continue; }
            cin[b].push_back(e); cout_[a].push_back(e);
        }
        std::vector<double> W(C, 0.0);
        for (uint32_t v = 0; v < C; ++v) for (uint32_t e : cin[v]) W[v] += wt[e];
        // reading: step-2 rule again on the condensed graph
        std::vector<char> inZ2(C, 0);
        for (uint32_t v = 0; v < C; ++v)
            if (cneed[v] && !cin[v].empty() && W[v] == 0.0) { inZ2[v] = 1; work.push_back(v); }
        while (!work.empty()) {
            uint32_t v = work.back(); work.pop_back();
            for (uint32_t e : cin[v]) {
                wt[e] = 1.0; fl[e] |= F_FIXUP2;
                uint32_t u = comp[cs_caller[e]];
                if (!inZ2[u] && !cin[u].empty() && W[u] == 0.0) { inZ2[u] = 1; work.push_back(u); }
            }
        }
        for (uint32_t v = 0; v < C; ++v) { W[v] = 0.0; for (uint32_t e : cin[v]) W[v] += wt[e]; }
        // step 4: bottom-up in Tarjan completion order (callees first)
        std::vector<std::vector<double>> incl(C, std::vector<double>(n_stall, 0.0));
        double* A = &g->a[(size_t)q * E * M];
        for (uint32_t v = 0; v < C; ++v) {
            for (uint32_t r = 0; r < n_stall; ++r) incl[v][r] = cex[v][r];
            for (uint32_t e : cout_[v]) {
                uint32_t h = comp[cs_callee[e]];
                double ratio = W[h] > 0.0 ? wt[e] / W[h] : 0.0;
                double tot = 0.0;
                for (uint32_t r = 0; r < n_stall; ++r) {
                    double x = ratio * incl[h][r];
                    incl[v][r] += x;
                    A[(size_t)e * M + r] = x;
                    tot += x;
                }
                A[(size_t)e * M + n_stall] = tot;
            }
        }
        double* I = &g->incl[(size_t)q * g->V * M];
        for (uint32_t v = 0; v < C; ++v) {
            double tot = 0.0;
            for (uint32_t r = 0; r < n_stall; ++r) { I[(size_t)cid[v] * M + r] = incl[v][r]; tot += incl[v][r]; }
            I[(size_t)cid[v] * M + n_stall] = tot;
        }
        std::memcpy(&g->flags[(size_t)q * E], fl.data(), E);
    }
    return g;
}

// ---------------------------------------------------------------------------
// result access (ctypes marshalling)
int orc_status(void* p) { return ((KeyList*)p)->status; }
uint64_t orc_bad(void* p) { return ((KeyList*)p)->bad; }
uint64_t orc_size(void* p) { return ((KeyList*)p)->val.size(); }
// The GPU calling context tree of one context as a tree (Section 6.3, step
// 4): every call path from a root of the condensed graph, breadth-first,
// carrying the product of the ratios r(e) = a(e) / incl(callee) (total
// column) of its call sites; children in call-site order; paths whose
// product or whose node's cost is zero are left out; at most `budget` nodes.
struct Tree {
    std::vector<uint32_t> parent, cnode, edge;
    std::vector<double> scale, incl;
    int truncated = 0;
};

void* orc_expand(uint32_t F, uint32_t V, uint32_t E, const uint32_t* cnode_of_func, const uint32_t* cs_caller,
                 const uint32_t* cs_callee, uint32_t M, const double* incl, const double* a, uint32_t budget) {
    Tree* t = new Tree();
    std::vector<uint8_t> live(V, 0), has_caller(V, 0);
    for (uint32_t f = 0; f < F; ++f) live[cnode_of_func[f]] = 1;
    std::vector<std::vector<uint32_t>> calls(V);             // external call sites of each condensed node
    for (uint32_t e = 0; e < E; ++e) {
        const uint32_t g = cnode_of_func[cs_caller[e]], h = cnode_of_func[cs_callee[e]];
        if (g == h) continue;
        calls[g].push_back(e);
        has_caller[h] = 1;
    }
    auto add = [&](uint32_t par, uint32_t v, uint32_t e, double sc) {
        if (t->cnode.size() >= budget) { t->truncated = 1; return; }
        t->parent.push_back(par); t->cnode.push_back(v); t->edge.push_back(e); t->scale.push_back(sc);
        for (uint32_t r = 0; r < M; ++r) t->incl.push_back(incl[(size_t)v * M + r] * sc);
    };
    for (uint32_t v = 0; v < V; ++v)
        if (live[v] && !has_caller[v] && incl[(size_t)v * M + M - 1] > 0.0) add(0xFFFFFFFFu, v, 0xFFFFFFFFu, 1.0);
    size_t begin = 0;
    while (begin < t->cnode.size()) {                        // one level per round
        const size_t end = t->cnode.size();
        for (size_t i = begin; i < end; ++i) {
            for (uint32_t e : calls[t->cnode[i]]) {
                const uint32_t h = cnode_of_func[cs_callee[e]];
                const double ih = incl[(size_t)h * M + M - 1];
                const double r = ih > 0.0 ? a[(size_t)e * M + M - 1] / ih : 0.0;
                const double sc = t->scale[i] * r;
                if (sc > 0.0) add((uint32_t)i, h, e, sc);
            }
        }
        begin = end;
    }
    return t;
}
uint64_t orc_expand_size(void* p) { return ((Tree*)p)->cnode.size(); }
int orc_expand_truncated(void* p) { return ((Tree*)p)->truncated; }
void orc_expand_fetch(void* p, uint32_t* parent, uint32_t* cnode, uint32_t* edge, double* scale, double* incl) {
    Tree* t = (Tree*)p;
    for (size_t i = 0; i < t->cnode.size(); ++i) {
        parent[i] = t->parent[i]; cnode[i] = t->cnode[i]; edge[i] = t->edge[i]; scale[i] = t->scale[i];
    }
    for (size_t i = 0; i < t->incl.size(); ++i) incl[i] = t->incl[i];
}
void orc_expand_free(void* p) { delete (Tree*)p; }

// Sparse layouts of several profiles (Section 6.2).  Input: the keys of all
// profiles flattened, with each key's profile index.  CMS orders everything
// by (context = (ctx, node), metric = stall, profile); PMS by (profile,
// context, metric).  Offsets are CSR-style, with one extra closing entry.
struct Sparse {
    std::vector<uint64_t> prof_off, plane_off, metric_off;
    std::vector<uint32_t> plane_ctx, plane_node, pid;
    std::vector<uint32_t> metric_id;
    std::vector<uint64_t> val;
};

void* orc_cms(uint64_t n, const uint32_t* kp, const uint32_t* kctx, const uint32_t* knode, const uint8_t* kstall,
              const uint64_t* kval) {
    Sparse* o = new Sparse();
    std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>, uint64_t> m;   // (ctx, node, stall, p)
    for (uint64_t i = 0; i < n; ++i) m[std::make_tuple(kctx[i], knode[i], (uint32_t)kstall[i], kp[i])] = kval[i];
    bool first = true;
    uint32_t pc = 0, pn = 0, ps = 0;
    for (auto& kv : m) {
        const uint32_t c = std::get<0>(kv.first), nd = std::get<1>(kv.first), r = std::get<2>(kv.first);
        const bool new_plane = first || c != pc || nd != pn;
        const bool new_metric = new_plane || r != ps;
        if (new_plane) { o->plane_ctx.push_back(c); o->plane_node.push_back(nd); o->plane_off.push_back(o->metric_id.size()); }
        if (new_metric) { o->metric_id.push_back(r); o->metric_off.push_back(o->val.size()); }
        o->pid.push_back(std::get<3>(kv.first));
        o->val.push_back(kv.second);
        first = false; pc = c; pn = nd; ps = r;
    }
    o->plane_off.push_back(o->metric_id.size());
    o->metric_off.push_back(o->val.size());
    return o;
}

void* orc_pms(uint32_t P, uint64_t n, const uint32_t* kp, const uint32_t* kctx, const uint32_t* knode,
              const uint8_t* kstall, const uint64_t* kval) {
    Sparse* o = new Sparse();
    std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>, uint64_t> m;   // (p, ctx, node, stall)
    for (uint64_t i = 0; i < n; ++i) m[std::make_tuple(kp[i], kctx[i], knode[i], (uint32_t)kstall[i])] = kval[i];
    o->prof_off.assign(P + 1, 0);
    bool first = true;
    uint32_t pp = 0, pc = 0, pn = 0;
    for (auto& kv : m) {
        const uint32_t p = std::get<0>(kv.first), c = std::get<1>(kv.first), nd = std::get<2>(kv.first);
        if (first || p != pp || c != pc || nd != pn) {
            o->plane_ctx.push_back(c); o->plane_node.push_back(nd); o->plane_off.push_back(o->val.size());
            o->prof_off[p + 1] = o->plane_ctx.size();
        }
        o->metric_id.push_back(std::get<3>(kv.first));
        o->val.push_back(kv.second);
        first = false; pp = p; pc = c; pn = nd;
    }
    for (uint32_t p = 1; p <= P; ++p) o->prof_off[p] = std::max(o->prof_off[p], o->prof_off[p - 1]);
    o->plane_off.push_back(o->val.size());
    return o;
}

void orc_sparse_sizes(void* p, uint64_t* sz) {
    Sparse* o = (Sparse*)p;
    sz[0] = o->plane_ctx.size(); sz[1] = o->metric_id.size(); sz[2] = o->val.size(); sz[3] = o->prof_off.size();
}
void orc_sparse_fetch(void* p, uint64_t* prof_off, uint32_t* plane_ctx, uint32_t* plane_node, uint64_t* plane_off,
                      uint32_t* metric_id, uint64_t* metric_off, uint32_t* pid, uint64_t* val) {
    Sparse* o = (Sparse*)p;
    for (size_t i = 0; i < o->prof_off.size(); ++i) prof_off[i] = o->prof_off[i];
    for (size_t i = 0; i < o->plane_ctx.size(); ++i) { plane_ctx[i] = o->plane_ctx[i]; plane_node[i] = o->plane_node[i]; }
    for (size_t i = 0; i < o->plane_off.size(); ++i) plane_off[i] = o->plane_off[i];
    for (size_t i = 0; i < o->metric_id.size(); ++i) metric_id[i] = o->metric_id[i];
    for (size_t i = 0; i < o->metric_off.size(); ++i) metric_off[i] = o->metric_off[i];
    for (size_t i = 0; i < o->pid.size(); ++i) pid[i] = o->pid[i];
    for (size_t i = 0; i < o->val.size(); ++i) val[i] = o->val[i];
}
void orc_sparse_free(void* p) { delete (Sparse*)p; }

// Call-path profile unification (Section 6.1): the nodes of all CCTs in
// order; a node is identified by its merged parent and its (module, offset);
// a new identity gets the next merged id.
struct Unified {
    std::vector<uint32_t> uid, parent, module;
    std::vector<uint64_t> offset;
    int status = OK;
};

void* orc_unify(uint32_t n_cct, const uint64_t* base, const uint32_t* parent, const uint16_t* module,
                const uint64_t* offset) {
    Unified* u = new Unified();
    std::map<std::tuple<uint32_t, uint32_t, uint64_t>, uint32_t> ids;
    const uint64_t N = base[n_cct];
    u->uid.assign(N, 0);
    for (uint32_t p = 0; p < n_cct; ++p)
        for (uint64_t i = base[p]; i < base[p + 1]; ++i) {
            const uint32_t par = parent[i];
            if (par != 0xFFFFFFFFu && base[p] + par >= i) { u->status = INVALID_ARG; return u; }
            const uint32_t up = par == 0xFFFFFFFFu ? 0xFFFFFFFFu : u->uid[base[p] + par];
            const auto key = std::make_tuple(up, (uint32_t)module[i], offset[i]);
            auto it = ids.find(key);
            if (it == ids.end()) {
                const uint32_t id = (uint32_t)u->parent.size();
                ids[key] = id;
                u->parent.push_back(up);
                u->module.push_back(module[i]);
                u->offset.push_back(offset[i]);
                u->uid[i] = id;
            } else {
                u->uid[i] = it->second;
            }
        }
    return u;
}
// Bottom-up view (Section 7): the costs of a function divided among the
// calling contexts in which it is called.  Its roots are the functions of
// the keys' structure nodes (UNKNOWN keys belong to no function).  Below a
// function, each node stands for one caller chain: the call sites met when
// walking up the calling context tree from a key's launch context -- the
// context's own call site first, then its parent's, up to the root's -- cut
// after `levels` sites; level k holds the chains of k sites.  A node's value
// per stall reason is the sum of the values of the keys of its function
// whose context's chain begins with the node's chain.  Nodes are numbered
// level by level and, within a level, in the order of the first key (in
// profile order) that reaches them.  Roots carry module 0xFFFF, offset 0.
struct BottomUp {
    std::vector<uint32_t> parent, func, module;
    std::vector<uint64_t> offset, level_off;
    std::vector<uint32_t> vnode, vstall;
    std::vector<uint64_t> val;
    int status = OK;
};

void* orc_bottom_up(uint64_t k, const uint32_t* kctx, const uint32_t* knode, const uint8_t* kstall,
                    const uint64_t* kval, uint32_t n_nodes, const uint32_t* node_func, uint32_t n_cct,
                    const uint32_t* cct_parent, const uint16_t* cct_module, const uint64_t* cct_offset,
                    uint32_t levels) {
    BottomUp* b = new BottomUp();
    for (uint32_t v = 0; v < n_cct; ++v)
        if ((cct_parent[v] != NO_PARENT && cct_parent[v] >= v) || cct_module[v] == 0xFFFFu ||
            (cct_offset[v] >> 48)) { b->status = INVALID_TABLE; return b; }
    // every key's chain of labels: its function, then the call sites upward
    std::vector<std::vector<std::pair<uint32_t, uint64_t>>> chain(k);
    for (uint64_t i = 0; i < k; ++i) {
        if (kctx[i] >= n_cct || (knode[i] != UNKNOWN && knode[i] >= n_nodes)) { b->status = INVALID_ARG; return b; }
        if (knode[i] == UNKNOWN) continue;
        chain[i].push_back(std::make_pair(0xFFFFu, (uint64_t)node_func[knode[i]]));
        for (uint32_t c = kctx[i]; c != NO_PARENT && chain[i].size() <= levels; c = cct_parent[c])
            chain[i].push_back(std::make_pair((uint32_t)cct_module[c], cct_offset[c]));
    }
    std::vector<uint32_t> at(k, NO_PARENT);        // each key's node at the previous level
    std::map<std::pair<uint32_t, uint32_t>, uint64_t> cost;
    b->level_off.push_back(0);
    for (uint32_t lev = 0; lev <= levels; ++lev) {
        std::map<std::tuple<uint32_t, uint32_t, uint64_t>, uint32_t> ids;
        for (uint64_t i = 0; i < k; ++i) {
            if (chain[i].size() <= lev) continue;
            const auto lab = chain[i][lev];
            const auto key = std::make_tuple(at[i], lab.first, lab.second);
            auto it = ids.find(key);
            uint32_t id;
            if (it == ids.end()) {
                id = (uint32_t)b->parent.size();
                ids[key] = id;
                b->parent.push_back(at[i]);
                b->func.push_back(node_func[knode[i]]);
                b->module.push_back(lab.first);
                b->offset.push_back(lev == 0 ? 0 : lab.second);
            } else {
                id = it->second;
            }
            cost[std::make_pair(id, (uint32_t)kstall[i])] += kval[i];
            at[i] = id;
        }
        b->level_off.push_back(b->parent.size());
    }
    for (auto& kv : cost) {
        b->vnode.push_back(kv.first.first);
        b->vstall.push_back(kv.first.second);
        b->val.push_back(kv.second);
    }
    return b;
}
int orc_bu_status(void* p) { return ((BottomUp*)p)->status; }
void orc_bu_sizes(void* p, uint64_t* n) {
    BottomUp* b = (BottomUp*)p;
    n[0] = b->parent.size(); n[1] = b->val.size(); n[2] = b->level_off.size();
}
void orc_bu_fetch(void* p, uint32_t* parent, uint32_t* func, uint16_t* module, uint64_t* offset, uint64_t* level_off,
                  uint32_t* vnode, uint8_t* vstall, uint64_t* val) {
    BottomUp* b = (BottomUp*)p;
    for (size_t i = 0; i < b->parent.size(); ++i) {
        parent[i] = b->parent[i]; func[i] = b->func[i]; module[i] = (uint16_t)b->module[i]; offset[i] = b->offset[i];
    }
    std::copy(b->level_off.begin(), b->level_off.end(), level_off);
    for (size_t i = 0; i < b->val.size(); ++i) { vnode[i] = b->vnode[i]; vstall[i] = (uint8_t)b->vstall[i]; val[i] = b->val[i]; }
}
void orc_bu_free(void* p) { delete (BottomUp*)p; }

uint64_t orc_unify_size(void* p) { return ((Unified*)p)->parent.size(); }
int orc_unify_status(void* p) { return ((Unified*)p)->status; }
void orc_unify_fetch(void* p, uint32_t* uid, uint32_t* parent, uint16_t* module, uint64_t* offset) {
    Unified* u = (Unified*)p;
    for (size_t i = 0; i < u->uid.size(); ++i) uid[i] = u->uid[i];
    for (size_t i = 0; i < u->parent.size(); ++i) {
        parent[i] = u->parent[i]; module[i] = (uint16_t)u->module[i]; offset[i] = u->offset[i];
    }
}
void orc_unify_free(void* p) { delete (Unified*)p; }

void orc_fetch(void* p, uint32_t* ctx, uint32_t* node, uint8_t* stall, uint64_t* val,
               uint64_t* total, uint64_t* unknown) {
    KeyList* k = (KeyList*)p;
    for (size_t i = 0; i < k->val.size(); ++i) {
        ctx[i] = k->ctx[i]; node[i] = k->node[i]; stall[i] = (uint8_t)k->stall[i]; val[i] = k->val[i];
    }
    if (total) for (size_t r = 0; r < k->total.size(); ++r) total[r] = k->total[r];
    if (unknown) for (size_t r = 0; r < k->unknown.size(); ++r) unknown[r] = k->unknown[r];
}
void orc_free(void* p) { delete (KeyList*)p; }

uint64_t orc_derive_size(void* p) { return ((Derived*)p)->sum.size(); }
void orc_derive_fetch(void* p, uint32_t* ctx, uint32_t* node, uint8_t* stall, uint64_t* sum,
                      double* mn, double* mx, double* mean, double* sd, double* cov,
                      uint64_t* S, uint64_t* S_issued, double* W, double* frac) {
    Derived* d = (Derived*)p;
    for (size_t i = 0; i < d->sum.size(); ++i) {
        ctx[i] = d->ctx[i]; node[i] = d->node[i]; stall[i] = (uint8_t)d->stall[i]; sum[i] = d->sum[i];
        mn[i] = d->mn[i]; mx[i] = d->mx[i]; mean[i] = d->mean[i]; sd[i] = d->sd[i]; cov[i] = d->cov[i];
    }
    for (size_t c = 0; c < d->S.size(); ++c) { S[c] = d->S[c]; S_issued[c] = d->S_issued[c]; W[c] = d->W[c]; }
    for (size_t i = 0; i < d->frac.size(); ++i) frac[i] = d->frac[i];
}
void orc_derive_free(void* p) { delete (Derived*)p; }

uint64_t orc_ratio_size(void* p) { return ((RatioRows*)p)->num.size(); }
void orc_ratio_fetch(void* p, uint32_t* ctx, uint32_t* node, uint8_t* stall, uint64_t* num, uint64_t* den,
                     double* ratio) {
    RatioRows* o = (RatioRows*)p;
    for (size_t i = 0; i < o->num.size(); ++i) {
        ctx[i] = o->ctx[i];
        node[i] = o->node[i];
        stall[i] = (uint8_t)o->stall[i];
        num[i] = o->num[i];
        den[i] = o->den[i];
        ratio[i] = o->ratio[i];
    }
}
void orc_ratio_free(void* p) { delete (RatioRows*)p; }

int orc_issue_status(void* p) { return ((IssueRows*)p)->status; }
uint64_t orc_issue_size(void* p) { return ((IssueRows*)p)->S.size(); }
void orc_issue_fetch(void* p, uint32_t* ctx, uint32_t* func, uint64_t* S, uint64_t* S_issued, double* W,
                     double* frac) {
    IssueRows* o = (IssueRows*)p;
    std::copy(o->ctx.begin(), o->ctx.end(), ctx);
    std::copy(o->func.begin(), o->func.end(), func);
    std::copy(o->S.begin(), o->S.end(), S);
    std::copy(o->S_issued.begin(), o->S_issued.end(), S_issued);
    std::copy(o->W.begin(), o->W.end(), W);
    std::copy(o->frac.begin(), o->frac.end(), frac);
}
void orc_issue_free(void* p) { delete (IssueRows*)p; }

int orc_apportion_status(void* p) { return ((GpuCct*)p)->status; }
uint32_t orc_apportion_V(void* p) { return ((GpuCct*)p)->V; }
void orc_apportion_fetch(void* p, uint32_t* cnode_of_func, double* incl, double* a, uint8_t* flags) {
    GpuCct* g = (GpuCct*)p;
    std::copy(g->cnode_of_func.begin(), g->cnode_of_func.end(), cnode_of_func);
    std::copy(g->incl.begin(), g->incl.end(), incl);
    std::copy(g->a.begin(), g->a.end(), a);
    std::copy(g->flags.begin(), g->flags.end(), flags);
}
void orc_apportion_free(void* p) { delete (GpuCct*)p; }

}  // extern "C"
