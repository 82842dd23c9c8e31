// Static GPU call graph of a binary (Section 6.3, steps 1 and 3): call edges
// from call instructions, strongly connected components by Tarjan's
// algorithm, the condensed DAG and its level order.  Built once at load time
// on the host; the per-context apportioning kernels read the device tables.

#include <algorithm>
#include <vector>

#include "hpa_host.h"

namespace hpa {

namespace {

// Tarjan's SCC algorithm with an explicit stack (no recursion, so call
// chains of any depth are safe).  comp[f] is the component of f; components
// are numbered in completion order, which lists every component after all the
// components it reaches (callees before callers).
uint32_t tarjan_scc(uint32_t F, const std::vector<uint32_t>& off, const std::vector<uint32_t>& adj,
                    std::vector<uint32_t>& comp) {
    const uint32_t UNSET = 0xFFFFFFFFu;
    std::vector<uint32_t> idx(F, UNSET), low(F, 0), next_edge(F, 0);
    std::vector<uint8_t> on(F, 0);
    std::vector<uint32_t> stk, dfs;
    comp.assign(F, UNSET);
    uint32_t counter = 0, ncomp = 0;
    for (uint32_t root = 0; root < F; ++root) {
        if (idx[root] != UNSET) continue;
        dfs.push_back(root);
        idx[root] = low[root] = counter++;
        stk.push_back(root);
        on[root] = 1;
        next_edge[root] = off[root];
        while (!dfs.empty()) {
            const uint32_t v = dfs.back();
            if (next_edge[v] < off[v + 1]) {
                const uint32_t w = adj[next_edge[v]++];
                if (idx[w] == UNSET) {
                    idx[w] = low[w] = counter++;
                    stk.push_back(w);
                    on[w] = 1;
                    next_edge[w] = off[w];
                    dfs.push_back(w);
                } else if (on[w]) {
                    low[v] = std::min(low[v], idx[w]);
                }
                continue;
            }
            dfs.pop_back();
            if (!dfs.empty()) low[dfs.back()] = std::min(low[dfs.back()], low[v]);
            if (low[v] == idx[v]) {
                uint32_t x;
                do {
                    x = stk.back();
                    stk.pop_back();
                    on[x] = 0;
                    comp[x] = ncomp;
                } while (x != v);
                ++ncomp;
            }
        }
    }
    return ncomp;
}

void csr(uint32_t n, const std::vector<uint32_t>& key, const std::vector<uint32_t>& items,
         std::vector<uint32_t>& off, std::vector<uint32_t>& out) {
    off.assign(n + 1, 0);
    for (uint32_t k : key) off[k + 1]++;
    for (uint32_t i = 0; i < n; ++i) off[i + 1] += off[i];
    out.assign(items.size(), 0);
    std::vector<uint32_t> cur(off.begin(), off.end() - 1);
    for (size_t i = 0; i < items.size(); ++i) out[cur[key[i]]++] = items[i];
}

}  // namespace

hpa_status build_callgraph(hpa_handle* h, Binary* B) {
    const uint32_t F = B->n_funcs, E = B->n_calls, M = B->n_nodes;
    // successor lists of the static call graph (step 1)
    std::vector<uint32_t> soff, sadj, eid(E);
    for (uint32_t e = 0; e < E; ++e) eid[e] = B->cs_callee[e];
    csr(F, B->cs_caller, eid, soff, sadj);
    std::vector<uint32_t> comp;
    const uint32_t C = tarjan_scc(F, soff, sadj, comp);
    // non-trivial components: >= 2 members or a self-call (step 3)
    std::vector<uint32_t> size(C, 0), minf(C, 0xFFFFFFFFu);
    std::vector<uint8_t> self(C, 0);
    for (uint32_t f = 0; f < F; ++f) { size[comp[f]]++; minf[comp[f]] = std::min(minf[comp[f]], f); }
    for (uint32_t e = 0; e < E; ++e)
        if (B->cs_caller[e] == B->cs_callee[e]) self[comp[B->cs_caller[e]]] = 1;
    std::vector<std::pair<uint32_t, uint32_t>> nt;
    for (uint32_t c = 0; c < C; ++c)
        if (size[c] >= 2 || self[c]) nt.push_back({minf[c], c});
    std::sort(nt.begin(), nt.end());
    std::vector<uint32_t> cnode_of_comp(C, 0xFFFFFFFFu);
    for (uint32_t i = 0; i < nt.size(); ++i) cnode_of_comp[nt[i].second] = F + i;
    const uint32_t V = F + (uint32_t)nt.size();
    std::vector<uint32_t> cof(F);
    std::vector<uint8_t> live(V, 0);
    for (uint32_t f = 0; f < F; ++f) {
        const uint32_t c = comp[f];
        cof[f] = cnode_of_comp[c] != 0xFFFFFFFFu ? cnode_of_comp[c] : f;
        live[cof[f]] = 1;
    }
    // condensed edges
    std::vector<uint8_t> intra(E, 0);
    std::vector<uint32_t> ckey_in, ckey_out, citems_in, citems_out;
    for (uint32_t e = 0; e < E; ++e) {
        if (comp[B->cs_caller[e]] == comp[B->cs_callee[e]]) { intra[e] = 1; continue; }
        ckey_out.push_back(cof[B->cs_caller[e]]); citems_out.push_back(e);
        ckey_in.push_back(cof[B->cs_callee[e]]); citems_in.push_back(e);
    }
    std::vector<uint32_t> cin_off, cin_edge, cout_off, cout_edge;
    csr(V, ckey_in, citems_in, cin_off, cin_edge);
    csr(V, ckey_out, citems_out, cout_off, cout_edge);
    std::vector<uint32_t> cout_head(cout_edge.size());
    for (size_t i = 0; i < cout_edge.size(); ++i) cout_head[i] = cof[B->cs_callee[cout_edge[i]]];
    // heights: components complete callees-first, so one pass in completion order
    std::vector<std::vector<uint32_t>> members(C);
    for (uint32_t f = 0; f < F; ++f) members[comp[f]].push_back(f);
    std::vector<uint32_t> height(V, 0);
    uint32_t max_h = 0;
    for (uint32_t c = 0; c < C; ++c) {
        const uint32_t v = cof[members[c][0]];
        uint32_t hgt = 0;
        for (uint32_t i = cout_off[v]; i < cout_off[v + 1]; ++i)
            hgt = std::max(hgt, height[cof[B->cs_callee[cout_edge[i]]]] + 1);
        height[v] = hgt;
        max_h = std::max(max_h, hgt);
    }
    const uint32_t n_levels = F ? max_h + 1 : 0;
    std::vector<uint32_t> lkey, litems;
    for (uint32_t v = 0; v < V; ++v)
        if (live[v]) { lkey.push_back(height[v]); litems.push_back(v); }
    std::vector<uint32_t> level_off, level_node;
    csr(n_levels, lkey, litems, level_off, level_node);
    // function in-edges (original graph) for the step-2 fix-up
    std::vector<uint32_t> fin_off, fin_edge, eids(E);
    for (uint32_t e = 0; e < E; ++e) eids[e] = e;
    csr(F, B->cs_callee, eids, fin_off, fin_edge);
    std::vector<uint32_t> node_cs(M, 0xFFFFFFFFu);
    for (uint32_t e = 0; e < E; ++e) node_cs[B->cs_node[e]] = e;
    std::vector<uint32_t> cs_head(E);
    for (uint32_t e = 0; e < E; ++e) cs_head[e] = cof[B->cs_callee[e]];
    std::vector<uint32_t> level_of(V, 0);
    for (uint32_t v = 0; v < V; ++v) level_of[v] = live[v] ? height[v] : 0;

    B->n_cnodes = V;
    B->n_scc = (uint32_t)nt.size();
    B->cdag_levels = n_levels;
    B->cnode_of_func = cof;
    DevCallGraph& g = B->cg;
    g.F = F; g.E = E; g.V = V; g.n_levels = n_levels; g.M = M;
    hpa_status st;
    uint32_t *p0, *p1, *p2, *p3, *p4, *p5, *p6, *p7, *p8, *p9, *p10, *p11, *p12, *p13, *p14, *p15;
    uint8_t *q0, *q1;
    if ((st = upload(h, B, B->node_func, &p0)) || (st = upload(h, B, node_cs, &p1)) ||
        (st = upload(h, B, B->cs_caller, &p2)) || (st = upload(h, B, B->cs_callee, &p3)) ||
        (st = upload(h, B, cof, &p4)) || (st = upload(h, B, fin_off, &p5)) || (st = upload(h, B, fin_edge, &p6)) ||
        (st = upload(h, B, cin_off, &p7)) || (st = upload(h, B, cin_edge, &p8)) ||
        (st = upload(h, B, cout_off, &p9)) || (st = upload(h, B, cout_edge, &p10)) ||
        (st = upload(h, B, cout_head, &p13)) ||
        (st = upload(h, B, level_off, &p11)) || (st = upload(h, B, level_node, &p12)) ||
        (st = upload(h, B, intra, &q0)) || (st = upload(h, B, live, &q1)) ||
        (st = upload(h, B, cs_head, &p14)) || (st = upload(h, B, level_of, &p15)))
        return st;
    g.node_func = p0; g.node_cs = p1; g.cs_caller = p2; g.cs_callee = p3; g.cnode_of_func = p4;
    g.fin_off = p5; g.fin_edge = p6; g.cin_off = p7; g.cin_edge = p8; g.cout_off = p9; g.cout_edge = p10; g.cout_head = p13;
    g.level_off = p11; g.level_node = p12; g.edge_intra = q0; g.cnode_live = q1;
    g.cs_head = p14; g.level_of = p15;
    uint32_t* par;
    if ((st = upload(h, B, B->node_parent, &par))) return st;
    B->d_node_parent = par;
    uint32_t* dep;
    if ((st = upload(h, B, B->node_depth, &dep))) return st;
    B->d_node_depth = dep;
    return HPA_OK;
}

}  // namespace hpa
