"""The pins are strong enough: each test compiles a copy of oracle.cpp with
one plausible mistake planted (a wrong boundary, a dropped term, a wrong
index or divisor) and checks that some pin now fails.  Mistakes are planted
in a private copy of the oracle on the CPU only."""
import os
import subprocess

import pytest

import oracle
import test_oracle_apportion as TA
import test_oracle_attribution as TT
import test_oracle_bottom_up as TB
import test_oracle_expand as TX
import test_oracle_flat as TF
import test_oracle_inclusive_derive as TI
import test_oracle_issue as TW
import test_oracle_ratio as TR
import test_oracle_sparse as TS
import test_oracle_unify as TU

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.cpp")

MUTATIONS = [
    ("closed-range", "if (pc[i] < range_hi[j]) node", "if (pc[i] <= range_hi[j]) node",
     [lambda o: TT.test_golden_fixture(o)]),
    ("keep-zero-keys", "if (kv.second == 0) continue;", "",
     [lambda o: TT.test_golden_fixture(o)]),
    ("no-unknown-total", "if (node == UNKNOWN) out->unknown[stall[i]] += c;", "",
     [lambda o: TT.test_golden_fixture(o)]),
    ("lower-bound-search", "const uint64_t* it = std::upper_bound(range_lo, range_lo + n_ranges, pc[i]);",
     "const uint64_t* it = std::lower_bound(range_lo, range_lo + n_ranges, pc[i]);",
     [lambda o: TT.test_golden_fixture(o)]),
    ("count-ignored", "uint64_t c = count ? count[i] : 1;", "uint64_t c = 1;",
     [lambda o: TT.test_golden_fixture(o)]),
    ("unknown-dropped-from-inclusive", "if (n == UNKNOWN) { agg[Key(kctx[i], n, kstall[i])] += kval[i]; continue; }",
     "if (n == UNKNOWN) continue;",
     [lambda o: TI.test_structure_inclusive_brute(o)]),
    ("step2-no-callers", "if (!inZ[h] && !in_edges[h].empty() && !measured_in[h]) { inZ[h] = 1; work.push_back(h); }", "",
     [lambda o: TA.test_golden(o, "gpucct_fig5.json")]),
    ("ratio-of-tail", "double ratio = W[h] > 0.0 ? wt[e] / W[h] : 0.0;", "double ratio = W[v] > 0.0 ? wt[e] / W[v] : 0.0;",
     [lambda o: TA.test_golden(o, "gpucct_fig5.json"), lambda o: TA.test_path_enumeration(o, 1, False)]),
    ("share-of-exclusive-cost", "double x = ratio * incl[h][r];", "double x = ratio * cex[h][r];",
     [lambda o: TA.test_golden(o, "gpucct_fig5.json"), lambda o: TA.test_golden(o, "gpucct_diamond.json")]),
    ("call-weight-one-stall", "if (call_of_node[knode[i]] >= 0) w[call_of_node[knode[i]]] += kval[i];",
     "if (call_of_node[knode[i]] >= 0 && kstall[i] == 0) w[call_of_node[knode[i]]] += kval[i];",
     [lambda o: TA.test_golden(o, "gpucct_fig5.json"), lambda o: TA.test_path_enumeration(o, 1, False)]),
    ("fixup-without-samples", "if (S[f] > 0 && !in_edges[f].empty() && !measured_in[f]) { inZ[f] = 1; work.push_back(f); }",
     "if (!in_edges[f].empty() && !measured_in[f]) { inZ[f] = 1; work.push_back(f); }",
     [lambda o: TA.test_golden(o, "gpucct_fig5.json"), lambda o: TA.test_golden(o, "gpucct_diamond.json")]),
    ("no-fixup2", "if (cneed[v] && !cin[v].empty() && W[v] == 0.0) { inZ2[v] = 1; work.push_back(v); }", "",
     [lambda o: TA.test_golden(o, "gpucct_fig5.json")]),
    ("scc-excl-dropped", "for (uint32_t r = 0; r < n_stall; ++r) cex[comp[f]][r] += excl[f][r];",
     "for (uint32_t r = 0; r < n_stall; ++r) cex[comp[f]][r] = excl[f][r];",
     [lambda o: TA.test_golden(o, "gpucct_fig5.json")]),
    ("issue-rate-of-stalls", "d->W[c] = (double)d->S_issued[c] / (double)d->S[c];",
     "d->W[c] = (double)(d->S[c] - d->S_issued[c]) / (double)d->S[c];",
     [lambda o: TI.test_derive_vs_numpy(o), lambda o: TI.test_derive_single_profile(o)]),
    ("issue-by-function-stalled-share", "o->W.push_back((double)issued / (double)S);",
     "o->W.push_back((double)(S - issued) / (double)S);",
     [lambda o: TW.test_hand_example(o, 0b001, [5 / 8, 2 / 8, 0.0, 1 / 2])]),
    ("issue-by-function-keyed-by-node", "std::vector<uint64_t>& v = per[std::make_pair(kctx[i], node_func[knode[i]])];",
     "std::vector<uint64_t>& v = per[std::make_pair(kctx[i], knode[i])];",
     [lambda o: TW.test_hand_example(o, 0b001, [5 / 8, 2 / 8, 0.0, 1 / 2])]),
    ("issue-by-function-first-reason-only", "if (r < 32 && ((issued_mask >> r) & 1u)) issued += kv.second[r];",
     "if (r == 0) issued += kv.second[r];",
     [lambda o: TW.test_hand_example(o, 0b101, [1.0, 2 / 8, 0.0, 1.0])]),
    ("issue-by-function-unknown-as-function", "if (knode[i] == UNKNOWN) continue;\n        if (knode[i] >= n_nodes",
     "if (knode[i] >= n_nodes",
     [lambda o: TW.test_hand_example(o, 0b001, [5 / 8, 2 / 8, 0.0, 1 / 2])]),
    ("ratio-first-denominator-in-numerator", "if (p < P_num) v.first += kval[p][i];",
     "if (p <= P_num) v.first += kval[p][i];",
     [lambda o: TR.test_hand_example(o)]),
    ("ratio-inverted", "(double)kv.second.first / (double)kv.second.second);",
     "(double)kv.second.second / (double)kv.second.first);",
     [lambda o: TR.test_hand_example(o)]),
    ("ratio-zero-denominator-as-zero", "o->ratio.push_back(kv.second.second == 0 ? NAN :",
     "o->ratio.push_back(kv.second.second == 0 ? 0.0 :",
     [lambda o: TR.test_hand_example(o)]),
    ("ratio-last-thread-only", "if (p < P_num) v.first += kval[p][i];\n            else v.second += kval[p][i];",
     "if (p < P_num) v.first = kval[p][i];\n            else v.second = kval[p][i];",
     [lambda o: TR.test_hand_example(o)]),
    ("min-over-present-only", "for (uint32_t p = 0; p < P; ++p) { s += x[p]; lo = std::min(lo, x[p]); hi = std::max(hi, x[p]); }",
     "for (uint32_t p = 0; p < P; ++p) { s += x[p]; if (x[p]) lo = std::min(lo, x[p]); hi = std::max(hi, x[p]); }",
     [lambda o: TI.test_derive_vs_numpy(o)]),
    ("sample-std", "double sd = std::sqrt(ss / P);", "double sd = std::sqrt(ss / (P > 1 ? P - 1 : 1));",
     [lambda o: TI.test_derive_vs_numpy(o)]),
    ("incl-stops-below-func", "while (n != NO_PARENT) {\n            agg[Key(kctx[i], n, kstall[i])] += kval[i];",
     "while (node_parent[n] != NO_PARENT) {\n            agg[Key(kctx[i], n, kstall[i])] += kval[i];",
     [lambda o: TI.test_structure_inclusive_brute(o)]),
    ("cct-skip-self", "while (h != NO_PARENT) {\n            host", "h = cct_parent[h];\n        while (h != NO_PARENT) {\n            host",
     [lambda o: TI.test_cct_inclusive(o)]),
    ("expand-no-product", "const double sc = t->scale[i] * r;", "const double sc = r;",
     [lambda o: TX.test_ratios_are_call_site_weights(o, 1)]),
    ("expand-budget-off-by-one", "if (t->cnode.size() >= budget) { t->truncated = 1; return; }",
     "if (t->cnode.size() + 1 >= budget) { t->truncated = 1; return; }",
     [lambda o: TX.test_budget_gives_a_prefix(o, TX.plain_bin())]),
    ("expand-parent-is-level-start", "if (sc > 0.0) add((uint32_t)i, h, e, sc);",
     "if (sc > 0.0) add((uint32_t)begin, h, e, sc);",
     [lambda o: TX.test_paths_by_depth_first_enumeration(o, TX.plain_bin())]),
    ("expand-keeps-zero-scale", "if (sc > 0.0) add((uint32_t)i, h, e, sc);", "add((uint32_t)i, h, e, sc);",
     [lambda o: TX.test_paths_by_depth_first_enumeration(o, TX.plain_bin()),
      lambda o: TX.test_each_nodes_scales_sum_to_one(o, TX.plain_bin())]),
    ("cms-profile-major-order", "m[std::make_tuple(kctx[i], knode[i], (uint32_t)kstall[i], kp[i])] = kval[i];",
     "m[std::make_tuple(kctx[i], knode[i], kp[i], (uint32_t)kstall[i])] = kval[i];",
     [lambda o: TS.test_hand_computed_cms(o), lambda o: TS.test_cms_reconstructs_every_profile(o)]),
    ("bottom-up-ignores-parent", "const auto key = std::make_tuple(at[i], lab.first, lab.second);",
     "const auto key = std::make_tuple(0u, lab.first, lab.second);",
     [lambda o: TB.test_hand_example(o), lambda o: TB.test_brute_force(o, 20, 16)]),
    ("bottom-up-context-not-site", "chain[i].push_back(std::make_pair((uint32_t)cct_module[c], cct_offset[c]));",
     "chain[i].push_back(std::make_pair((uint32_t)cct_module[c], (uint64_t)c));",
     [lambda o: TB.test_hand_example(o), lambda o: TB.test_brute_force(o, 20, 16)]),
    ("bottom-up-skips-launch-site", "for (uint32_t c = kctx[i]; c != NO_PARENT && chain[i].size() <= levels; c = cct_parent[c])",
     "for (uint32_t c = cct_parent[kctx[i]]; c != NO_PARENT && chain[i].size() <= levels; c = cct_parent[c])",
     [lambda o: TB.test_hand_example(o), lambda o: TB.test_brute_force(o, 20, 16)]),
    ("cms-metric-runs-across-planes", "const bool new_metric = new_plane || r != ps;", "const bool new_metric = first || r != ps;",
     [lambda o: TS.test_hand_computed_cms(o), lambda o: TS.test_cms_reconstructs_every_profile(o)]),
    ("cms-plane-offsets-in-values", "if (new_plane) { o->plane_ctx.push_back(c); o->plane_node.push_back(nd); o->plane_off.push_back(o->metric_id.size()); }",
     "if (new_plane) { o->plane_ctx.push_back(c); o->plane_node.push_back(nd); o->plane_off.push_back(o->val.size()); }",
     [lambda o: TS.test_hand_computed_cms(o), lambda o: TS.test_cms_reconstructs_every_profile(o)]),
    ("pms-plane-per-context", "if (first || p != pp || c != pc || nd != pn) {\n            o->plane_ctx.push_back(c); o->plane_node.push_back(nd); o->plane_off.push_back(o->val.size());\n            o->prof_off[p + 1]",
     "if (first || p != pp || c != pc) {\n            o->plane_ctx.push_back(c); o->plane_node.push_back(nd); o->plane_off.push_back(o->val.size());\n            o->prof_off[p + 1]",
     [lambda o: TS.test_hand_computed_pms(o), lambda o: TS.test_pms_reconstructs_every_profile(o)]),
    ("pms-empty-profile-offsets", "for (uint32_t p = 1; p <= P; ++p) o->prof_off[p] = std::max(o->prof_off[p], o->prof_off[p - 1]);", "",
     [lambda o: TS.test_hand_computed_pms(o), lambda o: TS.test_profiles_without_keys(o)]),
    ("unify-root-under-node-0", "const uint32_t up = par == 0xFFFFFFFFu ? 0xFFFFFFFFu : u->uid[base[p] + par];",
     "const uint32_t up = par == 0xFFFFFFFFu ? 0u : u->uid[base[p] + par];",
     [lambda o: TU.test_hand_example(o), lambda o: TU.test_paths_are_kept(o)]),
    ("unify-ignores-module", "const auto key = std::make_tuple(up, (uint32_t)module[i], offset[i]);",
     "const auto key = std::make_tuple(up, 0u, offset[i]);",
     [lambda o: TU.test_hand_example(o), lambda o: TU.test_sites_differ_by_module(o)]),
    ("bottom-up-one-site-short", "for (uint32_t c = kctx[i]; c != NO_PARENT && chain[i].size() <= levels; c = cct_parent[c])",
     "for (uint32_t c = kctx[i]; c != NO_PARENT && chain[i].size() < levels; c = cct_parent[c])",
     [lambda o: TB.test_hand_example(o), lambda o: TB.test_hand_example_cut(o)]),
    ("bottom-up-stalls-merged", "cost[std::make_pair(id, (uint32_t)kstall[i])] += kval[i];",
     "cost[std::make_pair(id, 0u)] += kval[i];",
     [lambda o: TB.test_hand_example(o), lambda o: TB.test_brute_force(o, 20, 16)]),
    ("unify-ignores-parent", "const auto key = std::make_tuple(up, (uint32_t)module[i], offset[i]);",
     "const auto key = std::make_tuple(0u, (uint32_t)module[i], offset[i]);",
     [lambda o: TU.test_hand_example(o), lambda o: TU.test_paths_are_kept(o)]),
    ("flat-drops-unknown", "agg[std::make_pair(knode[i], (uint32_t)kstall[i])] += kval[i];",
     "if (knode[i] != UNKNOWN) agg[std::make_pair(knode[i], (uint32_t)kstall[i])] += kval[i];",
     [lambda o: TF.test_hand_computed_example(o), lambda o: TF.test_conservation_and_order_on_a_profile(o)]),
    ("flat-keeps-first-context", "agg[std::make_pair(knode[i], (uint32_t)kstall[i])] += kval[i];",
     "agg[std::make_pair(knode[i], (uint32_t)kstall[i])] = kval[i];",
     [lambda o: TF.test_hand_computed_example(o), lambda o: TF.test_conservation_and_order_on_a_profile(o)]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, pins):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mut = tmp_path / "oracle_mut.cpp"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(so), str(mut)])
    saved = oracle._lib
    oracle._lib = oracle.load(str(so))
    try:
        caught = 0
        for pin in pins:
            try:
                pin(oracle)
            except (AssertionError, ValueError, KeyError, IndexError):
                caught += 1
        assert caught >= 1, f"planted mistake '{name}' passed every pin"
    finally:
        oracle._lib = saved
