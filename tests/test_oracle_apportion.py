"""Pins of the oracle's GPU calling-context tree (Section 6.3, steps 1-4).

* hand-computed fixtures built from the worked example's text (A->B gets one
  call sample, D and E form an SCC) and a self-call;
* brute force: on small DAGs whose call instructions are all sampled (no
  fix-up), the inclusive cost of v must equal the sum over every downward
  call path Q from v of excl(end(Q)) * prod_{e in Q} w(e)/W(head(e)) -- the
  calling context tree obtained by splitting the graph, summed directly;
* a call *tree*: every ratio is 1, so inclusive = plain subtree sum;
* invariants on a generated workload: sum of a over a node's incoming edges
  equals its inclusive cost when it has incoming weight, and the roots'
  inclusive costs add up to all exclusive cost.
"""
import json
import os
import types
from collections import defaultdict

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _binary(node_func, caller, callee, cs_node, F):
    return types.SimpleNamespace(node_func=np.array(node_func, np.uint32), n_funcs=F,
                                 cs_caller=np.array(caller, np.uint32), cs_callee=np.array(callee, np.uint32),
                                 cs_node=np.array(cs_node, np.uint32))


def _keys(oracle_lib, rows):
    rows = sorted(map(tuple, rows))
    a = np.array(rows, dtype=np.uint64).reshape(-1, 4)
    return oracle_lib.KeyList(a[:, 0].astype(np.uint32), a[:, 1].astype(np.uint32), a[:, 2].astype(np.uint8),
                              a[:, 3].astype(np.uint64))


@pytest.mark.parametrize("name", ["gpucct_fig5.json", "gpucct_selfcall.json", "gpucct_diamond.json",
                                  "gpucct_two_cycle.json", "gpucct_scc_two_callers.json"])
def test_golden(oracle_lib, name):
    g = json.load(open(os.path.join(GOLD, name)))
    F = len(g["functions"])
    cs = g["call_sites"]
    B = _binary(g["node_func"], cs["caller"], cs["callee"], cs["node"], F)
    k = _keys(oracle_lib, g["keys"])
    S = g["n_stall"]
    res = oracle_lib.apportion(B, S, k, np.array(g["req_ctx"], np.uint32))
    assert res.V == g["expected_V"]
    assert res.cnode_of_func.tolist() == g["expected_cnode_of_func"]
    E = len(cs["caller"])
    for q, c in enumerate(g["req_ctx"]):
        exp_i = np.zeros((res.V, S + 1))
        for v, row in g["expected_incl"][str(c)].items():
            exp_i[int(v)] = row
        exp_a = np.zeros((E, S + 1))
        for e, row in g["expected_a"][str(c)].items():
            exp_a[int(e)] = row
        np.testing.assert_allclose(res.incl[q], exp_i, rtol=1e-14, atol=0)
        np.testing.assert_allclose(res.a[q], exp_a, rtol=1e-14, atol=0)
        assert res.flags[q].tolist() == g["expected_flags"][str(c)]


def _tiny_dag(seed, F, extra, tree=False):
    """Random DAG over F functions (function 0 the single root); one CALL
    node per call site and one LINE node per function."""
    rng = np.random.default_rng(seed)
    caller, callee = [], []
    for f in range(1, F):
        caller.append(int(rng.integers(0, f))); callee.append(f)
    if not tree:
        for _ in range(extra):
            a, b = sorted(rng.choice(F, 2, replace=False))
            caller.append(int(a)); callee.append(int(b))
    # nodes: FUNC f = 2f, LINE f = 2f + 1, then CALL nodes
    node_func = [f // 2 for f in range(2 * F)]
    cs_node = []
    for e, c in enumerate(caller):
        cs_node.append(len(node_func)); node_func.append(c)
    return caller, callee, cs_node, node_func


def _brute_incl(F, caller, callee, excl, w):
    """Sum over all downward call paths Q from v of excl(end(Q)) * prod r."""
    W = defaultdict(float)
    for e in range(len(caller)):
        W[callee[e]] += w[e]
    out_edges = defaultdict(list)
    for e in range(len(caller)):
        out_edges[caller[e]].append(e)

    def paths(v, prod, acc):
        acc += prod * excl[v]
        for e in out_edges[v]:
            h = callee[e]
            acc = paths(h, prod * (w[e] / W[h]), acc)
        return acc

    return [paths(v, np.ones_like(excl[0]), np.zeros_like(excl[0])) for v in range(F)]


@pytest.mark.parametrize("seed,tree", [(1, False), (2, False), (3, True), (4, False)])
def test_path_enumeration(oracle_lib, seed, tree):
    F, S = 7, 3
    caller, callee, cs_node, node_func = _tiny_dag(seed, F, 6, tree)
    rng = np.random.default_rng(100 + seed)
    rows = []
    for n in range(len(node_func)):
        for r in range(S):
            if n >= 2 * F or rng.random() < 0.5:    # every CALL node sampled -> no fix-up
                rows.append((0, n, r, int(rng.integers(1, 9))))
    k = _keys(oracle_lib, rows)
    B = _binary(node_func, caller, callee, cs_node, F)
    res = oracle_lib.apportion(B, S, k, np.array([0], np.uint32))
    excl = [np.zeros(S) for _ in range(F)]
    w = np.zeros(len(caller))
    call_of = {n: e for e, n in enumerate(cs_node)}
    for (_, n, r, v) in rows:
        excl[node_func[n]][r] += v
        if n in call_of:
            w[call_of[n]] += v
    incl = _brute_incl(F, caller, callee, excl, w)
    assert (res.flags == 0).all()
    for f in range(F):
        np.testing.assert_allclose(res.incl[0, f, :S], incl[f], rtol=1e-12)
        np.testing.assert_allclose(res.incl[0, f, S], incl[f].sum(), rtol=1e-12)
    W = defaultdict(float)
    for e in range(len(caller)):
        W[callee[e]] += w[e]
    for e in range(len(caller)):
        np.testing.assert_allclose(res.a[0, e, :S], w[e] / W[callee[e]] * incl[callee[e]], rtol=1e-12)
    if tree:
        # call tree: all ratios are 1 -> inclusive = subtree sum of exclusive
        kids = defaultdict(list)
        for e in range(len(caller)):
            kids[caller[e]].append(callee[e])

        def sub(v):
            return excl[v] + sum((sub(c) for c in kids[v]), np.zeros(S))
        for f in range(F):
            np.testing.assert_allclose(res.incl[0, f, :S], sub(f), rtol=1e-12)


def test_unsampled_caller_chain(oracle_lib):
    """R -> G -> H -> f, only f sampled: step 2 walks up to R's callee edge."""
    caller, callee = [0, 1, 2], [1, 2, 3]
    node_func = [0, 0, 1, 1, 2, 2, 3, 3, 0, 1, 2]
    cs_node = [8, 9, 10]
    B = _binary(node_func, caller, callee, cs_node, 4)
    k = _keys(oracle_lib, [(0, 7, 0, 5)])
    res = oracle_lib.apportion(B, 1, k, np.array([0], np.uint32))
    assert res.flags[0].tolist() == [1, 1, 1]
    np.testing.assert_allclose(res.incl[0, :, 1], [5, 5, 5, 5])
    np.testing.assert_allclose(res.a[0, :, 1], [5, 5, 5])


def test_invariants_generated(oracle_lib):
    w = synth.scaled(synth.PLAIN, 0.2)
    B = w.binary()
    S = w.samples(B)
    k = oracle_lib.attribute_samples(B, S)
    req = np.arange(0, 500, 25, dtype=np.uint32)
    res = oracle_lib.apportion(B, 16, k, req)
    F = B.n_funcs
    cn = res.cnode_of_func
    head = cn[B.cs_callee]
    tail = cn[B.cs_caller]
    ext = head != tail
    M = 17
    for q, c in enumerate(req):
        m = (k.ctx == c) & (k.node != 0xFFFFFFFF)
        tot = np.zeros(16)
        np.add.at(tot, k.stall[m], k.val[m].astype(np.float64))
        # roots: condensed nodes without external incoming edges
        has_in = np.zeros(res.V, bool)
        has_in[head[ext]] = True
        roots = [v for v in set(cn.tolist()) if not has_in[v]]
        np.testing.assert_allclose(res.incl[q, roots, :16].sum(0), tot, rtol=1e-12)
        # sum of a over incoming edges = incl for nodes with incoming weight
        ain = np.zeros((res.V, M))
        np.add.at(ain, head[ext], res.a[q][ext])
        wpos = np.zeros(res.V, bool)
        carry = (res.flags[q] & 3).astype(bool) | (res.a[q, :, 16] > 0)
        wpos[head[ext & carry]] = True
        vv = [v for v in range(res.V) if has_in[v] and res.incl[q, v, 16] > 0]
        for v in vv:
            np.testing.assert_allclose(ain[v], res.incl[q, v], rtol=1e-12)
        assert (res.a[q][~ext] == 0).all() and ((res.flags[q][~ext] & 4) == 4).all()
