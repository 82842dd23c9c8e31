"""Pins of the oracle's materialised GPU calling context tree (Section 6.3,
step 4), independent of oracle.cpp's expansion code."""
import collections

import numpy as np
import pytest

import oracle
import synth

BIG = 1 << 22


def setup(binary, n, n_ctx, seed, q_ctx):
    s = synth.make_samples(seed, binary, n, n_ctx, 1.1, counts=True)
    keys = oracle.attribute_samples(binary, s)
    g = oracle.apportion(binary, 16, keys, np.array(q_ctx, np.uint32))
    return keys, g


def plain_bin():
    b = synth.PLAIN.binary()
    return (b,) + setup(b, 300_000, 4, 21, [0, 3])


@pytest.fixture(scope="module")
def plain():
    return plain_bin()


def test_each_nodes_scales_sum_to_one(oracle_lib, plain):
    """Every call path from a root carries the product of the fractions of the
    callee's cost given to its call sites; summed over the paths reaching a
    node that has callers and a cost, these products are 1."""
    b, keys, g = plain
    for q in range(2):
        t = oracle.expand(b, g, q, BIG)
        assert not t.truncated
        per = collections.defaultdict(float)
        for v, sc in zip(t.cnode.tolist(), t.scale.tolist()):
            per[v] += sc
        callers = np.zeros(g.V, bool)
        for e in range(len(b.cs_caller)):
            gv, hv = g.cnode_of_func[b.cs_caller[e]], g.cnode_of_func[b.cs_callee[e]]
            if gv != hv:
                callers[hv] = True
        cost = g.incl[q][:, -1] > 0
        checked = 0
        for v in range(g.V):
            if cost[v] and callers[v] and v in per:
                assert abs(per[v] - 1.0) < 1e-9, (v, per[v])
                checked += 1
        assert checked > 100


def test_roots_hold_all_attributed_cost(oracle_lib, plain):
    b, keys, g = plain
    ctx_of = [0, 3]
    for q in range(2):
        t = oracle.expand(b, g, q, BIG)
        roots = t.parent == 0xFFFFFFFF
        m = (keys.ctx == ctx_of[q]) & (keys.node != oracle.UNKNOWN)
        assert abs(t.incl[roots, -1].sum() - float(keys.val[m].sum())) <= 1e-9 * float(keys.val[m].sum())


def _tiny(oracle_lib, seed, tree):
    import test_oracle_apportion as TA
    F, S = 9, 3
    caller, callee, cs_node, node_func = TA._tiny_dag(seed, F, 7, tree)
    rng = np.random.default_rng(200 + seed)
    rows = [(0, n, r, int(rng.integers(1, 9))) for n in range(len(node_func)) for r in range(S)
            if n >= 2 * F or rng.random() < 0.6]
    B = TA._binary(node_func, caller, callee, cs_node, F)
    return B, rows, oracle.apportion(B, S, TA._keys(oracle_lib, rows), np.array([0], np.uint32)), cs_node


@pytest.mark.parametrize("seed", [3, 5])
def test_a_call_tree_has_unit_scales(oracle_lib, seed):
    """Every function has one caller: no cost is split, every function with
    a cost appears once at scale 1, under its caller."""
    B, rows, g, _ = _tiny(oracle_lib, seed, True)
    t = oracle.expand(B, g, 0, BIG)
    assert np.all(t.scale == 1.0)
    assert sorted(t.cnode.tolist()) == [v for v in range(g.V) if g.incl[0][v, -1] > 0]
    for i in range(len(t.cnode)):
        if t.parent[i] != 0xFFFFFFFF:
            assert B.cs_caller[t.edge[i]] == t.cnode[t.parent[i]] and B.cs_callee[t.edge[i]] == t.cnode[i]


@pytest.mark.parametrize("seed", [1, 2, 4])
def test_ratios_are_call_site_weights(oracle_lib, seed):
    """On tiny DAGs with every call instruction sampled, a child's scale is
    its parent's times w(e) / W(callee), from the samples written here."""
    B, rows, g, cs_node = _tiny(oracle_lib, seed, False)
    w = np.zeros(len(B.cs_caller))
    call_of = {n: e for e, n in enumerate(cs_node)}
    for (_, n, r, v) in rows:
        if n in call_of:
            w[call_of[n]] += v
    W = collections.defaultdict(float)
    for e in range(len(w)):
        W[int(B.cs_callee[e])] += w[e]
    t = oracle.expand(B, g, 0, BIG)
    assert len(t.cnode) > len(set(t.cnode.tolist()))      # some function reached by several paths
    for i in range(len(t.cnode)):
        if t.parent[i] != 0xFFFFFFFF:
            e = int(t.edge[i])
            assert abs(t.scale[i] - t.scale[t.parent[i]] * w[e] / W[int(B.cs_callee[e])]) <= 1e-12


def test_budget_gives_a_prefix(oracle_lib, plain):
    b, keys, g = plain
    full = oracle.expand(b, g, 0, BIG)
    cut = oracle.expand(b, g, 0, len(full.cnode) // 3)
    k = len(cut.cnode)
    assert cut.truncated and k == len(full.cnode) // 3
    assert np.array_equal(cut.cnode, full.cnode[:k]) and np.array_equal(cut.parent, full.parent[:k])


def test_paths_by_depth_first_enumeration(oracle_lib, plain):
    """The same paths, found by a depth-first walk written here."""
    b, keys, g = plain
    q = 1
    t = oracle.expand(b, g, q, BIG)
    inc, a = g.incl[q], g.a[q]
    out = collections.defaultdict(list)
    has_caller = np.zeros(g.V, bool)
    for e in range(len(b.cs_caller)):
        gv, hv = int(g.cnode_of_func[b.cs_caller[e]]), int(g.cnode_of_func[b.cs_callee[e]])
        if gv != hv:
            out[gv].append((e, hv))
            has_caller[hv] = True
    live = set(g.cnode_of_func.tolist())
    found = collections.Counter()
    stack = [(v, 1.0) for v in sorted(live) if not has_caller[v] and inc[v, -1] > 0]
    while stack:
        v, sc = stack.pop()
        found[(v, round(sc, 12))] += 1
        for e, h in out[v]:
            r = a[e, -1] / inc[h, -1] if inc[h, -1] > 0 else 0.0
            if sc * r > 0:
                stack.append((h, sc * r))
    got = collections.Counter((int(v), round(s, 12)) for v, s in zip(t.cnode, t.scale))
    assert got == found
    # the links: a child's parent comes before it, its call site leads from the
    # parent's condensed node to its own, and its scale is the parent's times
    # that call site's ratio
    NP = 0xFFFFFFFF
    for i in range(len(t.cnode)):
        p, e = int(t.parent[i]), int(t.edge[i])
        if p == NP:
            assert e == NP and t.scale[i] == 1.0
            continue
        assert p < i
        assert int(g.cnode_of_func[b.cs_caller[e]]) == int(t.cnode[p])
        assert int(g.cnode_of_func[b.cs_callee[e]]) == int(t.cnode[i])
        r = a[e, -1] / inc[int(t.cnode[i]), -1]
        assert abs(t.scale[i] - t.scale[p] * r) <= 1e-12 * t.scale[i]
