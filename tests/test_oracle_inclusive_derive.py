"""Pins of the oracle's inclusive propagation (Section 6.1) and derived
metrics (Section 4.5, Section 7).

Inclusive: brute-force subtree sums over explicit child lists, and the closed
form root-inclusive = sum of all exclusive values.  Derived: numpy's own
mean / population std / min / max on the dense profile matrix, the P = 1
special case, and W from its definition.
"""
from collections import defaultdict

import numpy as np
import pytest

import synth

U = 0xFFFFFFFF


def _keys(oracle_lib, rows):
    rows = sorted(map(tuple, rows))
    a = np.array(rows, dtype=np.uint64).reshape(-1, 4)
    return oracle_lib.KeyList(a[:, 0].astype(np.uint32), a[:, 1].astype(np.uint32), a[:, 2].astype(np.uint8),
                              a[:, 3].astype(np.uint64))


def test_structure_inclusive_brute(oracle_lib):
    w = synth.scaled(synth.PLAIN, 0.02)
    B = w.binary()
    k = oracle_lib.attribute_samples(B, w.samples(B))
    inc = oracle_lib.inclusive_structure(B.node_parent, k)
    # brute force: children lists, recursive subtree sum per (ctx, stall)
    kids = defaultdict(list)
    for n, p in enumerate(B.node_parent):
        if p != U:
            kids[int(p)].append(n)
    ex = defaultdict(int)
    for c, n, r, v in zip(k.ctx, k.node, k.stall, k.val):
        ex[(int(c), int(n), int(r))] += int(v)
    by_ctx_stall = defaultdict(dict)
    for (c, n, r), v in ex.items():
        by_ctx_stall[(c, r)][n] = v
    got = {(int(c), int(n), int(r)): int(v) for c, n, r, v in zip(inc.ctx, inc.node, inc.stall, inc.val)}
    checked = 0
    for (c, n, r), v in list(got.items())[::50]:
        if n == U:
            assert v == ex[(c, n, r)]
            continue
        stack, s = [n], 0
        while stack:
            x = stack.pop()
            s += by_ctx_stall[(c, r)].get(x, 0)
            stack.extend(kids[x])
        assert s == v
        checked += 1
    assert checked > 100
    # closed form: a function node's inclusive value = all its samples
    fsum = defaultdict(int)
    for (c, n, r), v in ex.items():
        if n != U:
            fsum[(c, int(B.func_node[B.node_func[n]]), r)] += v
    for key, v in fsum.items():
        assert got[key] == v
    # no key is invented: every output node is an ancestor-or-self of a sampled node
    assert len(got) >= len(ex)
    # UNKNOWN keys pass through unchanged (no function, no ancestors) ...
    unknown = {key: v for key, v in ex.items() if key[1] == U}
    assert unknown and all(got.get(key) == v for key, v in unknown.items())
    # ... so per (ctx, stall) the function nodes and UNKNOWN together hold every sample
    funcs = set(int(x) for x in B.func_node)
    tot_in, tot_out = defaultdict(int), defaultdict(int)
    for (c, n, r), v in ex.items():
        tot_in[(c, r)] += v
    for (c, n, r), v in got.items():
        if n == U or n in funcs:
            tot_out[(c, r)] += v
    assert tot_in == tot_out


def test_cct_inclusive(oracle_lib):
    par = synth.make_cct(9, 300, 12, 4)
    rng = np.random.default_rng(0)
    rows = {(int(rng.integers(0, 300)), int(rng.integers(0, 50)), int(rng.integers(0, 4))): int(rng.integers(1, 100))
            for _ in range(2000)}
    k = _keys(oracle_lib, [a + (v,) for a, v in rows.items()])
    host = oracle_lib.inclusive_cct(par, 4, k)
    # closed form at the root
    tot = np.zeros(4, np.uint64)
    np.add.at(tot, k.stall, k.val)
    assert host[0].tolist() == tot.tolist()
    # brute subtree sums
    kids = defaultdict(list)
    for v, p in enumerate(par):
        if p != U:
            kids[int(p)].append(v)
    exc = np.zeros((300, 4), np.uint64)
    np.add.at(exc, (k.ctx, k.stall), k.val)

    def sub(v):
        return exc[v] + sum((sub(c) for c in kids[v]), np.zeros(4, np.uint64))
    for v in range(0, 300, 7):
        assert host[v].tolist() == sub(v).tolist()


def test_derive_vs_numpy(oracle_lib):
    rng = np.random.default_rng(3)
    P, n_ctx, S = 5, 6, 4
    profiles, dense = [], {}
    for p in range(P):
        rows = {}
        for _ in range(60):
            key = (int(rng.integers(0, n_ctx)), int(rng.integers(0, 8)), int(rng.integers(0, S)))
            rows[key] = int(rng.integers(1, 1000))
        for key, v in rows.items():
            dense.setdefault(key, np.zeros(P))[p] = v
        profiles.append(_keys(oracle_lib, [a + (v,) for a, v in rows.items()]))
    d = oracle_lib.derive(profiles, n_ctx, S, issued_mask=0b0011)
    keys = sorted(dense)
    assert [(int(a), int(b), int(c)) for a, b, c in zip(d.ctx, d.node, d.stall)] == keys
    X = np.array([dense[k] for k in keys])
    np.testing.assert_array_equal(d.sum, X.sum(1))
    np.testing.assert_allclose(d.min, X.min(1), rtol=0)
    np.testing.assert_allclose(d.max, X.max(1), rtol=0)
    np.testing.assert_allclose(d.mean, X.mean(1), rtol=1e-15)
    np.testing.assert_allclose(d.std, X.std(1, ddof=0), rtol=1e-12)
    np.testing.assert_allclose(d.cov, X.std(1, ddof=0) / X.mean(1), rtol=1e-12)
    # W = (S - S_stall) / S with stall reasons 0 and 1 counted as issued
    for c in range(n_ctx):
        m = [i for i, k in enumerate(keys) if k[0] == c]
        s = X[m].sum()
        s_stall = sum(X[i].sum() for i in m if keys[i][2] >= 2)
        if s == 0:
            assert np.isnan(d.W[c])
        else:
            assert d.S[c] == s
            np.testing.assert_allclose(d.W[c], (s - s_stall) / s, rtol=1e-15)
            for r in range(S):
                np.testing.assert_allclose(d.frac[c, r], sum(X[i].sum() for i in m if keys[i][2] == r) / s,
                                           rtol=1e-15)


def test_derive_single_profile(oracle_lib):
    k = _keys(oracle_lib, [(0, 1, 0, 5), (0, 2, 1, 7), (1, 1, 0, 9)])
    d = oracle_lib.derive([k], 3, 2)
    np.testing.assert_array_equal(d.sum, [5, 7, 9])
    np.testing.assert_array_equal(d.min, d.max)
    np.testing.assert_array_equal(d.mean, [5, 7, 9])
    assert (d.std == 0).all() and (d.cov == 0).all()
    assert np.isnan(d.W[2]) and d.W[0] == 5 / 12 and d.W[1] == 1.0
