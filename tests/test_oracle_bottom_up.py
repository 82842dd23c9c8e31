"""Pins of the oracle's bottom-up view (Section 7: a function's costs divided
among the calling contexts in which it is called), independent of
oracle.cpp's own arithmetic: a hand example, the roots against the flat
view, and every node's value and the node set of every level by brute force
over the contexts' call-site chains."""
import collections

import numpy as np
import pytest

import oracle
import synth

U = oracle.UNKNOWN
NP = synth.NO_PARENT
F = 0xFFFF


def keys(rows):
    a = np.array(rows, dtype=np.uint64).reshape(-1, 4)
    return oracle.KeyList(a[:, 0].astype(np.uint32), a[:, 1].astype(np.uint32), a[:, 2].astype(np.uint8),
                          a[:, 3].astype(np.uint64))


# structure: nodes 0, 1 in function 0; nodes 2, 3 in function 1
HAND_FUNC = np.array([0, 0, 1, 1], np.uint32)
# CCT: 0 root; 1, 2 children of 0; 3 under 1 and 4 under 2 share call site (2, 0x40)
HAND_CCT = (np.array([NP, 0, 0, 1, 2], np.uint32), np.array([1, 1, 1, 2, 2], np.uint16),
            np.array([0x100, 0x200, 0x300, 0x40, 0x40], np.uint64))
HAND_KEYS = [(1, 2, 0, 5), (3, 0, 0, 1), (3, 1, 1, 2), (3, 2, 0, 4), (4, 1, 1, 8), (4, U, 0, 9)]


def test_hand_example(oracle_lib):
    b = oracle.bottom_up(HAND_FUNC, keys(HAND_KEYS), HAND_CCT, 3)
    assert b.parent.tolist() == [NP, NP, 0, 1, 0, 2, 3, 4, 3, 6, 7, 8]
    assert b.func.tolist() == [1, 0, 1, 0, 1, 1, 0, 1, 0, 0, 1, 0]
    assert b.module.tolist() == [F, F, 1, 2, 2, 1, 1, 1, 1, 1, 1, 1]
    assert b.offset.tolist() == [0, 0, 0x200, 0x40, 0x40, 0x100, 0x200, 0x200, 0x300, 0x100, 0x100, 0x100]
    assert b.level_off.tolist() == [0, 2, 5, 9, 12]
    got = list(zip(b.vnode.tolist(), b.vstall.tolist(), b.val.tolist()))
    assert got == [(0, 0, 9), (1, 0, 1), (1, 1, 10), (2, 0, 5), (3, 0, 1), (3, 1, 10), (4, 0, 4), (5, 0, 5),
                   (6, 0, 1), (6, 1, 2), (7, 0, 4), (8, 1, 8), (9, 0, 1), (9, 1, 2), (10, 0, 4), (11, 1, 8)]


def test_hand_example_cut(oracle_lib):
    b = oracle.bottom_up(HAND_FUNC, keys(HAND_KEYS), HAND_CCT, 1)
    assert b.level_off.tolist() == [0, 2, 5] and b.parent.tolist() == [NP, NP, 0, 1, 0]
    b0 = oracle.bottom_up(HAND_FUNC, keys(HAND_KEYS), HAND_CCT, 0)
    assert b0.level_off.tolist() == [0, 2] and b0.val.tolist() == [9, 1, 10]


def workload(seed, n_samples, n_ctx, n_sites):
    w = synth.PLAIN
    bn = w.binary()
    s = synth.make_samples(seed, bn, n_samples, n_ctx, 1.1, counts=True)
    p = oracle.attribute_samples(bn, s)
    par = synth.make_cct(seed, n_ctx, 12, 4)
    mod, off, _ = synth.cct_sites(seed, par, n_sites, fan=4)
    return bn, p, (par, mod, off)


def chains(cct):
    par, mod, off = cct
    out = []
    for c in range(len(par)):
        ch, v = [], c
        while v != NP:
            ch.append((int(mod[v]), int(off[v])))
            v = int(par[v])
        out.append(tuple(ch))
    return out


def node_label_path(b, i):
    path = []
    while i != NP:
        path.append(i)
        i = int(b.parent[i])
    path.reverse()
    return int(b.func[path[0]]), tuple((int(b.module[j]), int(b.offset[j])) for j in path[1:])


@pytest.mark.parametrize("levels,n_sites", [(20, 16), (2, 64), (20, 0)])
def test_brute_force(oracle_lib, levels, n_sites):
    bn, p, cct = workload(31, 4000, 120, n_sites)
    b = oracle.bottom_up(bn.node_func, p, cct, levels)
    ch = chains(cct)
    known = p.node != U
    kf = np.where(known, bn.node_func[np.minimum(p.node, len(bn.node_func) - 1)], U)
    # the node set of every level: the distinct (function, chain prefix) pairs
    for lev in range(levels + 1):
        want = {(int(f), ch[int(c)][:lev]) for f, c, ok in zip(kf, p.ctx, known)
                if ok and len(ch[int(c)]) >= lev}
        ids = range(int(b.level_off[lev]), int(b.level_off[lev + 1]))
        got = [node_label_path(b, i) for i in ids]
        assert len(got) == len(set(got)) and set(got) == want
    # every node's value per stall: the keys of its function whose chain begins with the node's
    vals = collections.defaultdict(dict)
    for n, r, v in zip(b.vnode.tolist(), b.vstall.tolist(), b.val.tolist()):
        vals[n][r] = v
    for i in range(0, len(b.parent), 3):
        f, pre = node_label_path(b, i)
        want = collections.Counter()
        for j in np.nonzero(known & (kf == f))[0]:
            if ch[int(p.ctx[j])][:len(pre)] == pre:
                want[int(p.stall[j])] += int(p.val[j])
        assert vals[i] == dict(want)
    # values ascending by (node, stall); parents in the level before
    o = b.vnode.astype(np.int64) * 64 + b.vstall
    assert np.all(np.diff(o) > 0)
    for lev in range(1, levels + 1):
        sl = slice(int(b.level_off[lev]), int(b.level_off[lev + 1]))
        assert np.all((b.parent[sl] >= b.level_off[lev - 1]) & (b.parent[sl] < b.level_off[lev]))


def test_roots_are_the_flat_view_by_function(oracle_lib):
    bn, p, cct = workload(32, 20_000, 300, 32)
    b = oracle.bottom_up(bn.node_func, p, cct, 4)
    f = oracle.flat(16, p)
    m = f.node != U
    want = collections.Counter()
    for n, r, v in zip(f.node[m], f.stall[m], f.val[m]):
        want[(int(bn.node_func[n]), int(r))] += int(v)
    got = {(int(b.func[n]), r): v for n, r, v in zip(b.vnode.tolist(), b.vstall.tolist(), b.val.tolist())
           if n < b.level_off[1]}
    assert got == dict(want)
    # the first level in order of the first key of each function
    firsts = []
    for n in p.node[p.node != U]:
        fn = int(bn.node_func[n])
        if fn not in firsts:
            firsts.append(fn)
    assert b.func[: int(b.level_off[1])].tolist() == firsts
