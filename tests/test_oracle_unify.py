"""Pins of the oracle's call-path profile unification (Section 6.1),
independent of its code: a hand example, unifying a tree with its own
copies, and every input node's call path found again at its merged node."""
import numpy as np

import oracle
import synth

NP = synth.NO_PARENT


def cct(rows):
    a = list(zip(*rows))
    return (np.array(a[0], np.uint32), np.array(a[1], np.uint16), np.array(a[2], np.uint64))


def test_hand_example(oracle_lib):
    # call site (3, 7) under two parents in A stays two nodes; B's copy of it
    # under (2, 5) merges with A's
    A = cct([(NP, 1, 10), (0, 1, 20), (0, 2, 5), (1, 3, 7), (2, 3, 7)])
    B = cct([(NP, 1, 10), (0, 2, 5), (1, 1, 99), (1, 3, 7)])
    uid, up, um, uo = oracle.unify([A, B])
    assert uid.tolist() == [0, 1, 2, 3, 4, 0, 2, 5, 4]
    assert up.tolist() == [NP, 0, 0, 1, 2, 2]
    assert um.tolist() == [1, 1, 2, 3, 3, 1] and uo.tolist() == [10, 20, 5, 7, 7, 99]


def test_sites_differ_by_module(oracle_lib):
    # two call sites at one offset in different load modules are different sites
    A = cct([(NP, 1, 10), (0, 1, 5), (0, 2, 5)])
    B = cct([(NP, 1, 10), (0, 2, 5)])
    uid, up, um, uo = oracle.unify([A, B])
    assert uid.tolist() == [0, 1, 2, 0, 2] and um.tolist() == [1, 1, 2] and uo.tolist() == [10, 5, 5]


def test_copies_unify_to_the_original(oracle_lib):
    c = synth.make_profile_ccts(5, 3000, 20, 1, 1.0)[0]
    uid, up, um, uo = oracle.unify([c, c, c])
    n = len(c[0])
    assert len(up) == n
    assert np.array_equal(uid, np.tile(np.arange(n, dtype=np.uint32), 3))
    assert np.array_equal(up, c[0]) and np.array_equal(um, c[1]) and np.array_equal(uo, c[2])


def _path(par, mod, off, i):
    out = []
    while i != NP:
        out.append((int(mod[i]), int(off[i])))
        i = int(par[i])
    return out


def test_paths_are_kept(oracle_lib):
    ccts = synth.make_profile_ccts(8, 4000, 24, 5, 0.2)
    uid, up, um, uo = oracle.unify(ccts)
    # the merged tree: parents first, no two children of one parent with one call site
    assert all(p == NP or p < i for i, p in enumerate(up.tolist()))
    assert len({(int(p), int(m), int(o)) for p, m, o in zip(up, um, uo)}) == len(up)
    k = 0
    for par, mod, off in ccts:
        for j in range(0, len(par), 17):
            assert _path(par, mod, off, j) == _path(up, um, uo, int(uid[k + j]))
        k += len(par)
    # every node of the union of the subsets, once: the master tree's kept nodes
    union = {tuple(_path(par, mod, off, j)) for par, mod, off in ccts for j in range(len(par))}
    assert len(union) == len(up)
    # call sites do repeat under different parents
    assert len({(int(m), int(o)) for m, o in zip(um, uo)}) < len(up) // 2
