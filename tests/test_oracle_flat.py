"""Pins of the oracle's flat view (Section 7: costs by static structure,
every calling context pooled), independent of oracle.cpp's own arithmetic."""
import numpy as np

import oracle
import synth

U = oracle.UNKNOWN


def keys(rows):
    a = np.array(rows, dtype=np.uint64).reshape(-1, 4)
    return oracle.KeyList(a[:, 0].astype(np.uint32), a[:, 1].astype(np.uint32), a[:, 2].astype(np.uint8),
                          a[:, 3].astype(np.uint64))


def test_hand_computed_example(oracle_lib):
    # contexts 0..2; node 4 stall 1 appears in three contexts, UNKNOWN in two
    k = keys([(0, 4, 1, 5), (0, 7, 0, 2), (0, U, 3, 1), (1, 2, 0, 9), (1, 4, 1, 6),
              (2, 4, 0, 1), (2, 4, 1, 10), (2, U, 3, 4)])
    f = oracle.flat(4, k)
    got = list(zip(f.ctx.tolist(), f.node.tolist(), f.stall.tolist(), f.val.tolist()))
    assert got == [(0, 2, 0, 9), (0, 4, 0, 1), (0, 4, 1, 21), (0, 7, 0, 2), (0, U, 3, 5)]
    assert f.total.tolist() == [12, 21, 0, 5] and f.unknown.tolist() == [0, 0, 0, 5]


def test_conservation_and_order_on_a_profile(oracle_lib):
    b = synth.PLAIN.binary()
    s = synth.make_samples(12, b, 60_000, 40, 1.1, counts=True)
    p = oracle.attribute_samples(b, s)
    f = oracle.flat(16, p)
    # per stall, the flat values add up to the samples' counts (the profile's totals)
    assert np.array_equal(f.total, p.total) and np.array_equal(f.unknown, p.unknown)
    assert f.val.sum() == s.count.numpy().astype(np.uint64).sum()
    # strictly ascending (node, stall), one context
    order = f.node.astype(np.uint64) << np.uint64(8) | f.stall.astype(np.uint64)
    assert np.all(np.diff(order.astype(np.float64)) > 0) and not f.ctx.any()
    # every (node, stall) of the flat view is the sum of that pair over contexts, by brute force
    for i in range(0, len(f), max(1, len(f) // 50)):
        m = (p.node == f.node[i]) & (p.stall == f.stall[i])
        assert int(p.val[m].sum()) == int(f.val[i])


def test_one_context_is_the_identity(oracle_lib):
    b = synth.PLAIN.binary()
    s = synth.make_samples(13, b, 30_000, 1, 1.1)
    p = oracle.attribute_samples(b, s)
    f = oracle.flat(16, p)
    assert np.array_equal(f.node, p.node) and np.array_equal(f.stall, p.stall) and np.array_equal(f.val, p.val)
