"""Pins of the oracle's ratio of raw metrics (Section 4.5: a quantity known
once per kernel invocation is recovered by dividing two raw metrics that were
summed over threads and ranks: the quantity summed over invocations, and the
count of invocations).  A hand-computed example in those terms, the closed
form of a numerator that is a multiple of the denominator, invariance under
splitting a profile into thread profiles, reciprocity when the groups swap,
and conservation of both sums."""
import numpy as np
import pytest

import synth

UNK = 0xFFFFFFFF


def _keys(o, rows):
    if not rows:
        z = np.zeros(0, np.uint64)
        return o.KeyList(z.astype(np.uint32), z.astype(np.uint32), z.astype(np.uint8), z)
    a = np.array(sorted(rows), dtype=np.uint64).reshape(-1, 4)
    return o.KeyList(a[:, 0].astype(np.uint32), a[:, 1].astype(np.uint32), a[:, 2].astype(np.uint8),
                     a[:, 3].astype(np.uint64))


# Two ranks ran two kernels.  Kernel A (context 0, node 3) used 32 registers
# per invocation: rank 0 saw 2 invocations, rank 1 saw 1.  Kernel B (context
# 1, node 3) used 40 registers: 3 invocations on rank 0 and 2 on rank 1.  The
# numerator profiles hold registers summed over invocations, the denominator
# profiles the invocation counts.  Context 2 appears only in the numerator
# (no invocation count recorded: NaN); context 3 only in the denominator
# (ratio 0).  An UNKNOWN node is a key like any other.
NUM = [[(0, 3, 0, 64), (1, 3, 0, 120), (2, 5, 1, 7)],
       [(0, 3, 0, 32), (1, 3, 0, 80), (4, UNK, 0, 9)]]
DEN = [[(0, 3, 0, 2), (1, 3, 0, 3), (3, 1, 0, 4)],
       [(0, 3, 0, 1), (1, 3, 0, 2), (4, UNK, 0, 3)]]


def test_hand_example(oracle_lib):
    o = oracle_lib
    r = o.ratio([_keys(o, p) for p in NUM], [_keys(o, p) for p in DEN])
    assert r.ctx.tolist() == [0, 1, 2, 3, 4]
    assert r.node.tolist() == [3, 3, 5, 1, UNK]
    assert r.stall.tolist() == [0, 0, 1, 0, 0]
    assert r.num.tolist() == [96, 200, 7, 0, 9]
    assert r.den.tolist() == [3, 5, 0, 4, 3]
    assert r.ratio[0] == 32.0 and r.ratio[1] == 40.0 and np.isnan(r.ratio[2])
    assert r.ratio[3] == 0.0 and r.ratio[4] == 3.0


def test_empty_groups(oracle_lib):
    o = oracle_lib
    r = o.ratio([_keys(o, [])], [_keys(o, [])])
    assert r.num.shape == (0,)
    r = o.ratio([_keys(o, NUM[0])], [])
    assert r.den.tolist() == [0, 0, 0] and np.isnan(r.ratio).all()


@pytest.fixture(scope="module")
def profile(oracle_lib):
    B = synth.PLAIN.binary()
    S = synth.make_samples(11, B, 60_000, 40, 1.1, counts=True)
    return oracle_lib.attribute_samples(B, S)


def _scaled(o, k, f):
    return o.KeyList(k.ctx, k.node, k.stall, (k.val * np.uint64(f)).astype(np.uint64))


def test_multiple_of_denominator(oracle_lib, profile):
    """num = 7 * den key by key gives ratio 7 exactly on every key."""
    o = oracle_lib
    r = o.ratio([_scaled(o, profile, 7)], [profile])
    assert r.num.shape[0] == profile.val.shape[0]
    np.testing.assert_array_equal(r.ctx, profile.ctx)
    np.testing.assert_array_equal(r.den, profile.val)
    np.testing.assert_array_equal(r.num, profile.val * np.uint64(7))
    assert (r.ratio == 7.0).all()


def _split(o, k, seed):
    """Two thread profiles whose values add up to k's, key by key; a key
    whose share is 0 is left out of that profile."""
    rng = np.random.default_rng(seed)
    a = (rng.random(k.val.shape[0]) * (k.val.astype(np.float64) + 1)).astype(np.uint64)
    a = np.minimum(a, k.val)
    b = k.val - a
    ma, mb = a > 0, b > 0
    pa = o.KeyList(k.ctx[ma], k.node[ma], k.stall[ma], a[ma])
    pb = o.KeyList(k.ctx[mb], k.node[mb], k.stall[mb], b[mb])
    return pa, pb


def test_split_into_threads(oracle_lib, profile):
    """Summing over threads first: a group of two thread profiles that add up
    to one profile gives the same rows as that profile."""
    o = oracle_lib
    den = _scaled(o, profile, 3)
    den.val[::5] = 1
    whole = o.ratio([profile], [den])
    pa, pb = _split(o, profile, 5)
    da, db = _split(o, den, 6)
    parts = o.ratio([pa, pb], [da, db])
    for f in ("ctx", "node", "stall", "num", "den"):
        np.testing.assert_array_equal(getattr(parts, f), getattr(whole, f))
    np.testing.assert_array_equal(parts.ratio, whole.ratio)


def test_swap_and_conservation(oracle_lib, profile):
    """Swapping the groups swaps num and den and inverts every ratio; the
    rows carry every numerator and denominator value once."""
    o = oracle_lib
    B = synth.PLAIN.binary()
    other = o.attribute_samples(B, synth.make_samples(12, B, 40_000, 40, 1.1, counts=True))
    r = o.ratio([profile], [other])
    s = o.ratio([other], [profile])
    np.testing.assert_array_equal(r.num, s.den)
    np.testing.assert_array_equal(r.den, s.num)
    both = (r.num > 0) & (r.den > 0)
    assert both.any() and (~both).any()
    np.testing.assert_allclose(r.ratio[both] * s.ratio[both], 1.0, rtol=1e-15)
    assert int(r.num.sum()) == int(profile.val.sum())
    assert int(r.den.sum()) == int(other.val.sum())
    keys = set(zip(profile.ctx.tolist(), profile.node.tolist(), profile.stall.tolist()))
    keys |= set(zip(other.ctx.tolist(), other.node.tolist(), other.stall.tolist()))
    assert r.num.shape[0] == len(keys)
    assert np.isnan(r.ratio[r.den == 0]).all()
