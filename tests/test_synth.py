"""Seeded input generators: the shapes the workloads promise (they hold none
of the method's arithmetic)."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("n,depth", [(1, 4), (1000, 8), (50_000, 64)])
def test_level_cct_shape(n, depth):
    p = synth.make_cct_levels(3, n, depth, 8)
    assert p.shape == (n,) and p[0] == synth.NO_PARENT
    assert np.all(p[1:] < np.arange(1, n))                       # parents come first
    assert np.bincount(p[1:].astype(np.int64), minlength=n).max(initial=0) <= 8
    d = np.zeros(n, np.int64)
    for v in range(1, n):
        d[v] = d[p[v]] + 1
    assert d.max() <= depth
    assert np.array_equal(p, synth.make_cct_levels(3, n, depth, 8))   # seeded


def test_tuple_samples_stay_on_their_tuples():
    b = synth.PLAIN.binary()
    s = synth.make_tuple_samples(9, b, 20_000, 5000, 300)
    rng = np.searchsorted(b.range_lo, s.pc.numpy().view(np.uint64), side="right") - 1
    keys = set(zip(s.ctx.numpy().tolist(), rng.tolist(), s.stall.numpy().tolist()))
    assert len(keys) <= 300
    assert np.all(s.pc.numpy().view(np.uint64) < b.range_hi[rng])

