"""Pins of the oracle's warp issue rate per (launch context, function)
(Section 7: W = (S - S_stall) / S read per kernel and function): a
hand-computed example with two issue masks, conservation against the
per-context figures of the derived-metrics oracle (UNKNOWN samples belong to
no function), and the special masks (everything issued, nothing issued)."""
import numpy as np
import pytest

import synth

UNK = 0xFFFFFFFF


def _keys(o, rows):
    a = np.array(sorted(rows), dtype=np.uint64).reshape(-1, 4)
    return o.KeyList(a[:, 0].astype(np.uint32), a[:, 1].astype(np.uint32), a[:, 2].astype(np.uint8),
                     a[:, 3].astype(np.uint64))


# three functions: f0 = nodes 0 (FUNC), 1; f1 = nodes 2 (FUNC), 3, 4; f2 = nodes 5 (FUNC), 6
NODE_FUNC = np.array([0, 0, 1, 1, 1, 2, 2], np.uint32)
ROWS = [(0, 1, 0, 5), (0, 1, 2, 3), (0, 3, 0, 2), (0, 4, 1, 6), (0, UNK, 0, 7),
        (1, 0, 1, 4), (1, 6, 0, 1), (1, 6, 2, 1)]


@pytest.mark.parametrize("mask,W", [(0b001, [5 / 8, 2 / 8, 0.0, 1 / 2]), (0b101, [1.0, 2 / 8, 0.0, 1.0])])
def test_hand_example(oracle_lib, mask, W):
    r = oracle_lib.issue_by_function(NODE_FUNC, 3, _keys(oracle_lib, ROWS), mask)
    assert r.status == 0
    assert r.ctx.tolist() == [0, 0, 1, 1] and r.func.tolist() == [0, 1, 0, 2]
    assert r.S.tolist() == [8, 8, 4, 2]
    issued = {0b001: [5, 2, 0, 1], 0b101: [8, 2, 0, 2]}[mask]
    assert r.S_issued.tolist() == issued
    np.testing.assert_allclose(r.W, W, rtol=0, atol=1e-15)
    np.testing.assert_allclose(r.frac, [[5 / 8, 0, 3 / 8], [2 / 8, 6 / 8, 0], [0, 1, 0], [1 / 2, 0, 1 / 2]],
                               rtol=0, atol=1e-15)


def test_invalid_key(oracle_lib):
    r = oracle_lib.issue_by_function(NODE_FUNC, 3, _keys(oracle_lib, [(0, 9, 0, 1)]), 1)
    assert r.status == 1
    r = oracle_lib.issue_by_function(NODE_FUNC, 3, _keys(oracle_lib, [(0, 2, 3, 1)]), 1)
    assert r.status == 1


@pytest.fixture(scope="module")
def workload(oracle_lib):
    B = synth.PLAIN.binary()
    S = synth.make_samples(7, B, 200_000, 50, 1.1, counts=True)
    return B, oracle_lib.attribute_samples(B, S)


def test_conservation_against_per_context(oracle_lib, workload):
    """Summed over its functions plus its UNKNOWN samples, a context has the
    S and S_issued of the per-context warp issue rate."""
    B, k = workload
    mask = 0b1011
    r = oracle_lib.issue_by_function(B.node_func, 16, k, mask)
    d = oracle_lib.derive([k], 50, 16, mask)
    S = np.zeros(50, np.uint64)
    Si = np.zeros(50, np.uint64)
    np.add.at(S, r.ctx, r.S)
    np.add.at(Si, r.ctx, r.S_issued)
    unk = k.node == UNK
    np.add.at(S, k.ctx[unk], k.val[unk])
    iss = unk & (((mask >> k.stall.astype(np.int64)) & 1) == 1)
    np.add.at(Si, k.ctx[iss], k.val[iss])
    assert np.array_equal(S, d.S) and np.array_equal(Si, d.S_issued)
    assert np.all(np.diff(r.ctx.astype(np.int64) * (1 << 32) + r.func) > 0)
    np.testing.assert_allclose(r.frac.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.W, r.S_issued / r.S, rtol=1e-15)


@pytest.mark.parametrize("mask,w", [(0xFFFF, 1.0), (0, 0.0)])
def test_special_masks(oracle_lib, workload, mask, w):
    B, k = workload
    r = oracle_lib.issue_by_function(B.node_func, 16, k, mask)
    assert len(r.W) > 0 and np.all(r.W == w)
