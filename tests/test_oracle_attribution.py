"""Pins of the oracle's attribution + aggregation (Sections 4.2, 4.5, 5).

Each check is independent of oracle.cpp: a hand-computed fixture, an O(N*R)
brute-force scan, conservation of counts, and the generator's own knowledge
of which function every sample was drawn from.
"""
import json
import os
from collections import Counter

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
U = 0xFFFFFFFF


def brute(lo, hi, node, pc, ctx, stall, count):
    """Linear scan over every range for every sample, then a Counter."""
    pc = np.asarray(pc, np.uint64)
    inside = (pc[:, None] >= lo[None, :]) & (pc[:, None] < hi[None, :])
    assert (inside.sum(1) <= 1).all()
    hit = inside.any(1)
    nd = np.where(hit, node[np.argmax(inside, 1)], U)
    agg = Counter()
    for i in range(pc.shape[0]):
        agg[(int(ctx[i]), int(nd[i]), int(stall[i]))] += 1 if count is None else int(count[i])
    return sorted((k + (v,)) for k, v in agg.items() if v)


def as_rows(k):
    return [(int(a), int(b), int(c), int(d)) for a, b, c, d in zip(k.ctx, k.node, k.stall, k.val)]


def test_golden_fixture(oracle_lib):
    g = json.load(open(os.path.join(GOLD, "attribution_small.json")))
    s = np.array(g["samples"], dtype=np.uint64)
    B = synth.Binary(np.array(g["range_lo"], np.uint64), np.array(g["range_hi"], np.uint64),
                     np.array(g["range_node"], np.uint32), *[np.zeros(0)] * 10, 0, 0)
    k = oracle_lib.attribute(B, s[:, 0], s[:, 1].astype(np.uint32), s[:, 2].astype(np.uint8),
                             s[:, 3].astype(np.uint32), g["n_ctx"], g["n_stall"])
    assert k.status == 0
    assert as_rows(k) == [tuple(r) for r in g["expected_keys"]]
    assert k.total.tolist() == g["expected_total"]
    assert k.unknown.tolist() == g["expected_unknown"]


@pytest.mark.parametrize("seed,counts", [(1, False), (2, True), (3, True)])
def test_brute_force_small(oracle_lib, seed, counts):
    B = synth.make_binary(seed, 10, 10 * 4096, 150, 15, n_scc=1 if seed == 3 else 0,
                          scc_size=(2, 3), min_fn_bytes=2048, max_fn_bytes=8192)
    S = synth.make_samples(seed, B, 3000, 7, 1.0, n_stall=5, counts=counts)
    # add boundary PCs: every lo, hi - 1, hi, and addresses outside the segment
    extra = np.concatenate([B.range_lo, B.range_hi - np.uint64(1), B.range_hi,
                            np.array([0, B.seg_lo - 1, B.seg_hi, 2 ** 64 - 1], np.uint64)])
    m = extra.shape[0]
    pc = np.concatenate([S.pc.numpy().view(np.uint64), extra])
    ctx = np.concatenate([S.ctx.numpy().view(np.uint32), (np.arange(m) % 7).astype(np.uint32)])
    st = np.concatenate([S.stall.numpy(), (np.arange(m) % 5).astype(np.uint8)])
    cnt = None
    if counts:
        cnt = np.concatenate([S.count.numpy().view(np.uint32), (np.arange(m) % 3).astype(np.uint32)])
    k = oracle_lib.attribute(B, pc, ctx, st, cnt, 7, 5)
    assert k.status == 0
    assert as_rows(k) == brute(B.range_lo, B.range_hi, B.range_node, pc, ctx, st, cnt)


def test_conservation_and_generator_truth(oracle_lib):
    """Sum of values + UNKNOWN = sum of counts per stall reason, and every
    attributed node lies in the function the generator drew the PC from."""
    w = synth.scaled(synth.PLAIN, 0.1)
    B = w.binary()
    S = w.samples(B)
    k = oracle_lib.attribute_samples(B, S)
    assert k.status == 0
    st = S.stall.numpy()
    tot = np.bincount(st, minlength=16)
    assert k.total.tolist() == tot.tolist()
    per = np.zeros(16, np.uint64)
    np.add.at(per, k.stall, k.val)
    assert per.tolist() == tot.tolist()
    unk = np.zeros(16, np.uint64)
    m = k.node == U
    np.add.at(unk, k.stall[m], k.val[m])
    assert unk.tolist() == k.unknown.tolist()
    # generator truth: the sample's function, from the function table alone
    pc = S.pc.numpy().view(np.uint64)
    f = np.searchsorted(B.func_lo, pc, side="right") - 1
    assert ((pc >= B.func_lo[f]) & (pc < B.func_hi[f])).all()
    # re-attribute each sample via the oracle's per-key output: keys of a ctx
    # must belong to functions that ctx actually sampled
    drawn = {}
    for c, fn in zip(S.ctx.numpy(), f):
        drawn.setdefault(int(c), set()).add(int(fn))
    for c, n in zip(k.ctx[~m], k.node[~m]):
        assert int(B.node_func[n]) in drawn[int(c)]
    # and per (ctx, function) totals agree with the draw
    got = Counter()
    for c, n, v in zip(k.ctx[~m], k.node[~m], k.val[~m]):
        got[(int(c), int(B.node_func[n]))] += int(v)
    exp = Counter()
    covered = np.ones(pc.shape[0], bool)
    # samples in a function's padding are UNKNOWN: padding = slots not in any range
    i = np.searchsorted(B.range_lo, pc, side="right") - 1
    covered = (i >= 0) & (pc < B.range_hi[np.maximum(i, 0)])
    for c, fn, cv in zip(S.ctx.numpy(), f, covered):
        if cv:
            exp[(int(c), int(fn))] += 1
    assert got == exp


def test_invalid_records_fail_whole_call(oracle_lib):
    B = synth.make_binary(4, 4, 4 * 4096, 20, 3, min_fn_bytes=2048, max_fn_bytes=8192)
    pc = np.array([B.range_lo[0]] * 4, np.uint64)
    k = oracle_lib.attribute(B, pc, np.array([0, 5, 1, 9], np.uint32), np.array([0, 1, 7, 1], np.uint8), None, 6, 4)
    assert k.status == 3 and k.bad == 2 and len(k) == 0


def test_empty_input(oracle_lib):
    B = synth.make_binary(4, 4, 4 * 4096, 20, 3, min_fn_bytes=2048, max_fn_bytes=8192)
    e = np.zeros(0, np.uint64)
    k = oracle_lib.attribute(B, e, e.astype(np.uint32), e.astype(np.uint8), None, 3, 4)
    assert k.status == 0 and len(k) == 0 and k.total.sum() == 0
