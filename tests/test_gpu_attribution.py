"""GPU parity of attribution + aggregation (Sections 4.2, 4.5, 5) against the
CPU oracle: every key, node id and count bit-exact."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_same_keys, samples_from_numpy

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def H():
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0)
    yield h
    h.close()


@pytest.fixture(scope="module")
def plain(H):
    B = synth.PLAIN.binary()
    return B, H.load_structure(B)


@pytest.fixture(scope="module")
def large_bin(H):
    B = synth.LARGE.binary()
    return B, H.load_structure(B)


def run(H, bid, S, **kw):
    out = H.attribute_samples(bid, S, **kw)
    H.sync()
    return out


def test_golden_fixture(H):
    g = json.load(open(os.path.join(GOLD, "attribution_small.json")))
    s = np.array(g["samples"], dtype=np.uint64)
    M = 10
    B = synth.Binary(np.array(g["range_lo"], np.uint64), np.array(g["range_hi"], np.uint64),
                     np.array(g["range_node"], np.uint32), np.full(M, synth.NO_PARENT, np.uint32),
                     np.zeros(M, np.uint8), np.arange(M, dtype=np.uint32), np.arange(M, dtype=np.uint32),
                     np.zeros(M, np.uint64), np.zeros(M, np.uint64), np.zeros(0, np.uint64),
                     np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.uint32), 0, 0)
    bid = H.load_structure(B)
    S = samples_from_numpy(s[:, 0], s[:, 1], s[:, 2], s[:, 3], g["n_ctx"], g["n_stall"])
    out = run(H, bid, S)
    got = list(zip(*[a.tolist() for a in out.numpy()]))
    assert [list(r) for r in got] == g["expected_keys"]
    assert out.total[:4].cpu().tolist() == g["expected_total"]
    assert out.unknown[:4].cpu().tolist() == g["expected_unknown"]


@pytest.mark.parametrize("frac,counts", [(0.01, False), (0.2, False), (1.0, False), (0.3, True)])
def test_plain_workload(H, plain, frac, counts):
    B, bid = plain
    w = synth.scaled(synth.PLAIN, frac)
    w.counts = counts
    S = w.samples(B, device="cuda")
    out = run(H, bid, S)
    assert_same_keys(out, oracle.attribute_samples(B, S))


@pytest.mark.parametrize("n", [0, 1, 31, 4095, 4096, 4097, 12289])
def test_ragged_sizes(H, plain, n):
    B, bid = plain
    S = synth.make_samples(77, B, n, 13, 1.1, device="cuda")
    out = run(H, bid, S)
    assert_same_keys(out, oracle.attribute_samples(B, S))


@pytest.mark.parametrize("n_ctx", [1, 2, 7])
def test_big_groups(H, plain, n_ctx):
    """Few contexts: every group exceeds a leaf and is split into sub-bins."""
    B, bid = plain
    S = synth.make_samples(5, B, 300_000, n_ctx, 1.1, counts=True, device="cuda")
    out = run(H, bid, S)
    assert_same_keys(out, oracle.attribute_samples(B, S))


def test_heavy_sub_bin(H, plain):
    """All samples in one function of one context: a sub-bin far larger than a
    leaf, aggregated in dense shared-memory windows."""
    B, bid = plain
    f = 17
    n = 400_000
    idx = np.arange(n)
    slots = int((B.func_hi[f] - B.func_lo[f]) // 16)
    pc = B.func_lo[f] + (synth.np_below(3, 1, idx, slots) * 16).astype(np.uint64)
    st = synth.np_below(3, 2, idx, 16).astype(np.uint8)
    S = samples_from_numpy(pc, np.zeros(n, np.uint32), st, None, 1, 16)
    out = run(H, bid, S)
    assert_same_keys(out, oracle.attribute_samples(B, S))


def test_skewed_contexts(H, large_bin):
    """A few hot contexts next to many cold ones, structure of the large binary."""
    B, bid = large_bin
    wts = np.ones(3000)
    wts[[5, 900, 2999]] = 2000.0
    S = synth.make_samples(9, B, 1_500_000, 3000, 0.9, counts=True, device="cuda", ctx_weights=wts)
    out = run(H, bid, S)
    assert_same_keys(out, oracle.attribute_samples(B, S))


@pytest.mark.parametrize("cap", [4096, 10240])
def test_leaf_capacity_variants_agree(cap, plain):
    from paper_2109_06931_gb300 import hpa
    B, _ = plain
    h = hpa.Hpa(0, leaf_capacity=cap)
    bid = h.load_structure(B)
    S = synth.make_samples(11, B, 500_000, 40, 1.1, counts=True, device="cuda")
    out = h.attribute_samples(bid, S)
    h.sync()
    assert_same_keys(out, oracle.attribute_samples(B, S))
    h.close()


def test_large_structure(H, large_bin):
    B, bid = large_bin
    S = synth.LARGE.samples(B, device="cuda", n=3_000_000)
    out = run(H, bid, S)
    assert_same_keys(out, oracle.attribute_samples(B, S))


def test_invalid_samples_fail_whole_call(H, plain):
    from paper_2109_06931_gb300 import hpa
    B, bid = plain
    S = synth.make_samples(2, B, 10_000, 8, 1.1, device="cuda")
    S.ctx[5] = 8
    S.ctx[77] = 1000
    S.stall[100] = 16
    out = H.attribute_samples(bid, S)
    st, bad = H.sync_status()
    assert st == hpa.HPA_E_INVALID_SAMPLE and bad == 3
    assert out.count() == 0
    # the handle keeps working afterwards
    S2 = synth.make_samples(2, B, 10_000, 8, 1.1, device="cuda")
    assert_same_keys(run(H, bid, S2), oracle.attribute_samples(B, S2))


def test_capacity_too_small(H, plain):
    from paper_2109_06931_gb300 import hpa
    B, bid = plain
    S = synth.make_samples(4, B, 50_000, 30, 1.1, device="cuda")
    ref = oracle.attribute_samples(B, S)
    out = H.attribute_samples(bid, S, capacity=len(ref) - 1)
    st, _ = H.sync_status()
    assert st == hpa.HPA_E_CAPACITY and out.count() == len(ref)
    out = H.attribute_samples(bid, S, capacity=len(ref))
    H.sync()
    assert_same_keys(out, ref)


def test_batch_equals_plain_runs(H, plain, large_bin):
    B1, b1 = plain
    B2, b2 = large_bin
    sizes = [0, 1, 5000, 70_000, 4096, 200_000, 33_333]
    ss, bins, bs = [], [], []
    for i, n in enumerate(sizes):
        B, bid = (B1, b1) if i % 2 == 0 else (B2, b2)
        ss.append(synth.make_samples(100 + i, B, n, 50 + 30 * i, 1.0, counts=(i % 3 == 0), device="cuda"))
        bins.append(bid); bs.append(B)
    outs = H.attribute_batch(bins, ss)
    H.sync()
    for o, S, B in zip(outs, ss, bs):
        assert_same_keys(o, oracle.attribute_samples(B, S))


def test_host_entry_point(H, plain):
    B, bid = plain
    S = synth.make_samples(21, B, 100_000, 64, 1.1, counts=True)
    out = H.attribute_samples_host(bid, S.pc.numpy(), S.ctx.numpy(), S.stall.numpy(), S.count.numpy(), 64, 16)
    ref = oracle.attribute_samples(B, S)
    k = int(out["n"][0])
    assert k == len(ref)
    for a, b in zip((out["ctx"], out["node"], out["stall"], out["val"]), (ref.ctx, ref.node, ref.stall, ref.val)):
        assert np.array_equal(a[:k], b)
    assert np.array_equal(out["total"][:16], ref.total)


def test_batch_graph_replay_with_new_buffers(H, plain, large_bin):
    """Two batched calls with the same shape replay one captured graph; the
    second call's buffers hold different samples and must give their own
    results."""
    B1, b1 = plain
    B2, b2 = large_bin
    sizes = [50_000, 3, 120_000, 9_000]
    bins = [b1, b2, b1, b2]
    Bs = [B1, B2, B1, B2]
    for rep in range(3):
        ss = [synth.make_samples(500 + 10 * rep + i, Bs[i], n, 40 + i, 1.0, counts=(i != 2), device="cuda")
              for i, n in enumerate(sizes)]
        outs = H.attribute_batch(bins, ss)
        H.sync()
        for o, S, B in zip(outs, ss, Bs):
            assert_same_keys(o, oracle.attribute_samples(B, S))


@pytest.mark.parametrize("partition", [True, False])
@pytest.mark.parametrize("counts", [False, True])
def test_grouping_paths_agree(plain, large_bin, partition, counts):
    """Both ways of grouping records by context (per-part counters with
    shared-memory cursors, or per-context cursor atomics) give the oracle's
    keys and totals, on the small and the large structure."""
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0, partition=partition)
    for B, seed, n, n_ctx, z in ((plain[0], 21, 700_001, 300, 1.1), (large_bin[0], 22, 1_200_000, 2000, 0.9)):
        bid = h.load_structure(B)
        S = synth.make_samples(seed, B, n, n_ctx, z, counts=counts, device="cuda")
        out = h.attribute_samples(bid, S)
        h.sync()
        assert_same_keys(out, oracle.attribute_samples(B, S))
    h.close()


def test_many_contexts(H, plain):
    """More contexts than the partition path keeps in shared memory: the
    per-context cursor path runs and agrees with the oracle."""
    B, bid = plain
    S = synth.make_samples(31, B, 900_000, 40_000, 1.1, counts=True, device="cuda")
    out = run(H, bid, S)
    assert_same_keys(out, oracle.attribute_samples(B, S))


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_leaf_ranking_modes_agree(plain, mode):
    from paper_2109_06931_gb300 import hpa
    B, _ = plain
    h = hpa.Hpa(0, sort_mode=mode)
    bid = h.load_structure(B)
    S = synth.make_samples(41, B, 600_000, 50, 1.1, counts=True, device="cuda")
    out = h.attribute_samples(bid, S)
    h.sync()
    assert_same_keys(out, oracle.attribute_samples(B, S))
    h.close()


def test_tuner_keeps_results_and_picks_a_candidate(plain):
    """hpa_tune times every candidate configuration; each computes the same
    keys, and the handle keeps the fastest for later calls."""
    from paper_2109_06931_gb300 import hpa
    B, _ = plain
    h = hpa.Hpa(0)
    bid = h.load_structure(B)
    S = synth.make_samples(51, B, 400_000, 60, 1.1, counts=True, device="cuda")
    chosen, ms = h.tune(bid, S)
    assert len(ms) == hpa.HPA_TUNE_CANDIDATES and all(t > 0 for t in ms)
    assert chosen["leaf_capacity"] in (4096, 10240) and chosen["grouping"] in (0, 1)
    assert chosen["leaf_hash"] in (0, 1) and chosen["leaf_ranking"] in (1, 3)
    ref = oracle.attribute_samples(B, S)
    out = h.attribute_samples(bid, S)
    h.sync()
    assert_same_keys(out, ref)
    h.close()


def test_batch_split_into_sub_batches(H, plain, large_bin):
    """A batch whose contexts add up to more than one sub-batch takes (1M
    groups) runs as consecutive pipelines, in the graph and outside it; each
    buffer still gets exactly its own keys."""
    B1, b1 = plain
    B2, b2 = large_bin
    n_ctx = [1_500_000, 2_000_000, 3, 2_500_000, 900_000]
    ss, bins, bs = [], [], []
    for i, c in enumerate(n_ctx):
        B, bid = (B1, b1) if i % 2 == 0 else (B2, b2)
        ss.append(synth.make_tuple_samples(700 + i, B, 150_000 + 10_000 * i, c, 20_000, device="cuda"))
        bins.append(bid); bs.append(B)
    refs = [oracle.attribute_samples(B, S) for B, S in zip(bs, ss)]
    for rep in range(2):                                   # capture, then replay
        outs = H.attribute_batch(bins, ss)
        H.sync()
        for o, r in zip(outs, refs):
            assert_same_keys(o, r)
    H.set_phase_timing(True)                               # phase timing runs the pipelines eagerly
    outs = H.attribute_batch(bins, ss)
    H.sync()
    ph, calls = H.phase_times()
    H.set_phase_timing(False)
    assert calls == 1
    for o, r in zip(outs, refs):
        assert_same_keys(o, r)


@pytest.mark.parametrize("small", [1, 2])
def test_small_leaf_kernel_on_and_off(plain, small):
    """Leaves of up to 1024 records in the small-CTA kernel (2) or in the leaf
    capacity's kernel (1): same keys, for few and for many samples per context."""
    from paper_2109_06931_gb300 import hpa
    B, _ = plain
    h = hpa.Hpa(0, small_leaves=small)
    bid = h.load_structure(B)
    for S in (synth.make_tuple_samples(61, B, 500_000, 40_000, 30_000, device="cuda"),
              synth.make_samples(62, B, 400_000, 100, 1.1, counts=True, device="cuda")):
        out = h.attribute_samples(bid, S)
        h.sync()
        assert_same_keys(out, oracle.attribute_samples(B, S))
    h.close()


@pytest.mark.parametrize("small", [1, 2])
def test_hash_leaves_agree(plain, large_bin, small):
    """Hash aggregation inside leaves: many repeats (tuple samples), few
    repeats with counts (the large structure, where most leaves fall back to
    sorting), zero counts, and split groups."""
    from paper_2109_06931_gb300 import hpa
    B1, _ = plain
    B2, _ = large_bin
    h = hpa.Hpa(0, leaf_hash=1, small_leaves=small)
    b1, b2 = h.load_structure(B1), h.load_structure(B2)
    cases = [(B1, b1, synth.make_tuple_samples(71, B1, 600_000, 30_000, 20_000, device="cuda")),
             (B2, b2, synth.make_samples(72, B2, 800_000, 300, 0.9, counts=True, device="cuda")),
             (B1, b1, synth.make_samples(73, B1, 300_000, 2, 1.1, counts=True, device="cuda"))]
    S = synth.make_samples(74, B1, 200_000, 50, 1.1, counts=True, device="cuda")
    S.count[::3] = 0                                        # zero counts: keys that only sum to 0 vanish
    cases.append((B1, b1, S))
    for B, bid, S in cases:
        out = h.attribute_samples(bid, S)
        h.sync()
        assert_same_keys(out, oracle.attribute_samples(B, S))
    h.close()


@pytest.mark.parametrize("n_ctx", [4097, 20_000, 65_536, 70_000])
def test_two_level_grouping(H, plain, large_bin, n_ctx):
    """More contexts than one partition pass takes: buckets of contexts,
    then each bucket by context (up to 65,536 contexts), else cursors."""
    B1, b1 = plain
    B2, b2 = large_bin
    for B, bid, counts in ((B1, b1, False), (B2, b2, True)):
        S = synth.make_samples(81 + n_ctx % 97, B, 1_300_000, n_ctx, 1.0, counts=counts, device="cuda")
        out = run(H, bid, S)
        assert_same_keys(out, oracle.attribute_samples(B, S))


def test_two_level_in_a_mixed_batch(H, plain, large_bin):
    """A batch whose largest buffer needs two passes, with small and empty
    buffers beside it."""
    B1, b1 = plain
    B2, b2 = large_bin
    spec = [(B2, b2, 900_000, 30_000), (B1, b1, 0, 10), (B1, b1, 5_000, 3), (B2, b2, 250_000, 5_000),
            (B1, b1, 77_777, 65_536)]
    ss = [synth.make_samples(90 + i, B, n, c, 1.0, counts=(i % 2 == 0), device="cuda")
          for i, (B, _, n, c) in enumerate(spec)]
    outs = H.attribute_batch([bid for _, bid, _, _ in spec], ss)
    H.sync()
    for o, S, (B, _, _, _) in zip(outs, ss, spec):
        assert_same_keys(o, oracle.attribute_samples(B, S))


def test_batch_with_many_sub_batches(H, plain):
    """70 buffers of 1.1M contexts each: one sub-batch per buffer, so the
    descriptors of the call need more than the smallest staging area."""
    B, bid = plain
    ss = [synth.make_samples(200 + i, B, 2_000 + 37 * i, 1_100_000, 1.1, counts=(i % 2 == 0), device="cuda")
          for i in range(70)]
    for rep in range(2):                                   # capture, then replay
        outs = H.attribute_batch([bid] * len(ss), ss)
        H.sync()
        for o, S in zip(outs, ss):
            assert_same_keys(o, oracle.attribute_samples(B, S))


@pytest.mark.parametrize("n_ctx,counts", [(300, True), (300, False), (20_000, True)])
@pytest.mark.parametrize("off", [1, 3])
def test_unaligned_sample_arrays(H, plain, n_ctx, counts, off):
    """Sample arrays that do not start on a 16-byte boundary (slices of
    larger tensors): tiles are then loaded by the threads instead of bulk
    copies, with the same result."""
    B, bid = plain
    S = synth.make_samples(91 + off, B, 700_000 + off, n_ctx, 1.1, counts=counts, device="cuda")
    T = synth.Samples(S.pc[off:], S.ctx[off:], S.stall[off:], None if S.count is None else S.count[off:],
                      S.n_ctx, S.n_stall)
    out = run(H, bid, T)
    assert_same_keys(out, oracle.attribute_samples(B, T))


def test_headline_regime_two_level_and_big_groups(H, large_bin):
    """The regime of the large workload: the large binary, more contexts than
    one partition pass takes (4,500: buckets of contexts, then each bucket by
    context), about 10^4 records per context with uint32 counts (so leaves
    hold up to 10,240 records and sort 26-bit keys) and 45 contexts three
    times that size, split into fine bins after the second pass.  Every key
    of a context depends only on that context's samples, so the oracle
    recomputes a subset of contexts (the 45 big ones and 100 others) from
    their samples alone and those keys must match bit for bit; the per-stall
    totals are checked against direct sums of the counts, the UNKNOWN totals
    against the UNKNOWN keys, and the whole key list for canonical order."""
    B, bid = large_bin
    n_ctx = 4500
    wts = np.ones(n_ctx)
    big = synth.np_below(41, 1, np.arange(45), n_ctx).astype(np.int64)
    wts[big] = 3.0
    n = int(10_000 * wts.sum())
    S = synth.make_samples(41, B, n, n_ctx, 0.9, counts=True, device="cuda", ctx_weights=wts)
    out = run(H, bid, S)
    K = out.count()
    kc, kn, ks, kv = out.numpy()
    # canonical order, no zero sums, totals
    key = (kc.astype(np.uint64) << np.uint64(37)) | (kn.astype(np.uint64) << np.uint64(5)) | ks.astype(np.uint64)
    assert K > 0.5 * n and np.all(key[1:] > key[:-1]) and np.all(kv > 0)
    cnt = S.count.cpu().numpy().astype(np.uint64)
    st = S.stall.cpu().numpy()
    total = np.bincount(st, weights=cnt.astype(np.float64), minlength=16).astype(np.uint64)
    assert np.array_equal(out.total[:16].cpu().numpy().view(np.uint64), total)
    assert int(kv.sum(dtype=np.uint64)) == int(cnt.sum(dtype=np.uint64))
    unk = np.bincount(ks[kn == 0xFFFFFFFF], weights=kv[kn == 0xFFFFFFFF].astype(np.float64), minlength=16)
    assert np.array_equal(out.unknown[:16].cpu().numpy().view(np.uint64), unk.astype(np.uint64))
    # the oracle on a subset of contexts
    rest = np.setdiff1d(np.arange(n_ctx), big)
    pick = np.union1d(big, rest[synth.np_below(41, 2, np.arange(100), rest.shape[0]).astype(np.int64)])
    cpu_ctx = S.ctx.cpu().numpy()
    sel = np.isin(cpu_ctx, pick)
    sub = synth.Samples(S.pc.cpu()[sel], S.ctx.cpu()[sel], S.stall.cpu()[sel], S.count.cpu()[sel], n_ctx, 16)
    ref = oracle.attribute_samples(B, sub)
    keep = np.isin(kc, pick)
    assert int(keep.sum()) == len(ref)
    for name, g, r in zip(("ctx", "node", "stall", "val"), (kc[keep], kn[keep], ks[keep], kv[keep]),
                          (ref.ctx, ref.node, ref.stall, ref.val)):
        assert np.array_equal(g, r), f"{name} differs from the oracle"


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two visible GPUs")
def test_two_devices_in_one_process(plain):
    """Handles on two devices of one process: the raised shared-memory
    limits of the aggregation kernels belong to each device, so the second
    device must get them too (a 10,240-record leaf needs about 197 KB)."""
    from paper_2109_06931_gb300 import hpa
    B, _ = plain
    for dev in (0, 1):
        h = hpa.Hpa(dev, leaf_capacity=10240)
        bid = h.load_structure(B)
        S = synth.make_samples(13, B, 400_000, 20, 1.1, counts=True, device=f"cuda:{dev}")
        out = h.attribute_samples(bid, S)
        h.sync()
        assert_same_keys(out, oracle.attribute_samples(B, S))
        h.close()


@pytest.mark.parametrize("n_ctx,counts", [(20_000, True), (300, False), (7, True)])
def test_leaves_writing_their_own_keys(large_bin, plain, n_ctx, counts):
    """leaf_emit = 1: a leaf whose predecessors have published their key
    counts writes its keys straight to the output (look-back over leaves),
    the others go through the separate pass; same keys and totals."""
    from paper_2109_06931_gb300 import hpa
    B, _ = large_bin if n_ctx > 1000 else plain
    h = hpa.Hpa(0, leaf_emit=1)
    bid = h.load_structure(B)
    S = synth.make_samples(61, B, 1_500_000, n_ctx, 0.9, counts=counts, device="cuda")
    out = h.attribute_samples(bid, S)
    h.sync()
    assert_same_keys(out, oracle.attribute_samples(B, S))
    h.close()
