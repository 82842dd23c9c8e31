"""GPU parity of derived metrics across profiles (Section 4.5) and the warp
issue rate (Section 7): sums, min and max exact; mean / std / CoV / W /
stall shares in FP32 within 1e-5 of the FP64 oracle; NaN where S = 0."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def H():
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0, issued_mask=0b11)
    yield h
    h.close()


def close(got, exp):
    got = np.asarray(got, np.float64)
    nan = np.isnan(exp)
    assert np.array_equal(np.isnan(got), nan)
    e, g = exp[~nan], got[~nan]
    zero = e == 0
    assert (g[zero] == 0).all()
    if (~zero).any():
        assert (np.abs(g[~zero] - e[~zero]) / np.abs(e[~zero])).max() <= RTOL


@pytest.mark.parametrize("P,n,n_ctx", [(1, 50_000, 40), (4, 200_000, 500), (16, 30_000, 3)])
def test_derive(H, P, n, n_ctx):
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    profs, refs = [], []
    for p in range(P):
        S = synth.make_samples(1000 + p, B, n, n_ctx, 1.1, counts=(p % 2 == 1), device="cuda")
        profs.append(H.attribute_samples(bid, S))
        refs.append(oracle.attribute_samples(B, S))
    H.sync()
    out = H.derive_metrics(profs, n_ctx=n_ctx + 2)
    H.sync()
    ref = oracle.derive(refs, n_ctx + 2, 16, issued_mask=0b11)
    k = int(out["n"].item())
    assert k == len(ref.sum)
    v = lambda t: t[:k].cpu().numpy()
    assert np.array_equal(v(out["ctx"]).view(np.uint32), ref.ctx)
    assert np.array_equal(v(out["node"]).view(np.uint32), ref.node)
    assert np.array_equal(v(out["stall"]), ref.stall)
    assert np.array_equal(v(out["sum"]).view(np.uint64), ref.sum)
    assert np.array_equal(v(out["min"]).view(np.uint64).astype(np.float64), ref.min)
    assert np.array_equal(v(out["max"]).view(np.uint64).astype(np.float64), ref.max)
    for name in ("mean", "std", "cov"):
        close(v(out[name]), getattr(ref, name))
    assert np.array_equal(out["S"].cpu().numpy().view(np.uint64), ref.S)
    assert np.array_equal(out["S_issued"].cpu().numpy().view(np.uint64), ref.S_issued)
    close(out["W"].cpu().numpy(), ref.W)
    close(out["frac"].cpu().numpy(), ref.frac)


def test_derive_hot_keys_many_profiles(H):
    """Many profiles of one context sampling the same function: an oversized
    sub-bin, handled by dense per-key accumulator windows."""
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    f = 5
    slots = int((B.func_hi[f] - B.func_lo[f]) // 16)
    from gpu_util import samples_from_numpy
    profs, refs = [], []
    for p in range(48):
        idx = np.arange(3000)
        pc = B.func_lo[f] + (synth.np_below(p, 1, idx, slots) * 16).astype(np.uint64)
        st = synth.np_below(p, 2, idx, 16).astype(np.uint8)
        cnt = (1 + synth.np_below(p, 3, idx, 1 << 20)).astype(np.uint32)
        S = samples_from_numpy(pc, np.zeros(3000, np.uint32), st, cnt, 1, 16)
        profs.append(H.attribute_samples(bid, S))
        refs.append(oracle.attribute_samples(B, S))
    H.sync()
    out = H.derive_metrics(profs)
    H.sync()
    ref = oracle.derive(refs, 1, 16, issued_mask=0b11)
    k = int(out["n"].item())
    assert k == len(ref.sum)
    assert np.array_equal(out["sum"][:k].cpu().numpy().view(np.uint64), ref.sum)
    close(out["std"][:k].cpu().numpy(), ref.std)
    close(out["cov"][:k].cpu().numpy(), ref.cov)


@pytest.mark.parametrize("wl,n,n_ctx", [("plain", 300_000, 500), ("large", 2_000_000, 20_000)])
def test_issue_by_function(H, wl, n, n_ctx):
    """Warp issue rate and stall shares per (context, function) (Section 7)
    against the oracle: rows, S and S_issued exact, W and shares within 1e-5;
    a too-small capacity reports the rows needed."""
    from paper_2109_06931_gb300 import hpa
    w = synth.PLAIN if wl == "plain" else synth.LARGE
    B = w.binary()
    bid = H.load_structure(B)
    S = synth.make_samples(77, B, n, n_ctx, w.zipf_s, counts=True, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    r = H.issue_by_function(bid, p)
    H.sync()
    ref = oracle.issue_by_function(B.node_func, 16, oracle.attribute_samples(B, S), 0b11)
    k = int(r["n_rows"].item())
    assert k == len(ref.S)
    assert np.array_equal(r["ctx"][:k].cpu().numpy().view(np.uint32), ref.ctx)
    assert np.array_equal(r["func"][:k].cpu().numpy().view(np.uint32), ref.func)
    assert np.array_equal(r["S"][:k].cpu().numpy().view(np.uint64), ref.S)
    assert np.array_equal(r["S_issued"][:k].cpu().numpy().view(np.uint64), ref.S_issued)
    close(r["W"][:k].cpu().numpy(), ref.W)
    close(r["frac"][:k].cpu().numpy().ravel(), ref.frac.ravel())
    H.issue_by_function(bid, p, capacity=k - 1)
    st, _ = H.sync_status()
    assert st == hpa.HPA_E_CAPACITY


def _gpu_profile(rows, n_ctx, n_stall, n_nodes):
    """A device profile holding the given (ctx, node, stall, value) keys, sorted."""
    import torch
    from paper_2109_06931_gb300 import hpa
    a = np.array(sorted(rows), dtype=np.uint64).reshape(-1, 4)
    k = a.shape[0]
    t = lambda x, dt: torch.as_tensor(np.ascontiguousarray(x.astype(dt)).view(
        {np.uint32: np.int32, np.uint64: np.int64, np.uint8: np.uint8}[dt]), device="cuda")
    return hpa.Profile(t(a[:, 0], np.uint32), t(a[:, 1], np.uint32), t(a[:, 2], np.uint8), t(a[:, 3], np.uint64),
                       torch.tensor([k], dtype=torch.int64, device="cuda"),
                       torch.zeros(n_stall, dtype=torch.int64, device="cuda"),
                       torch.zeros(n_stall, dtype=torch.int64, device="cuda"), n_ctx, n_stall, max(k, 1), n_nodes)


def _check_ratio(r, ref):
    k = int(r["n"].item())
    assert k == len(ref.num)
    assert np.array_equal(r["ctx"][:k].cpu().numpy().view(np.uint32), ref.ctx)
    assert np.array_equal(r["node"][:k].cpu().numpy().view(np.uint32), ref.node)
    assert np.array_equal(r["stall"][:k].cpu().numpy(), ref.stall)
    assert np.array_equal(r["num"][:k].cpu().numpy().view(np.uint64), ref.num)
    assert np.array_equal(r["den"][:k].cpu().numpy().view(np.uint64), ref.den)
    # FP64 quotient rounded once to FP32 on both sides: equal bit for bit
    got = r["ratio"][:k].cpu().numpy()
    exp = ref.ratio.astype(np.float32)
    assert np.array_equal(np.isnan(got), np.isnan(exp))
    assert np.array_equal(got[~np.isnan(got)], exp[~np.isnan(exp)])
    return k


def test_ratio_hand_example(H):
    """Registers per invocation from registers summed over invocations and the
    invocation counts of two ranks (Section 4.5), hand-computed: 96 / 3 = 32,
    200 / 5 = 40, NaN without a count, 0 without registers, UNKNOWN 9 / 3."""
    import test_oracle_ratio as TR
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    M = int(B.node_func.shape[0])
    num = [_gpu_profile(p, 5, 2, M) for p in TR.NUM]
    den = [_gpu_profile(p, 5, 2, M) for p in TR.DEN]
    r = H.ratio_of_sums(bid, num, den)
    H.sync()
    k = int(r["n"].item())
    assert k == 5
    assert r["ctx"][:k].tolist() == [0, 1, 2, 3, 4]
    assert r["node"][:k].cpu().numpy().view(np.uint32).tolist() == [3, 3, 5, 1, 0xFFFFFFFF]
    assert r["num"][:k].tolist() == [96, 200, 7, 0, 9] and r["den"][:k].tolist() == [3, 5, 0, 4, 3]
    q = r["ratio"][:k].cpu().numpy()
    assert q[0] == 32.0 and q[1] == 40.0 and np.isnan(q[2]) and q[3] == 0.0 and q[4] == 3.0
    ref = oracle.ratio([TR._keys(oracle, p) for p in TR.NUM], [TR._keys(oracle, p) for p in TR.DEN])
    _check_ratio(r, ref)


@pytest.mark.parametrize("wl,P_num,P_den,n,n_ctx", [("plain", 1, 1, 200_000, 300), ("plain", 3, 2, 100_000, 40),
                                                    ("plain", 2, 0, 50_000, 7), ("large", 2, 2, 1_000_000, 20_000)])
def test_ratio_of_sums(H, wl, P_num, P_den, n, n_ctx):
    """Ratio of two raw metrics per key against the oracle: keys, both sums
    exact, the FP32 ratio equal; a too-small capacity reports the rows needed."""
    from paper_2109_06931_gb300 import hpa
    w = synth.PLAIN if wl == "plain" else synth.LARGE
    B = w.binary()
    bid = H.load_structure(B)
    gp, cp = [], []
    for p in range(P_num + P_den):
        S = synth.make_samples(500 + p, B, n // (1 + p % 3), n_ctx, w.zipf_s, counts=(p % 2 == 0), device="cuda")
        gp.append(H.attribute_samples(bid, S))
        cp.append(oracle.attribute_samples(B, S))
    H.sync()
    r = H.ratio_of_sums(bid, gp[:P_num], gp[P_num:])
    H.sync()
    ref = oracle.ratio(cp[:P_num], cp[P_num:])
    k = _check_ratio(r, ref)
    H.ratio_of_sums(bid, gp[:P_num], gp[P_num:], capacity=k - 1)
    st, _ = H.sync_status()
    assert st == hpa.HPA_E_CAPACITY
