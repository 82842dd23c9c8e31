"""GPU parity of the flat view and of the GPU calling context tree of all
contexts pooled (Sections 6.3, 7) against the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_keys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0)
    yield h
    h.close()


@pytest.mark.parametrize("which", ["plain", "large"])
def test_flat_profile(H, which):
    w = synth.PLAIN if which == "plain" else synth.LARGE
    B = w.binary()
    bid = H.load_structure(B)
    S = w.samples(B, device="cuda", n=min(w.n_samples, 2_000_000))
    p = H.attribute_samples(bid, S)
    H.sync()
    f = H.flat_profile(bid, p)
    H.sync()
    ref = oracle.flat(S.n_stall, oracle.attribute_samples(B, S))
    assert_same_keys(f, ref)


def test_flat_capacity_reports_size(H):
    from paper_2109_06931_gb300 import hpa
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    S = synth.make_samples(3, B, 100_000, 30, 1.1, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    f = H.flat_profile(bid, p, capacity=10)
    with pytest.raises(hpa.HpaError):
        H.sync()
    assert f.count() == len(oracle.flat(16, oracle.attribute_samples(B, S)))


def test_global_gpu_cct_is_apportioning_of_the_flat_profile(H):
    """Apportioning the flat profile (context 0) gives the GPU CCT of all
    contexts pooled; it matches the oracle's apportioning of its flat view."""
    from test_gpu_gpucct import check
    w = synth.PLAIN
    B = w.binary()
    bid = H.load_structure(B)
    S = w.samples(B, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    f = H.flat_profile(bid, p)
    H.sync()
    res = H.apportion_callgraph(bid, f, [0])
    H.sync()
    ref = oracle.apportion(B, 16, oracle.flat(16, oracle.attribute_samples(B, S)), np.array([0], np.uint32))
    check(res, ref)


@pytest.mark.parametrize("which,ctxs,budget", [("plain", [0, 7, 499], 1 << 20), ("large", [3, 12_345], 1 << 20),
                                               ("plain", [5], 300)])
def test_expanded_gpu_cct(H, which, ctxs, budget):
    """Context q's GPU CCT as a tree: the same nodes, parents and call sites
    as the oracle's expansion of its own apportioning, scales and inclusive
    costs within 1e-5."""
    w = synth.PLAIN if which == "plain" else synth.LARGE
    B = w.binary()
    bid = H.load_structure(B)
    S = w.samples(B, device="cuda", n=min(w.n_samples, 3_000_000))
    p = H.attribute_samples(bid, S)
    H.sync()
    res = H.apportion_callgraph(bid, p, ctxs)
    H.sync()
    g = oracle.apportion(B, 16, oracle.attribute_samples(B, S), np.array(ctxs, np.uint32))
    for q in range(len(ctxs)):
        t = H.expand_gpucct(bid, res, ctxs, 16, q, budget)
        H.sync()
        ref = oracle.expand(B, g, q, budget)
        n = int(t["n"].item())
        assert n == len(ref.cnode) and bool(t["truncated"].item()) == ref.truncated
        assert np.array_equal(t["cnode"][:n].cpu().numpy().view(np.uint32), ref.cnode)
        assert np.array_equal(t["parent"][:n].cpu().numpy().view(np.uint32), ref.parent)
        assert np.array_equal(t["edge"][:n].cpu().numpy().view(np.uint32), ref.edge)
        np.testing.assert_allclose(t["scale"][:n].cpu().numpy(), ref.scale, rtol=1e-5, atol=1e-30)
        got = t["incl"][:n].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ref.incl) <= 1e-5 * np.abs(ref.incl) + 1e-30)
