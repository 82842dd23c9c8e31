"""GPU parity of the bottom-up view (Section 7) against the CPU oracle:
every node, level offset and (node, stall) value equal."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0)
    yield h
    h.close()


def dev_cct(cct):
    return (torch.from_numpy(cct[0].view(np.int32)).cuda(), torch.from_numpy(cct[1].view(np.int16)).cuda(),
            torch.from_numpy(cct[2].view(np.int64)).cuda())


def check(out, ref, levels):
    n, v = (int(x) for x in out["counts"].tolist())
    assert n == len(ref.parent) and v == len(ref.val)
    u = lambda t, k, dt: t[:k].cpu().numpy().view(dt)
    assert np.array_equal(u(out["parent"], n, np.uint32), ref.parent)
    assert np.array_equal(u(out["func"], n, np.uint32), ref.func)
    assert np.array_equal(u(out["module"], n, np.uint16), ref.module)
    assert np.array_equal(u(out["offset"], n, np.uint64), ref.offset)
    assert np.array_equal(u(out["level_off"], levels + 2, np.uint64), ref.level_off)
    assert np.array_equal(u(out["val_node"], v, np.uint32), ref.vnode)
    assert np.array_equal(u(out["val_stall"], v, np.uint8), ref.vstall)
    assert np.array_equal(u(out["val"], v, np.uint64), ref.val)


@pytest.mark.parametrize("n_samples,n_ctx,levels,n_sites", [
    (4000, 120, 20, 16), (200_000, 500, 12, 64), (200_000, 500, 0, 0), (1_000_000, 2000, 3, 256), (1, 1, 4, 0)])
def test_bottom_up(H, n_samples, n_ctx, levels, n_sites):
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    S = synth.make_samples(41, B, n_samples, n_ctx, 1.1, counts=True, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    par = synth.make_cct(41, n_ctx, 16, 4)
    mod, off, _ = synth.cct_sites(41, par, n_sites, fan=4)
    out = H.bottom_up(bid, p, dev_cct((par, mod, off)), levels)
    H.sync()
    ref = oracle.bottom_up(B.node_func, oracle.attribute_samples(B, S), (par, mod, off), levels)
    check(out, ref, levels)


def test_more_tree_nodes_than_contexts(H):
    """Launch contexts are the first nodes of a larger tree (ids by level)."""
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    S = synth.make_samples(42, B, 100_000, 300, 1.1, counts=True, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    par = synth.make_cct_levels(42, 5000, 20, 8)
    mod, off, _ = synth.cct_sites(42, par, 40)
    out = H.bottom_up(bid, p, dev_cct((par, mod, off)), 25)
    H.sync()
    check(out, oracle.bottom_up(B.node_func, oracle.attribute_samples(B, S), (par, mod, off), 25), 25)


def test_capacity_reports_sizes(H):
    from paper_2109_06931_gb300 import hpa
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    S = synth.make_samples(43, B, 50_000, 100, 1.1, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    par = synth.make_cct(43, 100, 10, 4)
    mod, off, _ = synth.cct_sites(43, par, 32, fan=4)
    cct = dev_cct((par, mod, off))
    out = H.bottom_up(bid, p, cct, 6, cap_nodes=10, cap_values=10)
    with pytest.raises(hpa.HpaError):
        H.sync()
    ref = oracle.bottom_up(B.node_func, oracle.attribute_samples(B, S), (par, mod, off), 6)
    assert out["counts"].tolist() == [len(ref.parent), len(ref.val)]


def test_parent_after_child_is_refused(H):
    from paper_2109_06931_gb300 import hpa
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    S = synth.make_samples(44, B, 1000, 3, 1.1, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    bad = (np.array([synth.NO_PARENT, 2, 0], np.uint32), np.array([1, 1, 1], np.uint16), np.array([1, 2, 3], np.uint64))
    with pytest.raises(hpa.HpaError):
        H.bottom_up(bid, p, dev_cct(bad), 3)
        H.sync()
