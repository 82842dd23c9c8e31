"""GPU parity of inclusive propagation (Section 6.1): over the structure tree
within each context and over the host calling-context tree; exact integers."""
import numpy as np
import pytest
import torch

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


@pytest.mark.parametrize("frac,counts,n_ctx", [(0.05, False, 500), (0.5, True, 500), (0.3, True, 3)])
def test_structure_inclusive(H, frac, counts, n_ctx):
    import dataclasses
    w = dataclasses.replace(synth.scaled(synth.PLAIN, frac), counts=counts, n_ctx=n_ctx)
    B = w.binary()
    bid = H.load_structure(B)
    S = w.samples(B, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    tree, _ = H.propagate_inclusive(bid, p)
    H.sync()
    ref = oracle.inclusive_structure(B.node_parent, oracle.attribute_samples(B, S))
    assert_same_keys(tree, ref, check_totals=False)


@pytest.mark.parametrize("n_cct,depth,fan", [(500, 32, 8), (20_000, 32, 8), (300_000, 64, 3)])
def test_cct_inclusive(H, n_cct, depth, fan):
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    par = synth.make_cct(3, n_cct, depth, fan)
    n_ctx = min(n_cct, 20_000)
    S = synth.make_samples(8, B, 400_000, n_ctx, 1.1, counts=True, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    _, host = H.propagate_inclusive(bid, p, tree=False,
                                    cct_parent=torch.from_numpy(par.view(np.int32)).cuda())
    H.sync()
    ref = oracle.inclusive_cct(par, 16, oracle.attribute_samples(B, S))
    assert np.array_equal(host.cpu().numpy().view(np.uint64), ref)


def test_cct_cycle_is_reported(H):
    from paper_2109_06931_gb300 import hpa
    B = synth.PLAIN.binary()
    bid = H.load_structure(B)
    par = synth.make_cct(4, 100, 8, 4)
    par[50] = 60
    par[60] = 50          # a cycle (both are non-roots)
    S = synth.make_samples(8, B, 10_000, 100, 1.1, device="cuda")
    p = H.attribute_samples(bid, S)
    H.sync()
    H.propagate_inclusive(bid, p, tree=False, cct_parent=torch.from_numpy(par.view(np.int32)).cuda())
    st, _ = H.sync_status()
    assert st == hpa.HPA_E_INVALID_TABLE
