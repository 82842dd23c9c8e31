"""hpa_attribute_samples_noalloc, the entry point for callers that must not
allocate device memory while they analyse samples (a tool inside the
application it measures, whose caching allocator owns the device memory; a
serving loop where cudaFree would synchronise the whole GPU).  On two calls in
a row it must give exactly what hpa_attribute_samples gives (counts are exact,
so the comparison is bit-exact), and it must refuse a call whose scratch
exceeds its fixed array.  This file is collected last so that a failure here
leaves every other test already run."""
import numpy as np
import pytest

import synth
from gpu_util import assert_same_keys

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_call_twice():
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0)
    B = synth.PLAIN.binary()
    bid = h.load_structure(B)
    for seed, n, n_ctx, counts in ((31, 700_000, 500, False), (32, 400_000, 37, True)):
        S = synth.make_samples(seed, B, n, n_ctx, 1.1, counts=counts, device="cuda")
        ref = h.attribute_samples(bid, S)
        h.sync()
        out = hpa.new_profile(S.n, S.n_stall, h.device)
        out.val.fill_(-1)
        h.attribute_samples_noalloc(bid, S, out)
        h.sync()
        k = ref.count()
        assert out.count() == k
        for a, b in zip(out.numpy(), ref.numpy()):
            assert np.array_equal(a, b)
        assert np.array_equal(out.total.cpu().numpy(), ref.total.cpu().numpy())
        assert np.array_equal(out.unknown.cpu().numpy(), ref.unknown.cpu().numpy())
    h.close()


def test_noalloc_rejects_oversized_calls():
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0)
    B = synth.PLAIN.binary()
    bid = h.load_structure(B)
    S = synth.make_samples(5, B, 3_000_000, 500, 1.1, counts=True, device="cuda")
    out = hpa.new_profile(S.n, S.n_stall, h.device)
    with pytest.raises(hpa.HpaError) as e:
        h.attribute_samples_noalloc(bid, S, out)
    assert e.value.status == hpa.HPA_E_INVALID_ARG and "static scratch" in str(e.value)
    h.close()
