"""GPU parity of the sparse layouts (Section 6.2): every array of the
context-major and profile-major forms equal to the oracle's."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0)
    yield h
    h.close()


def _same(got, ref, n):
    assert np.array_equal(got[:n].cpu().numpy().astype(np.uint64), np.asarray(ref)[:n].astype(np.uint64))


@pytest.mark.parametrize("which,nprof", [("plain", 4), ("plain", 1), ("large", 3), ("plain", 37)])
def test_sparse_layouts(H, which, nprof):
    w = synth.PLAIN if which == "plain" else synth.LARGE
    B = w.binary()
    bid = H.load_structure(B)
    gpu, ref = [], []
    for i in range(nprof):
        n_ctx = [500, 300, 7][i % 3] if which == "plain" else 2000
        S = synth.make_samples(900 + i, B, 150_000 + 20_000 * (i % 5), n_ctx, 1.0, counts=(i % 2 == 0), device="cuda")
        gpu.append(H.attribute_samples(bid, S))
        ref.append(oracle.attribute_samples(B, S))
    H.sync()
    c = H.build_cms(gpu)
    H.sync()
    rc = oracle.cms(ref)
    npl, nm, nv = (int(x) for x in c["counts"].cpu().tolist())
    assert (npl, nm, nv) == (len(rc.plane_ctx), len(rc.metric_id), len(rc.val))
    u32 = lambda t, n: t[:n].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(u32(c["plane_ctx"], npl), rc.plane_ctx)
    np.testing.assert_array_equal(u32(c["plane_node"], npl), rc.plane_node)
    np.testing.assert_array_equal(u32(c["pid"], nv), rc.pid)
    _same(c["plane_off"], rc.plane_off, npl + 1)
    _same(c["metric_id"], rc.metric_id, nm)
    _same(c["metric_off"], rc.metric_off, nm + 1)
    _same(c["val"], rc.val, nv)
    p = H.build_pms(gpu)
    H.sync()
    rp = oracle.pms(ref)
    npl, nv = (int(x) for x in p["counts"].cpu().tolist())
    assert (npl, nv) == (len(rp.plane_ctx), len(rp.val))
    np.testing.assert_array_equal(p["prof_off"].cpu().numpy().astype(np.uint64), rp.prof_off)
    np.testing.assert_array_equal(p["plane_ctx"][:npl].cpu().numpy().view(np.uint32), rp.plane_ctx)
    np.testing.assert_array_equal(p["plane_node"][:npl].cpu().numpy().view(np.uint32), rp.plane_node)
    _same(p["plane_off"], rp.plane_off, npl + 1)
    _same(p["metric_id"], rp.metric_id, nv)
    _same(p["val"], rp.val, nv)
