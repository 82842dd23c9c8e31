"""GPU parity of call-path profile unification (Section 6.1): merged ids,
parents and call sites equal to the oracle's."""
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


def dev(c):
    return (torch.from_numpy(c[0].view(np.int32)).cuda(), torch.from_numpy(c[1].view(np.int16)).cuda(),
            torch.from_numpy(c[2].view(np.int64)).cuda())


@pytest.mark.parametrize("n_master,depth,P,keep", [(5000, 16, 3, 0.3), (200_000, 64, 8, 0.1), (1, 4, 1, 1.0),
                                                    (50_000, 40, 32, 0.02)])
def test_unify(H, n_master, depth, P, keep):
    ccts = synth.make_profile_ccts(17, n_master, depth, P, keep)
    out = H.unify_ccts([dev(c) for c in ccts])
    H.sync()
    uid, up, um, uo = oracle.unify(ccts)
    n = int(out["n"].item())
    assert n == len(up)
    assert np.array_equal(out["uid"].cpu().numpy().view(np.uint32), uid)
    assert np.array_equal(out["parent"][:n].cpu().numpy().view(np.uint32), up)
    assert np.array_equal(out["module"][:n].cpu().numpy().view(np.uint16), um)
    assert np.array_equal(out["offset"][:n].cpu().numpy().view(np.uint64), uo)


def test_parent_after_child_is_refused(H):
    from paper_2109_06931_gb300 import hpa
    bad = (np.array([synth.NO_PARENT, 2, 0], np.uint32), np.array([1, 1, 1], np.uint16), np.array([1, 2, 3], np.uint64))
    H.unify_ccts([dev(bad)])
    with pytest.raises(hpa.HpaError):
        H.sync()
