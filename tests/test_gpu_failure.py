"""Failure detection on the GPU without a fault: a bounded device wait on a
flag that nothing sets gives up, reports HPA_E_TIMEOUT through hpa_sync,
and the context keeps working; a flag set before the wait passes at once."""
import time

import pytest
import torch

import oracle
import synth
from gpu_util import assert_same_keys

pytestmark = pytest.mark.gpu


def test_wait_gives_up_and_the_context_stays_usable():
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0, timeout_iters=2000)          # about 2 ms of polls
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t = time.perf_counter()
    h.wait_flag(flag, 1)                        # nothing ever sets it
    with pytest.raises(hpa.HpaError) as e:
        h.sync()
    assert e.value.status == hpa.HPA_E_TIMEOUT
    assert time.perf_counter() - t < 10
    flag.fill_(1)                               # set before the wait is enqueued
    torch.cuda.synchronize()
    h.wait_flag(flag, 1)
    h.sync()
    B = synth.PLAIN.binary()
    bid = h.load_structure(B)
    S = synth.make_samples(5, B, 20_000, 10, 1.1, device="cuda")
    out = h.attribute_samples(bid, S)
    h.sync()
    assert_same_keys(out, oracle.attribute_samples(B, S))
    h.close()
