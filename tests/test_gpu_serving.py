"""Serving (continuous batching with admission by free device memory): every
request's result is the same as the plain call on its samples alone, whatever
mix of requests it was batched with; a request that can never fit is refused."""
import random

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def host_samples(S):
    pin = lambda t: None if t is None else t.cpu().pin_memory()
    return pin(S.pc), pin(S.ctx), pin(S.stall), pin(S.count)


@pytest.mark.parametrize("mem_cap,max_batch,max_inflight", [(0, 0, 0), (64 << 20, 8, 0), (0, 1, 6)])
def test_mixed_requests_equal_alone(mem_cap, max_batch, max_inflight):
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0)
    B1, B2 = synth.PLAIN.binary(), synth.make_binary(77, 300, 300 * 13_422, 15_000, 900, n_scc=3)
    b1, b2 = h.load_structure(B1), h.load_structure(B2)
    rng = random.Random(5)
    reqs = []
    for i in range(40):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(3e5))))
        B, bid = (B1, b1) if i % 3 else (B2, b2)
        S = synth.make_samples(900 + i, B, n, 1 + (i * 37) % 600, 1.0, counts=(i % 2 == 0))
        reqs.append((bid, S))
    # alone: the plain call on the device
    alone, totals = [], []
    for bid, S in reqs:
        p = h.attribute_samples(bid, S.to("cuda"))
        h.sync()
        alone.append(p.numpy())
        totals.append((p.total[: S.n_stall].cpu().numpy().view(np.uint64).copy(),
                       p.unknown[: S.n_stall].cpu().numpy().view(np.uint64).copy()))
    srv = hpa.Server(h, mem_cap_bytes=mem_cap, max_batch=max_batch, max_inflight=max_inflight)
    tickets = []
    for i, (bid, S) in enumerate(reqs):
        pc, ctx, st, cnt = host_samples(S)
        out = None
        if i % 2:       # pageable result arrays for half of the requests
            cap = max(1, S.n)
            out = dict(ctx=torch.empty(cap, dtype=torch.int32), node=torch.empty(cap, dtype=torch.int32),
                       stall=torch.empty(cap, dtype=torch.uint8), val=torch.empty(cap, dtype=torch.int64),
                       n=torch.zeros(1, dtype=torch.int64), total=torch.zeros(32, dtype=torch.int64),
                       unknown=torch.zeros(32, dtype=torch.int64))
        tickets.append(srv.submit(bid, pc, ctx, st, cnt, S.n_ctx, S.n_stall, out=out))
    for (t, ref), (tot, unk), (bid, S) in zip(zip(tickets, alone), totals, reqs):
        while (st := srv.poll(t, 1000)) == hpa.HPA_PENDING:
            pass
        assert st == hpa.HPA_OK
        out = srv.result(t)
        k = int(out["n"][0])
        assert k == len(ref[0])
        assert np.array_equal(out["ctx"][:k].numpy().view(np.uint32), ref[0])
        assert np.array_equal(out["node"][:k].numpy().view(np.uint32), ref[1])
        assert np.array_equal(out["stall"][:k].numpy(), ref[2])
        assert np.array_equal(out["val"][:k].numpy().view(np.uint64), ref[3])
        assert np.array_equal(out["total"][: S.n_stall].numpy().view(np.uint64), tot)
        assert np.array_equal(out["unknown"][: S.n_stall].numpy().view(np.uint64), unk)
    stats = srv.stats()
    assert stats["compute_ms"] > 0 and stats["h2d_ms"] >= 0 and stats["d2h_ms"] >= 0
    assert stats["completed"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    if max_batch:
        assert stats["batches"] >= len(reqs) / max_batch
    srv.close()
    h.close()


def test_request_larger_than_pool_is_refused():
    from paper_2109_06931_gb300 import hpa
    h = hpa.Hpa(0)
    B = synth.PLAIN.binary()
    bid = h.load_structure(B)
    srv = hpa.Server(h, mem_cap_bytes=1 << 20)
    S = synth.make_samples(3, B, 200_000, 10, 1.0)
    t = srv.submit(bid, *host_samples(S), S.n_ctx, S.n_stall)
    st = srv.poll(t, 5000)
    assert st == hpa.HPA_E_OOM
    srv.close()
    h.close()
