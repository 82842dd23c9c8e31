"""Shared helpers of the GPU parity tests."""
import numpy as np
import torch

import oracle
import synth


def samples_from_numpy(pc, ctx, stall, count, n_ctx, n_stall, device="cuda"):
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(device)
    return synth.Samples(t(np.asarray(pc, np.uint64), np.int64), t(np.asarray(ctx, np.uint32), np.int32),
                         t(np.asarray(stall, np.uint8), np.uint8),
                         None if count is None else t(np.asarray(count, np.uint32), np.int32), n_ctx, n_stall)


def assert_same_keys(prof, ref, check_totals=True):
    """Bit-exact comparison of a device profile with an oracle KeyList."""
    n = prof.count()
    assert n == len(ref), f"key count {n} != oracle {len(ref)}"
    got = prof.numpy()
    names = ("ctx", "node", "stall", "val")
    for name, g, r in zip(names, got, (ref.ctx, ref.node, ref.stall, ref.val)):
        if not np.array_equal(g, r):
            bad = np.nonzero(g != r)[0]
            i = int(bad[0])
            raise AssertionError(f"{name} differs at {len(bad)} keys; first {i}: gpu "
                                 f"({got[0][i]},{got[1][i]},{got[2][i]},{got[3][i]}) oracle "
                                 f"({ref.ctx[i]},{ref.node[i]},{ref.stall[i]},{ref.val[i]})")
    if check_totals and ref.total is not None:
        S = len(ref.total)
        assert np.array_equal(prof.total[:S].cpu().numpy().view(np.uint64), ref.total)
        assert np.array_equal(prof.unknown[:S].cpu().numpy().view(np.uint64), ref.unknown)
