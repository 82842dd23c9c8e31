"""Host dump and reload of a profile's sorted keys (a debugging aid), on CPU tensors."""
def test_profile_dump_round_trip(tmp_path):
    """Profile.save / load_profile keep every key, total and the shape."""
    import numpy as np
    import torch
    from paper_2109_06931_gb300 import hpa
    p = hpa.new_profile(8, 3, "cpu")
    k = 5
    p.key_ctx[:k] = torch.tensor([0, 0, 1, 2, 2], dtype=torch.int32)
    p.key_node[:k] = torch.tensor([3, 7, 1, 0, -1], dtype=torch.int32)      # -1: UNKNOWN
    p.key_stall[:k] = torch.tensor([0, 2, 1, 0, 2], dtype=torch.uint8)
    p.val[:k] = torch.tensor([5, 1, 9, 2 ** 40, 4], dtype=torch.int64)
    p.n_keys.fill_(k)
    p.total[:3] = torch.tensor([7, 9, 5], dtype=torch.int64)
    p.unknown[:3] = torch.tensor([0, 0, 4], dtype=torch.int64)
    p.n_ctx, p.n_nodes = 3, 10
    path = str(tmp_path / "prof.npz")
    p.save(path)
    q = hpa.load_profile(path, "cpu")
    for a, b in zip(p.numpy(), q.numpy()):
        assert np.array_equal(a, b)
    assert q.count() == k and (q.n_ctx, q.n_stall, q.n_nodes) == (3, 3, 10)
    assert torch.equal(q.total[:3], p.total[:3]) and torch.equal(q.unknown[:3], p.unknown[:3])
