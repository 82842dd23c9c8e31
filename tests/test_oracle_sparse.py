"""Pins of the oracle's sparse layouts (Section 6.2), independent of the
oracle's own code: a hand-computed example and reconstruction of every
input profile from each layout."""
import numpy as np

import oracle
import synth

U = oracle.UNKNOWN


def keys(rows):
    a = np.array(sorted(rows), dtype=np.uint64).reshape(-1, 4)
    return oracle.KeyList(a[:, 0].astype(np.uint32), a[:, 1].astype(np.uint32), a[:, 2].astype(np.uint8),
                          a[:, 3].astype(np.uint64))


P0 = [(0, 3, 0, 5), (0, 3, 2, 1), (1, 7, 0, 4), (2, U, 1, 9)]
P1 = [(0, 3, 2, 6), (1, 2, 1, 2), (1, 7, 0, 8)]


def test_hand_computed_cms(oracle_lib):
    c = oracle.cms([keys(P0), keys(P1)])
    # contexts (ctx, node): (0,3) (1,2) (1,7) (2,U)
    assert c.plane_ctx.tolist() == [0, 1, 1, 2] and c.plane_node.tolist() == [3, 2, 7, U]
    # metrics: (0,3):{0,2} (1,2):{1} (1,7):{0} (2,U):{1}
    assert c.plane_off.tolist() == [0, 2, 3, 4, 5]
    assert c.metric_id.tolist() == [0, 2, 1, 0, 1]
    # (0,3,0):{p0:5} (0,3,2):{p0:1, p1:6} (1,2,1):{p1:2} (1,7,0):{p0:4, p1:8} (2,U,1):{p0:9}
    assert c.metric_off.tolist() == [0, 1, 3, 4, 6, 7]
    assert c.pid.tolist() == [0, 0, 1, 1, 0, 1, 0]
    assert c.val.tolist() == [5, 1, 6, 2, 4, 8, 9]


def test_hand_computed_pms(oracle_lib):
    p = oracle.pms([keys(P0), keys(P1)])
    assert p.prof_off.tolist() == [0, 3, 6]
    assert p.plane_ctx.tolist() == [0, 1, 2, 0, 1, 1] and p.plane_node.tolist() == [3, 7, U, 3, 2, 7]
    assert p.plane_off.tolist() == [0, 2, 3, 4, 5, 6, 7]
    assert p.metric_id.tolist() == [0, 2, 0, 1, 2, 1, 0] and p.val.tolist() == [5, 1, 4, 9, 6, 2, 8]


def _empty():
    z = np.zeros(0, np.uint32)
    return oracle.KeyList(z, z, np.zeros(0, np.uint8), np.zeros(0, np.uint64))


def test_profiles_without_keys(oracle_lib):
    """An empty profile owns no plane (PMS: its offsets repeat) and no entry (CMS)."""
    p = oracle.pms([keys(P0), _empty(), keys(P1), _empty()])
    assert p.prof_off.tolist() == [0, 3, 3, 6, 6]
    assert p.plane_ctx.tolist() == [0, 1, 2, 0, 1, 1] and p.val.tolist() == [5, 1, 4, 9, 6, 2, 8]
    c = oracle.cms([_empty(), keys(P0), keys(P1)])
    assert c.pid.tolist() == [1, 1, 2, 2, 1, 2, 1] and c.val.tolist() == [5, 1, 6, 2, 4, 8, 9]


def _profiles():
    b = synth.PLAIN.binary()
    out = []
    for i, n_ctx in enumerate((30, 30, 5, 30)):
        s = synth.make_samples(40 + i, b, 20_000 + 3000 * i, n_ctx, 1.1, counts=(i % 2 == 0))
        out.append(oracle.attribute_samples(b, s))
    return out


def _rows(k):
    return list(zip(k.ctx.tolist(), k.node.tolist(), k.stall.tolist(), k.val.tolist()))


def test_cms_reconstructs_every_profile(oracle_lib):
    profs = _profiles()
    c = oracle.cms(profs)
    back = [[] for _ in profs]
    for i in range(len(c.plane_ctx)):
        for m in range(int(c.plane_off[i]), int(c.plane_off[i + 1])):
            for j in range(int(c.metric_off[m]), int(c.metric_off[m + 1])):
                back[int(c.pid[j])].append((int(c.plane_ctx[i]), int(c.plane_node[i]), int(c.metric_id[m]), int(c.val[j])))
    for k, b in zip(profs, back):
        assert sorted(b) == _rows(k)
    # sizes: union contexts, union (context, metric) pairs, all values
    ctxs = {(r[0], r[1]) for k in profs for r in _rows(k)}
    pairs = {(r[0], r[1], r[2]) for k in profs for r in _rows(k)}
    assert len(c.plane_ctx) == len(ctxs) and len(c.metric_id) == len(pairs)
    assert len(c.val) == sum(len(k) for k in profs)
    # profiles ascend within each metric entry
    for m in range(len(c.metric_id)):
        seg = c.pid[int(c.metric_off[m]):int(c.metric_off[m + 1])]
        assert np.all(np.diff(seg.astype(np.int64)) > 0)


def test_pms_reconstructs_every_profile(oracle_lib):
    profs = _profiles()
    p = oracle.pms(profs)
    for q, k in enumerate(profs):
        rows = []
        for i in range(int(p.prof_off[q]), int(p.prof_off[q + 1])):
            for j in range(int(p.plane_off[i]), int(p.plane_off[i + 1])):
                rows.append((int(p.plane_ctx[i]), int(p.plane_node[i]), int(p.metric_id[j]), int(p.val[j])))
        assert rows == _rows(k)
