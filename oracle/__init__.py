"""ctypes wrapper of the CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The CUDA library never imports or links it.

`build()` compiles oracle.cpp with g++ into oracle/_build/liboracle.so.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "_build", "liboracle.so")
UNKNOWN = 0xFFFFFFFF

_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "oracle.cpp")
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(LIB)
    return _lib


def load(path: str):
    """Load and type an oracle library built from oracle.cpp at `path`."""
    L = C.CDLL(path)
    vp, u64, u32, i32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int
    L.orc_attribute.restype = vp
    L.orc_attribute.argtypes = [u64, vp, vp, vp, u64, vp, vp, vp, vp, u32, u32]
    L.orc_inclusive_structure.restype = vp
    L.orc_inclusive_structure.argtypes = [u32, vp, u64, vp, vp, vp, vp]
    L.orc_expand.restype = vp
    L.orc_expand.argtypes = [u32, u32, u32, vp, vp, vp, u32, vp, vp, u32]
    L.orc_expand_size.restype = u64; L.orc_expand_size.argtypes = [vp]
    L.orc_expand_truncated.restype = i32; L.orc_expand_truncated.argtypes = [vp]
    L.orc_expand_fetch.argtypes = [vp] * 6
    L.orc_expand_free.argtypes = [vp]
    L.orc_unify.restype = vp
    L.orc_unify.argtypes = [u32, vp, vp, vp, vp]
    L.orc_unify_size.restype = u64; L.orc_unify_size.argtypes = [vp]
    L.orc_unify_status.restype = i32; L.orc_unify_status.argtypes = [vp]
    L.orc_unify_fetch.argtypes = [vp] * 5
    L.orc_unify_free.argtypes = [vp]
    L.orc_bottom_up.restype = vp
    L.orc_bottom_up.argtypes = [u64, vp, vp, vp, vp, u32, vp, u32, vp, vp, vp, u32]
    L.orc_bu_status.restype = i32; L.orc_bu_status.argtypes = [vp]
    L.orc_bu_sizes.argtypes = [vp, vp]
    L.orc_bu_fetch.argtypes = [vp] * 9
    L.orc_bu_free.argtypes = [vp]
    L.orc_cms.restype = vp
    L.orc_cms.argtypes = [u64, vp, vp, vp, vp, vp]
    L.orc_pms.restype = vp
    L.orc_pms.argtypes = [u32, u64, vp, vp, vp, vp, vp]
    L.orc_sparse_sizes.argtypes = [vp, vp]
    L.orc_sparse_fetch.argtypes = [vp] * 9
    L.orc_sparse_free.argtypes = [vp]
    L.orc_flat.restype = vp
    L.orc_flat.argtypes = [u32, u64, vp, vp, vp]
    L.orc_inclusive_cct.restype = i32
    L.orc_inclusive_cct.argtypes = [u32, vp, u32, u64, vp, vp, vp, vp]
    L.orc_derive.restype = vp
    L.orc_derive.argtypes = [u32, vp, vp, vp, vp, vp, u32, u32, u32]
    L.orc_issue_by_function.restype = vp
    L.orc_issue_by_function.argtypes = [u32, vp, u32, u32, u64, vp, vp, vp, vp]
    L.orc_ratio.restype = vp
    L.orc_ratio.argtypes = [u32, u32, vp, vp, vp, vp, vp]
    L.orc_ratio_size.restype = u64; L.orc_ratio_size.argtypes = [vp]
    L.orc_ratio_fetch.argtypes = [vp] * 7
    L.orc_ratio_free.argtypes = [vp]
    L.orc_issue_status.restype = i32; L.orc_issue_status.argtypes = [vp]
    L.orc_issue_size.restype = u64; L.orc_issue_size.argtypes = [vp]
    L.orc_issue_fetch.argtypes = [vp] * 7
    L.orc_issue_free.argtypes = [vp]
    L.orc_apportion.restype = vp
    L.orc_apportion.argtypes = [u32, vp, u32, u32, vp, vp, vp, u32, u64, vp, vp, vp, vp, u32, vp]
    for name in ("orc_status", "orc_apportion_status"):
        getattr(L, name).restype = i32; getattr(L, name).argtypes = [vp]
    for name in ("orc_bad", "orc_size", "orc_derive_size"):
        getattr(L, name).restype = u64; getattr(L, name).argtypes = [vp]
    L.orc_apportion_V.restype = u32; L.orc_apportion_V.argtypes = [vp]
    L.orc_fetch.argtypes = [vp] * 7
    L.orc_derive_fetch.argtypes = [vp] * 14
    L.orc_apportion_fetch.argtypes = [vp] * 5
    for name in ("orc_free", "orc_derive_free", "orc_apportion_free"):
        getattr(L, name).argtypes = [vp]
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


@dataclass
class KeyList:
    """Sorted (ctx, node, stall) -> value list."""
    ctx: np.ndarray
    node: np.ndarray
    stall: np.ndarray
    val: np.ndarray
    total: np.ndarray | None = None
    unknown: np.ndarray | None = None
    status: int = 0
    bad: int = 0

    def __len__(self):
        return int(self.val.shape[0])


def _take(L, h, n_stall, with_totals):
    st, bad, n = L.orc_status(h), L.orc_bad(h), L.orc_size(h)
    ctx = np.empty(n, np.uint32); node = np.empty(n, np.uint32)
    stall = np.empty(n, np.uint8); val = np.empty(n, np.uint64)
    tot = np.zeros(n_stall, np.uint64) if with_totals else None
    unk = np.zeros(n_stall, np.uint64) if with_totals else None
    L.orc_fetch(h, _p(ctx), _p(node), _p(stall), _p(val), _p(tot), _p(unk))
    L.orc_free(h)
    return KeyList(ctx, node, stall, val, tot, unk, st, bad)


def attribute(binary, pc, ctx, stall, count, n_ctx: int, n_stall: int) -> KeyList:
    """Attribution + raw-metric aggregation (Sections 4.2, 4.5, 5)."""
    L = lib()
    lo, hi, nd = _c(binary.range_lo, np.uint64), _c(binary.range_hi, np.uint64), _c(binary.range_node, np.uint32)
    pc = _c(np.asarray(pc).view(np.uint64) if np.asarray(pc).dtype == np.int64 else pc, np.uint64)
    ctx = _c(np.asarray(ctx).view(np.uint32) if np.asarray(ctx).dtype == np.int32 else ctx, np.uint32)
    stall = _c(stall, np.uint8)
    if count is not None:
        count = _c(np.asarray(count).view(np.uint32) if np.asarray(count).dtype == np.int32 else count, np.uint32)
    h = L.orc_attribute(lo.shape[0], _p(lo), _p(hi), _p(nd), pc.shape[0], _p(pc), _p(ctx),
                        _p(stall), _p(count), n_ctx, n_stall)
    return _take(L, h, n_stall, True)


def attribute_samples(binary, s) -> KeyList:
    """attribute() on a synth.Samples (moved to host)."""
    return attribute(binary, s.pc.cpu().numpy(), s.ctx.cpu().numpy(), s.stall.cpu().numpy(),
                     None if s.count is None else s.count.cpu().numpy(), s.n_ctx, s.n_stall)


def inclusive_structure(node_parent, keys: KeyList) -> KeyList:
    """Inclusive metrics over the structure tree within each context (Section 6.1)."""
    L = lib()
    par = _c(node_parent, np.uint32)
    k = [_c(keys.ctx, np.uint32), _c(keys.node, np.uint32), _c(keys.stall, np.uint8), _c(keys.val, np.uint64)]
    h = L.orc_inclusive_structure(par.shape[0], _p(par), k[0].shape[0], *[_p(x) for x in k])
    return _take(L, h, 0, False)


def flat(n_stall: int, keys: KeyList) -> KeyList:
    """Flat view (Section 7): values summed over contexts per (node, stall)."""
    L = lib()
    k = [_c(keys.node, np.uint32), _c(keys.stall, np.uint8), _c(keys.val, np.uint64)]
    h = L.orc_flat(n_stall, k[0].shape[0], *[_p(x) for x in k])
    return _take(L, h, n_stall, True)


def inclusive_cct(cct_parent, n_stall: int, keys: KeyList) -> np.ndarray:
    """Inclusive per-stall totals over the host calling-context tree (Section 6.1)."""
    L = lib()
    par = _c(cct_parent, np.uint32)
    out = np.zeros((par.shape[0], n_stall), np.uint64)
    k = [_c(keys.ctx, np.uint32), _c(keys.stall, np.uint8), _c(keys.val, np.uint64)]
    st = L.orc_inclusive_cct(par.shape[0], _p(par), n_stall, k[0].shape[0], *[_p(x) for x in k], _p(out))
    if st:
        raise ValueError(f"oracle inclusive_cct status {st}")
    return out


@dataclass
class Derived:
    ctx: np.ndarray
    node: np.ndarray
    stall: np.ndarray
    sum: np.ndarray
    min: np.ndarray
    max: np.ndarray
    mean: np.ndarray
    std: np.ndarray
    cov: np.ndarray
    S: np.ndarray
    S_issued: np.ndarray
    W: np.ndarray
    frac: np.ndarray


def derive(profiles, n_ctx: int, n_stall: int, issued_mask: int = 1) -> Derived:
    """Cross-profile statistics (Section 4.5) and warp issue rate (Section 7)."""
    L = lib()
    P = len(profiles)
    ks = [[_c(p.ctx, np.uint32), _c(p.node, np.uint32), _c(p.stall, np.uint8), _c(p.val, np.uint64)] for p in profiles]
    nk = np.array([k[0].shape[0] for k in ks], np.uint64)
    ptrs = [np.array([k[j].ctypes.data for k in ks], np.uint64) for j in range(4)]
    h = L.orc_derive(P, _p(nk), *[_p(x) for x in ptrs], n_ctx, n_stall, issued_mask)
    n = L.orc_derive_size(h)
    d = Derived(np.empty(n, np.uint32), np.empty(n, np.uint32), np.empty(n, np.uint8), np.empty(n, np.uint64),
                *[np.empty(n, np.float64) for _ in range(5)],
                np.empty(n_ctx, np.uint64), np.empty(n_ctx, np.uint64), np.empty(n_ctx, np.float64),
                np.empty((n_ctx, n_stall), np.float64))
    L.orc_derive_fetch(h, _p(d.ctx), _p(d.node), _p(d.stall), _p(d.sum), _p(d.min), _p(d.max), _p(d.mean),
                       _p(d.std), _p(d.cov), _p(d.S), _p(d.S_issued), _p(d.W), _p(d.frac))
    L.orc_derive_free(h)
    del ks
    return d


@dataclass
class IssueRows:
    ctx: np.ndarray        # uint32[n]
    func: np.ndarray       # uint32[n]
    S: np.ndarray          # uint64[n]
    S_issued: np.ndarray   # uint64[n]
    W: np.ndarray          # float64[n]
    frac: np.ndarray       # float64[n, n_stall]
    status: int = 0


def issue_by_function(node_func, n_stall: int, keys: KeyList, issued_mask: int = 1) -> IssueRows:
    """Warp issue rate and stall shares per (context, function) (Section 7)."""
    L = lib()
    nf = _c(node_func, np.uint32)
    k = [_c(keys.ctx, np.uint32), _c(keys.node, np.uint32), _c(keys.stall, np.uint8), _c(keys.val, np.uint64)]
    h = L.orc_issue_by_function(nf.shape[0], _p(nf), n_stall, issued_mask, k[0].shape[0], *[_p(x) for x in k])
    st = L.orc_issue_status(h)
    n = L.orc_issue_size(h)
    r = IssueRows(np.empty(n, np.uint32), np.empty(n, np.uint32), np.empty(n, np.uint64), np.empty(n, np.uint64),
                  np.empty(n, np.float64), np.empty((n, n_stall), np.float64), st)
    L.orc_issue_fetch(h, _p(r.ctx), _p(r.func), _p(r.S), _p(r.S_issued), _p(r.W), _p(r.frac))
    L.orc_issue_free(h)
    return r


@dataclass
class RatioRows:
    ctx: np.ndarray        # uint32[n]
    node: np.ndarray       # uint32[n]
    stall: np.ndarray      # uint8[n]
    num: np.ndarray        # uint64[n]
    den: np.ndarray        # uint64[n]
    ratio: np.ndarray      # float64[n] (NaN where den = 0)


def ratio(num_profiles, den_profiles) -> RatioRows:
    """Ratio of two raw metrics, each summed over its group of profiles (Section 4.5)."""
    L = lib()
    profiles = list(num_profiles) + list(den_profiles)
    ks = [[_c(p.ctx, np.uint32), _c(p.node, np.uint32), _c(p.stall, np.uint8), _c(p.val, np.uint64)] for p in profiles]
    nk = np.array([k[0].shape[0] for k in ks] or [0], np.uint64)
    ptrs = [np.array([k[j].ctypes.data for k in ks] or [0], np.uint64) for j in range(4)]
    h = L.orc_ratio(len(num_profiles), len(den_profiles), _p(nk), *[_p(x) for x in ptrs])
    n = L.orc_ratio_size(h)
    r = RatioRows(np.empty(n, np.uint32), np.empty(n, np.uint32), np.empty(n, np.uint8), np.empty(n, np.uint64),
                  np.empty(n, np.uint64), np.empty(n, np.float64))
    L.orc_ratio_fetch(h, _p(r.ctx), _p(r.node), _p(r.stall), _p(r.num), _p(r.den), _p(r.ratio))
    L.orc_ratio_free(h)
    del ks
    return r


@dataclass
class GpuCct:
    V: int
    cnode_of_func: np.ndarray    # uint32[F]
    incl: np.ndarray             # float64[n_req, V, n_stall + 1]
    a: np.ndarray                # float64[n_req, E, n_stall + 1]
    flags: np.ndarray            # uint8[n_req, E]


def apportion(binary, n_stall: int, keys: KeyList, req_ctx) -> GpuCct:
    """Approximate GPU calling context tree, Section 6.3 steps 1-4."""
    L = lib()
    nf = _c(binary.node_func, np.uint32)
    cc, ce, cn = _c(binary.cs_caller, np.uint32), _c(binary.cs_callee, np.uint32), _c(binary.cs_node, np.uint32)
    k = [_c(keys.ctx, np.uint32), _c(keys.node, np.uint32), _c(keys.stall, np.uint8), _c(keys.val, np.uint64)]
    rq = _c(req_ctx, np.uint32)
    F, E = int(binary.n_funcs), int(cc.shape[0])
    h = L.orc_apportion(nf.shape[0], _p(nf), F, E, _p(cc), _p(ce), _p(cn), n_stall,
                        k[0].shape[0], *[_p(x) for x in k], rq.shape[0], _p(rq))
    st = L.orc_apportion_status(h)
    if st:
        L.orc_apportion_free(h)
        raise ValueError(f"oracle apportion status {st}")
    V = L.orc_apportion_V(h)
    M = n_stall + 1
    g = GpuCct(V, np.empty(F, np.uint32), np.empty((rq.shape[0], V, M)), np.empty((rq.shape[0], E, M)),
               np.empty((rq.shape[0], E), np.uint8))
    L.orc_apportion_fetch(h, _p(g.cnode_of_func), _p(g.incl), _p(g.a), _p(g.flags))
    L.orc_apportion_free(h)
    return g


@dataclass
class Tree:
    parent: np.ndarray
    cnode: np.ndarray
    edge: np.ndarray
    scale: np.ndarray
    incl: np.ndarray        # [n, n_stall + 1]
    truncated: bool


def expand(binary, g: "GpuCct", q: int, budget: int) -> Tree:
    """Context q of an apportioning result as a tree (Section 6.3, step 4)."""
    L = lib()
    cof = _c(g.cnode_of_func, np.uint32)
    cc, ce = _c(binary.cs_caller, np.uint32), _c(binary.cs_callee, np.uint32)
    inc, a = _c(g.incl[q], np.float64), _c(g.a[q], np.float64)
    M = int(inc.shape[1])
    h = L.orc_expand(int(binary.n_funcs), int(g.V), int(cc.shape[0]), _p(cof), _p(cc), _p(ce), M,
                     _p(inc), _p(a), int(budget))
    n = int(L.orc_expand_size(h))
    t = Tree(np.empty(n, np.uint32), np.empty(n, np.uint32), np.empty(n, np.uint32), np.empty(n),
             np.empty((n, M)), bool(L.orc_expand_truncated(h)))
    L.orc_expand_fetch(h, _p(t.parent), _p(t.cnode), _p(t.edge), _p(t.scale), _p(t.incl))
    L.orc_expand_free(h)
    return t


@dataclass
class Sparse:
    prof_off: np.ndarray      # PMS only
    plane_ctx: np.ndarray
    plane_node: np.ndarray
    plane_off: np.ndarray
    metric_id: np.ndarray
    metric_off: np.ndarray    # CMS only
    pid: np.ndarray           # CMS only
    val: np.ndarray


def _flatten(profiles):
    pid = np.concatenate([np.full(len(k), p, np.uint32) for p, k in enumerate(profiles)])
    cat = lambda f, dt: _c(np.concatenate([getattr(k, f) for k in profiles]).astype(dt), dt)
    return _c(pid, np.uint32), cat("ctx", np.uint32), cat("node", np.uint32), cat("stall", np.uint8), cat("val", np.uint64)


def _sparse(L, h):
    sz = np.zeros(4, np.uint64)
    L.orc_sparse_sizes(h, _p(sz))
    npl, nm, nv, npo = (int(x) for x in sz)
    o = Sparse(np.zeros(npo, np.uint64), np.zeros(npl, np.uint32), np.zeros(npl, np.uint32), np.zeros(npl + 1, np.uint64),
               np.zeros(nm, np.uint32), np.zeros(nm + 1 if nm or nv else 1, np.uint64), np.zeros(nv, np.uint32),
               np.zeros(nv, np.uint64))
    L.orc_sparse_fetch(h, _p(o.prof_off), _p(o.plane_ctx), _p(o.plane_node), _p(o.plane_off), _p(o.metric_id),
                       _p(o.metric_off), _p(o.pid), _p(o.val))
    L.orc_sparse_free(h)
    return o


def cms(profiles) -> Sparse:
    """Context-major sparse layout of several key lists (Section 6.2)."""
    L = lib()
    a = _flatten(profiles)
    return _sparse(L, L.orc_cms(a[0].shape[0], *[_p(x) for x in a]))


def pms(profiles) -> Sparse:
    """Profile-major sparse layout of several key lists (Section 6.2)."""
    L = lib()
    a = _flatten(profiles)
    return _sparse(L, L.orc_pms(len(profiles), a[0].shape[0], *[_p(x) for x in a]))


def unify(ccts):
    """Call-path profile unification (Section 6.1).  ccts: [(parent, module,
    offset)] per profile.  Returns (uid per input node, concatenated; merged
    parent, module, offset)."""
    L = lib()
    base = np.zeros(len(ccts) + 1, np.uint64)
    base[1:] = np.cumsum([len(c[0]) for c in ccts])
    par = _c(np.concatenate([c[0] for c in ccts]), np.uint32)
    mod = _c(np.concatenate([c[1] for c in ccts]), np.uint16)
    off = _c(np.concatenate([c[2] for c in ccts]), np.uint64)
    h = L.orc_unify(len(ccts), _p(base), _p(par), _p(mod), _p(off))
    st = L.orc_unify_status(h)
    if st:
        L.orc_unify_free(h)
        raise ValueError(f"oracle unify status {st}")
    n = int(L.orc_unify_size(h))
    uid = np.empty(par.shape[0], np.uint32)
    up, um, uo = np.empty(n, np.uint32), np.empty(n, np.uint16), np.empty(n, np.uint64)
    L.orc_unify_fetch(h, _p(uid), _p(up), _p(um), _p(uo))
    L.orc_unify_free(h)
    return uid, up, um, uo


@dataclass
class BottomUp:
    """Bottom-up view: nodes (parent, func, module, offset), level_off, and
    the values (node, stall, val) ascending by (node, stall)."""
    parent: np.ndarray
    func: np.ndarray
    module: np.ndarray
    offset: np.ndarray
    level_off: np.ndarray
    vnode: np.ndarray
    vstall: np.ndarray
    val: np.ndarray


def bottom_up(node_func, keys: KeyList, cct, levels: int) -> BottomUp:
    """Bottom-up view (Section 7) of a profile.  cct = (parent, module,
    offset) of the calling context tree whose node c is launch context c."""
    L = lib()
    nf = _c(node_func, np.uint32)
    k = [_c(keys.ctx, np.uint32), _c(keys.node, np.uint32), _c(keys.stall, np.uint8), _c(keys.val, np.uint64)]
    par, mod, off = _c(cct[0], np.uint32), _c(cct[1], np.uint16), _c(cct[2], np.uint64)
    h = L.orc_bottom_up(k[0].shape[0], *[_p(x) for x in k], nf.shape[0], _p(nf), par.shape[0], _p(par), _p(mod),
                        _p(off), levels)
    st = L.orc_bu_status(h)
    if st:
        L.orc_bu_free(h)
        raise ValueError(f"oracle bottom_up status {st}")
    n = np.zeros(3, np.uint64)
    L.orc_bu_sizes(h, _p(n))
    nn, nv, nl = (int(x) for x in n)
    b = BottomUp(np.empty(nn, np.uint32), np.empty(nn, np.uint32), np.empty(nn, np.uint16), np.empty(nn, np.uint64),
                 np.empty(nl, np.uint64), np.empty(nv, np.uint32), np.empty(nv, np.uint8), np.empty(nv, np.uint64))
    L.orc_bu_fetch(h, *[_p(x) for x in (b.parent, b.func, b.module, b.offset, b.level_off, b.vnode, b.vstall, b.val)])
    L.orc_bu_free(h)
    return b
