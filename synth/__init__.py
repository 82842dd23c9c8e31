"""Seeded synthetic inputs: GPU binaries' program structure, static call graphs,
host calling-context trees and PC-sample buffers.

This module only *generates* inputs.  It holds none of the analysis arithmetic
(no attribution, aggregation, apportioning or propagation): both the CUDA
library and the CPU oracle consume what it produces.

Every random draw is a counter-based hash (the SplitMix64 finaliser of
Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) of (seed, stream, index), so a sample's fields depend only on its
index: the same buffer comes out identical on the CPU and on a CUDA device,
whole or generated in slices.

Shapes follow the workloads of the paper's setting (Section 4.2: a PC sample
is an instruction address, a stall reason and a count; Section 5: a GPU
binary's instructions map to lines, loops, inlined code and functions;
Section 6.3: a static call graph with call instructions).  The paper's
application profiles are not available, so these seeded stand-ins replace
them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

# node kinds of the program-structure tree (Section 5)
FUNC, INLINE, LOOP, LINE, CALL = 0, 1, 2, 3, 4
NO_PARENT = 0xFFFFFFFF

_GOLD = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _s64(x: int) -> int:
    """Two's-complement int64 view of an unsigned 64-bit constant."""
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= (1 << 63) else x


# ---------------------------------------------------------------- numpy side
def _np_mix(z):
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def np_u64(seed: int, stream: int, idx) -> np.ndarray:
    """uint64 hash of (seed, stream, idx) for an integer array idx."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = _np_mix(np.uint64(seed & ((1 << 64) - 1)) + np.uint64(stream) * np.uint64(_GOLD))
        return _np_mix(base + (idx + np.uint64(1)) * np.uint64(_GOLD))


def np_unif(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform float64 in [0, 1) with 53 random bits."""
    return (np_u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def np_below(seed: int, stream: int, idx, n) -> np.ndarray:
    """Integer uniform in [0, n) (n may be an array)."""
    u = np_unif(seed, stream, idx)
    r = np.floor(u * np.asarray(n, dtype=np.float64)).astype(np.int64)
    return np.minimum(r, np.asarray(n, dtype=np.int64) - 1)


# ---------------------------------------------------------------- torch side
def _t_srl(x: torch.Tensor, k: int) -> torch.Tensor:
    return (x >> k) & ((1 << (64 - k)) - 1)


def _t_mix(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _t_srl(z, 30)) * _s64(_M1)
    z = (z ^ _t_srl(z, 27)) * _s64(_M2)
    return z ^ _t_srl(z, 31)


def t_u64(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Same hash as np_u64, as int64 bit patterns, on idx's device."""
    with np.errstate(over="ignore"):
        b = _np_mix(np.uint64(seed & ((1 << 64) - 1)) + np.uint64(stream) * np.uint64(_GOLD))
    z = (idx.to(torch.int64) + 1) * _s64(_GOLD) + _s64(int(b))
    return _t_mix(z)


def t_unif(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    return _t_srl(t_u64(seed, stream, idx), 11).to(torch.float64) * (2.0 ** -53)


# ---------------------------------------------------------------- structures
@dataclasses.dataclass
class Binary:
    """Program structure of one synthetic GPU binary (all numpy, host side).

    Ranges are disjoint, sorted by lo, half-open [lo, hi); every range maps to
    a LINE or CALL node.  Function f occupies [func_lo[f], func_hi[f]); its
    last `pad` slots are covered by no range (alignment padding), so samples
    there are attributed to no node.
    """
    range_lo: np.ndarray      # uint64[R]
    range_hi: np.ndarray      # uint64[R]
    range_node: np.ndarray    # uint32[R]
    node_parent: np.ndarray   # uint32[M]  (NO_PARENT for FUNC nodes)
    node_kind: np.ndarray     # uint8[M]
    node_func: np.ndarray     # uint32[M]
    func_node: np.ndarray     # uint32[F]  FUNC node of each function
    func_lo: np.ndarray       # uint64[F]
    func_hi: np.ndarray       # uint64[F]
    cs_pc: np.ndarray         # uint64[E]  address of the call instruction
    cs_caller: np.ndarray     # uint32[E]
    cs_callee: np.ndarray     # uint32[E]
    cs_node: np.ndarray       # uint32[E]  CALL node of the call instruction
    seg_lo: int
    seg_hi: int

    @property
    def n_funcs(self): return int(self.func_lo.shape[0])

    @property
    def n_nodes(self): return int(self.node_parent.shape[0])

    @property
    def n_ranges(self): return int(self.range_lo.shape[0])

    @property
    def n_calls(self): return int(self.cs_pc.shape[0])


def _call_graph(seed: int, F: int, E: int, n_scc: int, scc_lo: int, scc_hi: int):
    """Static call graph over F functions with E call sites.

    Functions get a seeded topological position; every non-root function has
    at least one caller earlier in that order.  With n_scc > 0, groups of
    scc_lo..scc_hi functions are closed into cycles by back edges.
    Returns (caller, callee, topo) with topo[pos] = function id.
    """
    topo = np.argsort(np_u64(seed, 101, np.arange(F)), kind="stable").astype(np.int64)
    n_roots = max(1, F // 100)
    callers, callees = [], []
    # one guaranteed caller per non-root function
    pos = np.arange(n_roots, F)
    par = np_below(seed, 102, pos, pos)
    callers.append(topo[par]); callees.append(topo[pos])
    # cycles
    if n_scc > 0:
        starts = np.sort(np_below(seed, 103, np.arange(n_scc), F - scc_hi - 1 - n_roots) + n_roots)
        cur = 0
        for g in range(n_scc):
            k = scc_lo + int(np_below(seed, 104, [g], scc_hi - scc_lo + 1)[0])
            s0 = max(int(starts[g]), cur)
            if s0 + k > F:
                break
            members = topo[s0:s0 + k]
            callers.append(members); callees.append(np.roll(members, -1))
            cur = s0 + k
    have = sum(len(c) for c in callers)
    rest = max(0, E - have)
    if rest:
        idx = np.arange(rest)
        a = np_below(seed, 105, idx, F)
        b = np_below(seed, 106, idx, F)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        hi = np.where(hi == lo, np.minimum(lo + 1, F - 1), hi)
        ok = hi > lo
        callers.append(topo[lo[ok]]); callees.append(topo[hi[ok]])
    caller = np.concatenate(callers).astype(np.uint32)
    callee = np.concatenate(callees).astype(np.uint32)
    return caller, callee, topo


def make_binary(seed: int, n_funcs: int, seg_bytes: int, n_line_ranges: int,
                n_calls: int, n_scc: int = 0, scc_size=(2, 12),
                seg_base: int = 0x7F0000000000, min_fn_bytes: int = 1024,
                max_fn_bytes: int = 65536) -> Binary:
    """One binary: functions tiling a code segment, a scope tree per function
    (<= 3 inlined scopes, loop nests <= 4 deep, line ranges, call
    instructions), and a static call graph."""
    F = n_funcs
    # --- function sizes: log-uniform, rescaled to fill 99 % of the segment, 16-B aligned
    u = np_unif(seed, 1, np.arange(F))
    raw = np.exp(np.log(min_fn_bytes) + u * (np.log(max_fn_bytes) - np.log(min_fn_bytes)))
    body = seg_bytes * 0.99
    sizes = np.maximum(64, np.floor(raw * (body / raw.sum()) / 16) * 16).astype(np.int64)
    gap_total = max(0, seg_bytes - int(sizes.sum()))
    gu = np_unif(seed, 2, np.arange(F))
    gaps = np.floor(gu / gu.sum() * gap_total / 16).astype(np.int64) * 16
    starts = seg_base + np.concatenate([[0], np.cumsum(sizes + gaps)[:-1]]) + gaps[0] * 0
    func_lo = starts.astype(np.uint64)
    func_hi = (starts + sizes).astype(np.uint64)
    slots = sizes // 16

    caller, callee, _topo = _call_graph(seed, F, n_calls, n_scc, *scc_size)
    E = caller.shape[0]
    # call sites grouped by caller
    order = np.argsort(caller, kind="stable")
    caller, callee = caller[order], callee[order]
    calls_of = np.split(np.arange(E), np.searchsorted(caller, np.arange(1, F)))

    lines_per_slot = n_line_ranges / float(slots.sum())
    node_parent, node_kind, node_func = [], [], []
    r_lo, r_hi, r_node = [], [], []
    func_node = np.zeros(F, np.uint32)
    cs_pc = np.zeros(E, np.uint64)
    cs_node = np.zeros(E, np.uint32)

    def new_node(parent, kind, f):
        node_parent.append(parent); node_kind.append(kind); node_func.append(f)
        return len(node_parent) - 1

    for f in range(F):
        fs = seed * 1_000_003 + f * 7919 + 17
        n_sl = int(slots[f])
        pad = max(1, n_sl // 100)
        cov = n_sl - pad
        fn = new_node(NO_PARENT, FUNC, f)
        func_node[f] = fn
        my_calls = calls_of[f]
        nc = len(my_calls)
        # call instruction slots: distinct slots in [0, cov)
        if nc > cov:
            raise ValueError("function too small for its call sites")
        cslots = np.sort(np.argsort(np_u64(fs, 3, np.arange(cov)))[:nc]) if nc else np.zeros(0, np.int64)
        # line ranges: cut [0, cov) into L pieces
        L = int(max(1, min(cov, round(lines_per_slot * n_sl))))
        if L > 1:
            cuts = np.sort(np.argsort(np_u64(fs, 4, np.arange(1, cov)))[:L - 1] + 1)
        else:
            cuts = np.zeros(0, np.int64)
        bounds = np.concatenate([[0], cuts, [cov]]).astype(np.int64)
        # scopes over line-range indices [0, L): up to 3 inlined scopes, one loop nest <= 4
        scope_of = np.full(L, fn, dtype=np.int64)  # innermost scope node per line range
        su = np_u64(fs, 5, np.arange(32))
        n_inl = min(int(su[0] % np.uint64(4)), (L + 1) // 2) if L >= 2 else 0
        containers = [(0, L, fn)]
        if n_inl:
            pts = np.sort(np.argsort(np_u64(fs, 6, np.arange(L + 1)))[:2 * n_inl])
            for k in range(n_inl):
                a, b = int(pts[2 * k]), int(pts[2 * k + 1])
                if b > a:
                    nd = new_node(fn, INLINE, f)
                    scope_of[a:b] = nd
                    containers.append((a, b, nd))
        depth = int(su[1] % np.uint64(5))
        if depth and L >= 1:
            a, b, par = containers[int(su[2] % np.uint64(len(containers)))]
            for d in range(depth):
                if b - a < 1:
                    break
                w = b - a
                x0 = a + int(su[3 + 2 * d] % np.uint64(max(1, w)))
                x1 = x0 + 1 + int(su[4 + 2 * d] % np.uint64(max(1, b - x0)))
                x1 = min(x1, b)
                nd = new_node(par, LOOP, f)
                scope_of[x0:x1] = nd
                a, b, par = x0, x1, nd
        # line nodes: one per range, ~10 % reuse an earlier line of the same scope
        lu = np_unif(fs, 7, np.arange(L))
        line_of = np.zeros(L, np.int64)
        last_line = {}
        for j in range(L):
            sc = int(scope_of[j])
            if lu[j] < 0.1 and sc in last_line:
                line_of[j] = last_line[sc]
            else:
                line_of[j] = new_node(sc, LINE, f)
                last_line[sc] = line_of[j]
        # CALL nodes under the line containing each call slot
        rng_of_call = np.searchsorted(bounds, cslots, side="right") - 1
        call_nodes = np.zeros(nc, np.int64)
        for k in range(nc):
            call_nodes[k] = new_node(int(line_of[rng_of_call[k]]), CALL, f)
        # final ranges: line ranges split around call slots
        pts = np.unique(np.concatenate([bounds, cslots, cslots + 1]))
        lo_s, hi_s = pts[:-1], pts[1:]
        is_call = np.isin(lo_s, cslots) & (hi_s == lo_s + 1)
        line_idx = np.searchsorted(bounds, lo_s, side="right") - 1
        nodes = np.where(is_call, 0, line_of[np.minimum(line_idx, L - 1)])
        if nc:
            ck = np.searchsorted(cslots, lo_s[is_call])
            nodes[is_call] = call_nodes[ck]
            cs_pc[my_calls] = func_lo[f] + (cslots * 16).astype(np.uint64)
            cs_node[my_calls] = call_nodes.astype(np.uint32)
        r_lo.append(func_lo[f] + (lo_s * 16).astype(np.uint64))
        r_hi.append(func_lo[f] + (hi_s * 16).astype(np.uint64))
        r_node.append(nodes.astype(np.uint32))

    return Binary(
        range_lo=np.concatenate(r_lo).astype(np.uint64),
        range_hi=np.concatenate(r_hi).astype(np.uint64),
        range_node=np.concatenate(r_node).astype(np.uint32),
        node_parent=np.array(node_parent, dtype=np.uint32),
        node_kind=np.array(node_kind, dtype=np.uint8),
        node_func=np.array(node_func, dtype=np.uint32),
        func_node=func_node, func_lo=func_lo, func_hi=func_hi,
        cs_pc=cs_pc, cs_caller=caller.astype(np.uint32), cs_callee=callee.astype(np.uint32),
        cs_node=cs_node, seg_lo=int(func_lo[0]), seg_hi=int(func_hi[-1]))


def make_cct(seed: int, n_nodes: int, max_depth: int, max_fanout: int) -> np.ndarray:
    """Host calling-context tree: parent[v] < v, parent[0] = NO_PARENT,
    depth <= max_depth, at most max_fanout children per node."""
    parent = np.full(n_nodes, NO_PARENT, dtype=np.uint32)
    depth = np.zeros(n_nodes, np.int64)
    fan = np.zeros(n_nodes, np.int64)
    r = np_u64(seed, 201, np.arange(n_nodes * 4))
    open_nodes = [0]          # nodes that may still take children
    for v in range(1, n_nodes):
        while True:
            k = int(r[v * 4] % np.uint64(len(open_nodes)))
            p = open_nodes[k]
            if fan[p] < max_fanout and depth[p] < max_depth:
                break
            open_nodes[k] = open_nodes[-1]; open_nodes.pop()
        parent[v] = p; depth[v] = depth[p] + 1; fan[p] += 1
        if fan[p] >= max_fanout:
            open_nodes.remove(p)
        if depth[v] < max_depth:
            open_nodes.append(v)
    return parent


def make_cct_levels(seed: int, n_nodes: int, max_depth: int, max_fanout: int) -> np.ndarray:
    """Large host calling-context tree built level by level (vectorised):
    every node of a level draws 0..max_fanout children so that about n_nodes
    nodes fit in max_depth levels; node ids follow the levels, so
    parent[v] < v, parent[0] = NO_PARENT, depth <= max_depth."""
    m = max(1.05, min(float(max_fanout), n_nodes ** (1.0 / max(2, (3 * max_depth) // 4))))
    parent = [np.array([NO_PARENT], dtype=np.uint32)]
    level = np.array([0], dtype=np.int64)
    total = 1
    d = 0
    while total < n_nodes and d < max_depth:
        u = np_unif(seed, 211 + d, np.arange(level.shape[0]))
        kids = np.minimum(np.floor(-np.log1p(-u) * (m + 0.5)).astype(np.int64), max_fanout)   # ~ geometric
        if kids.sum() == 0:
            kids[0] = 1
        kids = kids[: np.searchsorted(np.cumsum(kids), n_nodes - total, side="left") + 1]
        par = np.repeat(level[: kids.shape[0]], kids)[: n_nodes - total]
        nxt = np.arange(total, total + par.shape[0], dtype=np.int64)
        parent.append(par.astype(np.uint32))
        total += par.shape[0]
        level = nxt
        d += 1
    out = np.concatenate(parent)
    if out.shape[0] < n_nodes:
        # depth limit reached first: the remaining nodes go to nodes above the
        # last level that still have room for children, in id order
        depth = np.concatenate([np.full(p.shape[0], k, np.int64) for k, p in enumerate(parent)])
        while out.shape[0] < n_nodes:
            fan = np.bincount(out[1:].astype(np.int64), minlength=out.shape[0])
            room = np.where(depth < max_depth, max_fanout - fan, 0)
            slots = np.repeat(np.arange(out.shape[0]), room)[: n_nodes - out.shape[0]]
            if slots.shape[0] == 0:
                raise ValueError("n_nodes does not fit in max_depth levels of max_fanout children")
            out = np.concatenate([out, slots.astype(np.uint32)])
            depth = np.concatenate([depth, depth[slots] + 1])
    return out


def cct_sites(seed: int, par: np.ndarray, n_sites: int = 0, fan: int = 8):
    """Call sites (module, offset) of the nodes of a calling context tree
    (parent < child) that repeat under different parents, as a callee's call
    sites do under each of its calling contexts: site = a seeded pick per
    depth among n_sites // fan groups, plus the node's rank among its
    siblings, so that siblings never share one; module = site % 8, offset =
    0x1000 + 16 site.  Returns (module u16, offset u64, depth i64)."""
    n = par.shape[0]
    dep = np.zeros(n, np.int64)
    anc = par.astype(np.int64)
    while True:                                         # depth by walking every node up one step at a time
        up = anc != NO_PARENT
        if not up.any():
            break
        dep += up
        anc[up] = par[anc[up]].astype(np.int64)
    order = np.argsort(par, kind="stable")
    first = np.searchsorted(par[order], par[order], side="left")
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n) - first
    assert rank.max(initial=0) < fan
    groups = max(1, (n_sites or max(64, n // 4)) // fan)
    site = np_below(seed, 503, dep, groups).astype(np.int64) * fan + rank
    return (site % 8).astype(np.uint16), (0x1000 + 16 * site).astype(np.uint64), dep


def make_profile_ccts(seed: int, n_master: int, depth: int, n_profiles: int, keep: float, n_sites: int = 0):
    """Per-profile calling context trees for unification: a master tree whose
    call sites repeat under different parents (cct_sites); profile p keeps a
    seeded subset of the master's nodes closed under parents, in master
    order.  Returns [(parent, module, offset)] with parents as indices within
    the profile (HPA_NO_PARENT for a root)."""
    par = make_cct_levels(seed, n_master, depth, 8)
    idx = np.arange(n_master)
    module, offset, dep = cct_sites(seed, par, n_sites)
    lv = np.argsort(dep, kind="stable")
    by_level = np.split(lv, np.searchsorted(dep[lv], np.arange(1, int(dep.max(initial=0)) + 1)))
    out = []
    for p in range(n_profiles):
        kept = np_unif(seed, 510 + p, idx) < keep
        for d in range(int(dep.max(initial=0)), 0, -1):   # close under parents, deepest level first
            v = by_level[d]
            kept[par[v[kept[v]]]] = True
        local = np.cumsum(kept) - 1
        sel = np.nonzero(kept)[0]
        mp = par[sel]
        lp = np.where(mp == NO_PARENT, NO_PARENT, local[np.minimum(mp, n_master - 1)]).astype(np.uint32)
        out.append((lp, module[sel], offset[sel]))
    return out


# ---------------------------------------------------------------- samples
@dataclasses.dataclass
class Samples:
    pc: torch.Tensor                # int64 bit patterns of uint64 PCs
    ctx: torch.Tensor               # int32 bit patterns of uint32 ids
    stall: torch.Tensor             # uint8
    count: torch.Tensor | None      # int32 bit patterns of uint32 counts
    n_ctx: int
    n_stall: int

    @property
    def n(self): return int(self.pc.shape[0])

    def to(self, device):
        return Samples(self.pc.to(device), self.ctx.to(device), self.stall.to(device),
                       None if self.count is None else self.count.to(device),
                       self.n_ctx, self.n_stall)

    def slice(self, a, b):
        return Samples(self.pc[a:b], self.ctx[a:b], self.stall[a:b],
                       None if self.count is None else self.count[a:b], self.n_ctx, self.n_stall)


def stall_cdf(n_stall: int, q: float = 0.6) -> np.ndarray:
    p = q ** np.arange(n_stall, dtype=np.float64)
    c = np.cumsum(p / p.sum())
    c[-1] = 1.0
    return c


def zipf_cdf(n: int, s: float) -> np.ndarray:
    p = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(p / p.sum())
    c[-1] = 1.0
    return c


def make_samples(seed: int, b: Binary, n: int, n_ctx: int, zipf_s: float,
                 n_stall: int = 16, counts: bool = False, device="cpu",
                 start: int = 0, ctx_weights: np.ndarray | None = None,
                 chunk: int = 1 << 25) -> Samples:
    """PC samples [start, start + n) of a seeded stream.

    Function ~ Zipf(zipf_s) over a seeded permutation; PC uniform over the
    function's 16-byte slots; stall reason r with p ∝ 0.6^r; context uniform
    over n_ctx (or drawn from ctx_weights); count 1 + Geometric(1/2) if counts.
    """
    dev = torch.device(device)
    F = b.n_funcs
    perm = torch.from_numpy(np.argsort(np_u64(seed, 301, np.arange(F)), kind="stable").astype(np.int64)).to(dev)
    fcdf = torch.from_numpy(zipf_cdf(F, zipf_s)).to(dev)
    scdf = torch.from_numpy(stall_cdf(n_stall)).to(dev)
    ccdf = None
    if ctx_weights is not None:
        w = np.asarray(ctx_weights, np.float64)
        c = np.cumsum(w / w.sum()); c[-1] = 1.0
        ccdf = torch.from_numpy(c).to(dev)
    flo = torch.from_numpy(b.func_lo.view(np.int64)).to(dev)
    nsl = torch.from_numpy(((b.func_hi - b.func_lo) // np.uint64(16)).astype(np.int64)).to(dev)
    pcs = [torch.zeros(0, dtype=torch.int64, device=dev)]
    ctxs = [torch.zeros(0, dtype=torch.int32, device=dev)]
    stalls = [torch.zeros(0, dtype=torch.uint8, device=dev)]
    cnts = [torch.zeros(0, dtype=torch.int32, device=dev)]
    for a in range(start, start + n, chunk):
        e = min(start + n, a + chunk)
        idx = torch.arange(a, e, device=dev, dtype=torch.int64)
        rank = torch.searchsorted(fcdf, t_unif(seed, 1, idx), right=True).clamp_(max=F - 1)
        f = perm[rank]
        slot = torch.floor(t_unif(seed, 2, idx) * nsl[f].to(torch.float64)).to(torch.int64)
        slot = torch.minimum(slot, nsl[f] - 1)
        pcs.append(flo[f] + slot * 16)
        st = torch.searchsorted(scdf, t_unif(seed, 3, idx), right=True).clamp_(max=n_stall - 1)
        stalls.append(st.to(torch.uint8))
        if ccdf is None:
            cx = torch.floor(t_unif(seed, 4, idx) * n_ctx).to(torch.int64).clamp_(max=n_ctx - 1)
        else:
            cx = torch.searchsorted(ccdf, t_unif(seed, 4, idx), right=True).clamp_(max=n_ctx - 1)
        ctxs.append(cx.to(torch.int32))
        if counts:
            r = t_u64(seed, 5, idx)
            low = r & (-r)                      # lowest set bit: P(bit k) = 2^-(k+1)
            k = torch.where(low == 0, torch.zeros_like(r),
                            torch.log2(low.to(torch.float64).abs()).to(torch.int64))
            cnts.append((1 + k).to(torch.int32))
        del idx
    return Samples(torch.cat(pcs), torch.cat(ctxs), torch.cat(stalls),
                   torch.cat(cnts) if counts else None, n_ctx, n_stall)


def make_tuple_samples(seed: int, b: Binary, n: int, n_ctx: int, n_tuples: int,
                       n_stall: int = 16, device="cpu") -> Samples:
    """Many-context workload: n_tuples distinct (ctx, range, stall) tuples are
    drawn first; samples are uniform over the tuples, PC uniform within the
    tuple's range."""
    dev = torch.device(device)
    ti = np.arange(n_tuples)
    t_ctx = np_below(seed, 401, ti, n_ctx)
    t_rng = np_below(seed, 402, ti, b.n_ranges)
    t_st = np_below(seed, 403, ti, n_stall)
    lo = torch.from_numpy(b.range_lo.view(np.int64)).to(dev)
    nsl = torch.from_numpy(((b.range_hi - b.range_lo) // np.uint64(16)).astype(np.int64)).to(dev)
    t_ctx_t = torch.from_numpy(t_ctx).to(dev)
    t_rng_t = torch.from_numpy(t_rng).to(dev)
    t_st_t = torch.from_numpy(t_st).to(dev)
    idx = torch.arange(n, device=dev, dtype=torch.int64)
    t = torch.floor(t_unif(seed, 404, idx) * n_tuples).to(torch.int64).clamp_(max=n_tuples - 1)
    rg = t_rng_t[t]
    slot = torch.floor(t_unif(seed, 405, idx) * nsl[rg].to(torch.float64)).to(torch.int64)
    slot = torch.minimum(slot, nsl[rg] - 1)
    return Samples(lo[rg] + slot * 16, t_ctx_t[t].to(torch.int32), t_st_t[t].to(torch.uint8),
                   None, n_ctx, n_stall)


# ---------------------------------------------------------------- workloads
@dataclasses.dataclass
class Workload:
    name: str
    seed: int
    n_funcs: int
    seg_bytes: int
    n_line_ranges: int
    n_calls: int
    n_samples: int
    n_ctx: int
    zipf_s: float
    counts: bool
    n_scc: int = 0
    cct_depth: int = 32
    cct_fanout: int = 8
    n_stall: int = 16

    def binary(self) -> Binary:
        return make_binary(self.seed, self.n_funcs, self.seg_bytes, self.n_line_ranges,
                           self.n_calls, self.n_scc)

    def samples(self, b: Binary, device="cpu", n: int | None = None, start: int = 0) -> Samples:
        return make_samples(self.seed, b, self.n_samples if n is None else n, self.n_ctx,
                            self.zipf_s, self.n_stall, self.counts, device, start)

    def cct(self) -> np.ndarray:
        return make_cct(self.seed, self.n_ctx, self.cct_depth, self.cct_fanout)


SEED_BASE = 2109_06931

# plain, single profile: 2,000 functions / 32 MB / 60,000 line ranges / 4,000 call sites /
# 10^6 samples, Zipf 1.1, 500 launch contexts, no counts
PLAIN = Workload("plain-1M", SEED_BASE + 1, 2000, 32 << 20, 60_000, 4000, 1_000_000, 500, 1.1, False)
# plain, large single profile: 40,000 functions / 512 MB / 2,000,000 line ranges /
# 120,000 call sites with 50 recursive SCCs / 2x10^8 samples, Zipf 0.9, 20,000 contexts,
# uint32 counts
LARGE = Workload("plain-large-200M", SEED_BASE + 2, 40_000, 512 << 20, 2_000_000, 120_000,
                 200_000_000, 20_000, 0.9, True, n_scc=50)


def scaled(w: Workload, frac: float, name: str | None = None) -> Workload:
    """Same recipe with the sample count scaled (structure unchanged)."""
    return dataclasses.replace(w, name=name or f"{w.name}@{frac:g}",
                               n_samples=max(1, int(w.n_samples * frac)))


def batch_sizes(seed: int, n_buf: int, lo: float, hi: float) -> np.ndarray:
    """Log-uniform buffer sizes in [lo, hi]."""
    u = np_unif(seed, 501, np.arange(n_buf))
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


# batched: 256 per-rank buffers, sizes log-uniform in [1e4, 5e7], against 8
# binaries of 2,000-40,000 functions (assigned round-robin)
@dataclasses.dataclass
class BatchWorkload:
    name: str
    seed: int
    n_buffers: int
    size_lo: float
    size_hi: float
    n_binaries: int
    funcs_lo: int
    funcs_hi: int
    n_ctx: int
    zipf_s: float
    counts: bool
    n_stall: int = 16

    def sizes(self) -> np.ndarray:
        return batch_sizes(self.seed, self.n_buffers, self.size_lo, self.size_hi)

    def binary_params(self):
        """(functions, code bytes, line ranges, call sites) per binary: the
        large workload's densities scaled by the function count."""
        u = np_unif(self.seed, 601, np.arange(self.n_binaries))
        F = np.floor(np.exp(math.log(self.funcs_lo) + u * (math.log(self.funcs_hi) - math.log(self.funcs_lo))))
        out = []
        for f in F.astype(np.int64):
            out.append((int(f), int(f) * 13_422, int(f) * 50, int(f) * 3))   # ~13 KB, 50 lines, 3 calls / function
        return out

    def binaries(self):
        return [make_binary(self.seed * 31 + i, f, seg, lines, calls)
                for i, (f, seg, lines, calls) in enumerate(self.binary_params())]

    def buffer(self, b: int, binary: Binary, n: int, device="cpu") -> Samples:
        return make_samples(self.seed * 1_000 + b, binary, n, self.n_ctx, self.zipf_s, self.n_stall,
                            self.counts, device)


@dataclasses.dataclass
class ManyCtxWorkload:
    """Batched buffers over a large merged calling-context tree: per buffer,
    n_tuples distinct (ctx, range, stall) tuples are drawn first and the
    samples are uniform over the tuples (no counts); one binary."""
    name: str
    seed: int
    n_buffers: int
    n_samples: int
    n_tuples: int
    cct_nodes: int
    cct_depth: int
    base: "Workload"
    n_stall: int = 16

    def binary(self) -> Binary:
        return self.base.binary()

    def cct(self) -> np.ndarray:
        return make_cct_levels(self.seed, self.cct_nodes, self.cct_depth, 8)

    def buffer(self, b: int, binary: Binary, n: int | None = None, device="cpu") -> Samples:
        return make_tuple_samples(self.seed * 1_000 + b, binary, self.n_samples if n is None else n,
                                  self.cct_nodes, self.n_tuples, self.n_stall, device)


BATCHED = BatchWorkload("batched-256x", SEED_BASE + 3, 256, 1e4, 5e7, 8, 2000, 40_000, 500, 1.0, True)
# batched, many contexts: 64 buffers x 3x10^7 samples, 10^6 (ctx, range, stall)
# tuples per buffer over a merged CCT of 2x10^6 nodes (depth <= 64); the large
# workload's binary
MANY_CTX = ManyCtxWorkload("batched-many-ctx-64x", SEED_BASE + 4, 64, 30_000_000, 1_000_000, 2_000_000, 64, LARGE)
