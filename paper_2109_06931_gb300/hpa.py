"""Python binding of libhpa.so (include/hpa.h): argument marshalling only.

Every analysis step runs in the library's CUDA kernels; this module converts
torch tensors and numpy arrays into the C structures and calls the C ABI.
It raises if the library or a CUDA device is missing -- there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

HPA_OK, HPA_E_INVALID_ARG, HPA_E_INVALID_TABLE, HPA_E_INVALID_SAMPLE = 0, 1, 2, 3
HPA_E_CAPACITY, HPA_E_OOM, HPA_E_CUDA, HPA_E_TIMEOUT, HPA_E_INTERNAL = 4, 5, 6, 7, 8
HPA_BUILD_CHECKED = 1
HPA_PENDING = 9
HPA_UNKNOWN_NODE = 0xFFFFFFFF
HPA_NO_PARENT = 0xFFFFFFFF
HPA_MAX_STALL = 32
HPA_TUNE_CANDIDATES = 16
HPA_EDGE_FIXUP, HPA_EDGE_FIXUP2, HPA_EDGE_INTRA_SCC = 1, 2, 4
LEAF_CAPS = (4096, 10240)   # leaf capacities of the aggregation (small, large)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "INVALID_TABLE", 3: "INVALID_SAMPLE", 4: "CAPACITY",
                5: "OOM", 6: "CUDA", 7: "TIMEOUT", 8: "INTERNAL", 9: "PENDING"}

vp, u8p, u32p, u64p = C.c_void_p, C.POINTER(C.c_uint8), C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)


class hpa_options(C.Structure):
    _fields_ = [("issued_mask", C.c_uint32), ("leaf_capacity", C.c_uint32), ("timeout_iters", C.c_uint32),
                ("cursor_pad", C.c_uint32), ("leaf_ranking", C.c_uint32), ("grouping", C.c_uint32),
                ("small_leaves", C.c_uint32), ("leaf_hash", C.c_uint32), ("leaf_emit", C.c_uint32)]


class hpa_structure(C.Structure):
    _fields_ = [("n_ranges", C.c_uint64), ("range_lo", vp), ("range_hi", vp), ("range_node", vp),
                ("n_nodes", C.c_uint32), ("node_parent", vp), ("node_kind", vp), ("node_func", vp),
                ("n_funcs", C.c_uint32), ("n_calls", C.c_uint32), ("cs_caller", vp), ("cs_callee", vp),
                ("cs_node", vp)]


class hpa_binary_info(C.Structure):
    _fields_ = [("n_nodes", C.c_uint32), ("n_funcs", C.c_uint32), ("n_calls", C.c_uint32),
                ("n_cnodes", C.c_uint32), ("n_scc", C.c_uint32), ("cdag_levels", C.c_uint32),
                ("n_ranges", C.c_uint64), ("max_depth", C.c_uint32), ("reserved", C.c_uint32)]


class hpa_samples(C.Structure):
    _fields_ = [("n", C.c_uint64), ("pc", vp), ("ctx", vp), ("stall", vp), ("count", vp),
                ("n_ctx", C.c_uint32), ("n_stall", C.c_uint32)]


class hpa_profile(C.Structure):
    _fields_ = [("capacity", C.c_uint64), ("key_ctx", vp), ("key_node", vp), ("key_stall", vp), ("val", vp),
                ("n_keys", vp), ("total", vp), ("unknown", vp), ("n_ctx", C.c_uint32), ("n_stall", C.c_uint32),
                ("n_nodes", C.c_uint32), ("reserved", C.c_uint32)]


class hpa_gpucct(C.Structure):
    _fields_ = [("n_req", C.c_uint32), ("req_ctx", vp), ("incl", vp), ("a", vp), ("flags", vp)]


class hpa_gpucct_all(C.Structure):
    _fields_ = [("cap_nodes", C.c_uint64), ("cap_edges", C.c_uint64), ("node_off", vp), ("node_id", vp),
                ("incl", vp), ("edge_off", vp), ("edge_id", vp), ("ratio", vp), ("a", vp), ("flags", vp),
                ("counts", vp)]


class hpa_issue_rows(C.Structure):
    _fields_ = [("capacity", C.c_uint64), ("ctx", vp), ("func", vp), ("S", vp), ("S_issued", vp), ("W", vp),
                ("frac", vp), ("n_rows", vp)]


class hpa_ratio_rows(C.Structure):
    _fields_ = [("capacity", C.c_uint64), ("key_ctx", vp), ("key_node", vp), ("key_stall", vp), ("num", vp),
                ("den", vp), ("ratio", vp), ("n_keys", vp)]


class hpa_cct(C.Structure):
    _fields_ = [("n_nodes", C.c_uint32), ("parent", vp)]


class hpa_server_options(C.Structure):
    _fields_ = [("mem_cap_bytes", C.c_uint64), ("max_batch", C.c_uint32), ("max_inflight", C.c_uint32),
                ("reserved", C.c_uint32 * 4)]


class hpa_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("samples", C.c_uint64), ("batches", C.c_uint64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("max_ms", C.c_double), ("mean_ms", C.c_double), ("busy_s", C.c_double),
                ("h2d_ms", C.c_double), ("wait_compute_ms", C.c_double), ("compute_ms", C.c_double),
                ("wait_d2h_ms", C.c_double), ("d2h_ms", C.c_double), ("launch_ms", C.c_double)]


class hpa_cct_tree(C.Structure):
    _fields_ = [("budget", C.c_uint32), ("parent", vp), ("cnode", vp), ("edge", vp), ("scale", vp), ("incl", vp),
                ("n_nodes", vp), ("truncated", vp)]


class hpa_cms(C.Structure):
    _fields_ = [("cap_planes", C.c_uint64), ("cap_metrics", C.c_uint64), ("cap_values", C.c_uint64),
                ("plane_ctx", vp), ("plane_node", vp), ("plane_off", vp), ("metric_id", vp), ("metric_off", vp),
                ("pid", vp), ("val", vp), ("counts", vp)]


class hpa_pms(C.Structure):
    _fields_ = [("cap_planes", C.c_uint64), ("cap_values", C.c_uint64), ("prof_off", vp), ("plane_ctx", vp),
                ("plane_node", vp), ("plane_off", vp), ("metric_id", vp), ("val", vp), ("counts", vp)]


class hpa_cct_nodes(C.Structure):
    _fields_ = [("n_nodes", C.c_uint32), ("parent", vp), ("module", vp), ("offset", vp)]


class hpa_cct_unified(C.Structure):
    _fields_ = [("capacity", C.c_uint32), ("uid", vp), ("parent", vp), ("module", vp), ("offset", vp),
                ("n_unified", vp)]


class hpa_bottom_up(C.Structure):
    _fields_ = [("levels", C.c_uint32), ("cap_nodes", C.c_uint64), ("cap_values", C.c_uint64),
                ("parent", vp), ("func", vp), ("module", vp), ("offset", vp), ("level_off", vp),
                ("val_node", vp), ("val_stall", vp), ("val", vp), ("counts", vp)]


class hpa_derived(C.Structure):
    _fields_ = [("capacity", C.c_uint64), ("key_ctx", vp), ("key_node", vp), ("key_stall", vp),
                ("sum", vp), ("min", vp), ("max", vp), ("mean", vp), ("std", vp), ("cov", vp),
                ("n_keys", vp), ("n_ctx", C.c_uint32), ("S", vp), ("S_issued", vp), ("W", vp), ("frac", vp)]


EXPORTS = ["hpa_create", "hpa_destroy", "hpa_last_error", "hpa_sync", "hpa_reserve", "hpa_kernel_launches",
           "hpa_load_structure", "hpa_unload_structure", "hpa_binary_info_get", "hpa_attribute_samples",
           "hpa_attribute_samples_host", "hpa_attribute_batch", "hpa_apportion_callgraph",
           "hpa_propagate_inclusive", "hpa_derive_metrics", "hpa_apportion_all", "hpa_issue_by_function", "hpa_ratio_of_sums", "hpa_build_flags", "hpa_set_phase_timing", "hpa_phase_times",
           "hpa_attribute_samples_noalloc", "hpa_server_create", "hpa_server_submit", "hpa_server_poll",
           "hpa_server_stats_get", "hpa_server_destroy"]
PHASES = ["hist+plan", "attribute+scatter", "big-split", "leaf sort/reduce", "emit"]

_libs = {}


def lib(build_if_needed: bool = True, checked: bool | None = None):
    """Load libhpa.so (building it first if needed); checked=True loads the
    bounds-checked flavour libhpa_checked.so instead (default: the
    HPA_CHECKED environment variable)."""
    if checked is None:
        checked = os.environ.get("HPA_CHECKED", "0") not in ("", "0")
    if checked not in _libs:
        path = _build.lib_path(checked)
        if build_if_needed:
            path = _build.build(checked=checked)
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not built at {path}")
        L = C.CDLL(path)
        H = vp
        L.hpa_create.argtypes = [C.POINTER(H), C.c_int, vp, C.POINTER(hpa_options)]
        L.hpa_destroy.argtypes = [H]
        L.hpa_last_error.argtypes = [H]
        L.hpa_last_error.restype = C.c_char_p
        L.hpa_sync.argtypes = [H, u64p]
        L.hpa_reserve.argtypes = [H, C.c_uint64, C.c_uint64]
        L.hpa_kernel_launches.argtypes = [H]
        L.hpa_build_flags.argtypes = []
        L.hpa_build_flags.restype = C.c_uint32
        L.hpa_kernel_launches.restype = C.c_uint64
        L.hpa_load_structure.argtypes = [H, C.POINTER(hpa_structure), u32p]
        L.hpa_validate_structure.argtypes = [C.POINTER(hpa_structure), C.c_char_p, C.c_size_t]
        L.hpa_unload_structure.argtypes = [H, C.c_uint32]
        L.hpa_binary_info_get.argtypes = [H, C.c_uint32, C.POINTER(hpa_binary_info), vp]
        L.hpa_attribute_samples.argtypes = [H, C.c_uint32, C.POINTER(hpa_samples), C.POINTER(hpa_profile)]
        L.hpa_attribute_samples_host.argtypes = [H, C.c_uint32, C.POINTER(hpa_samples), C.POINTER(hpa_profile)]
        L.hpa_attribute_batch.argtypes = [H, C.c_uint32, u32p, C.POINTER(hpa_samples), C.POINTER(hpa_profile)]
        L.hpa_expand_gpucct.argtypes = [H, C.c_uint32, C.POINTER(hpa_gpucct), C.c_uint32, C.c_uint32,
                                         C.POINTER(hpa_cct_tree)]
        L.hpa_bottom_up_view.argtypes = [H, C.c_uint32, C.POINTER(hpa_profile), C.POINTER(hpa_cct_nodes),
                                         C.POINTER(hpa_bottom_up)]
        L.hpa_wait_flag.argtypes = [H, vp, C.c_uint32]
        L.hpa_unify_ccts.argtypes = [H, vp, C.c_uint32, C.POINTER(hpa_cct_unified)]
        L.hpa_build_cms.argtypes = [H, vp, C.c_uint32, C.POINTER(hpa_cms)]
        L.hpa_build_pms.argtypes = [H, vp, C.c_uint32, C.POINTER(hpa_pms)]
        L.hpa_flat_profile.argtypes = [H, C.c_uint32, C.POINTER(hpa_profile), C.POINTER(hpa_profile)]
        L.hpa_tune.argtypes = [H, C.c_uint32, C.POINTER(hpa_samples), C.POINTER(hpa_profile), C.c_uint32,
                               C.POINTER(hpa_options), vp]
        L.hpa_apportion_callgraph.argtypes = [H, C.c_uint32, C.POINTER(hpa_profile), C.POINTER(hpa_gpucct)]
        L.hpa_apportion_all.argtypes = [H, C.c_uint32, C.POINTER(hpa_profile), C.POINTER(hpa_gpucct_all)]
        L.hpa_issue_by_function.argtypes = [H, C.c_uint32, C.POINTER(hpa_profile), C.POINTER(hpa_issue_rows)]
        L.hpa_ratio_of_sums.argtypes = [H, C.c_uint32, C.POINTER(C.POINTER(hpa_profile)), C.c_uint32,
                                        C.POINTER(C.POINTER(hpa_profile)), C.c_uint32, C.POINTER(hpa_ratio_rows)]
        L.hpa_propagate_inclusive.argtypes = [H, C.c_uint32, C.POINTER(hpa_profile), C.POINTER(hpa_profile),
                                              C.POINTER(hpa_cct), vp]
        L.hpa_derive_metrics.argtypes = [H, C.POINTER(C.POINTER(hpa_profile)), C.c_uint32, C.POINTER(hpa_derived)]
        L.hpa_attribute_samples_noalloc.argtypes = [H, C.c_uint32, C.POINTER(hpa_samples), C.POINTER(hpa_profile)]
        L.hpa_set_phase_timing.argtypes = [H, C.c_int]
        L.hpa_server_create.argtypes = [H, C.POINTER(hpa_server_options), C.POINTER(vp)]
        L.hpa_server_submit.argtypes = [vp, C.c_uint32, C.POINTER(hpa_samples), C.POINTER(hpa_profile), u64p]
        L.hpa_server_poll.argtypes = [vp, C.c_uint64, C.c_int]
        L.hpa_server_stats_get.argtypes = [vp, C.POINTER(hpa_server_stats)]
        L.hpa_server_destroy.argtypes = [vp]
        L.hpa_phase_times.argtypes = [H, C.c_uint32, vp, u64p, u32p]
        for f in EXPORTS:
            if f not in ("hpa_last_error", "hpa_kernel_launches"):
                getattr(L, f).restype = C.c_int32
        _libs[checked] = L
    return _libs[checked]


class HpaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return C.c_void_p(t.data_ptr())
    return t.ctypes.data_as(C.c_void_p)


def _u32(t):
    return t.view(torch.int32) if t.dtype in (torch.int32, torch.uint32) else t.to(torch.int32)


@dataclass
class Profile:
    """Device-resident raw-metric profile (sorted unique keys)."""
    key_ctx: torch.Tensor    # int32 view of uint32
    key_node: torch.Tensor   # int32 view of uint32 (-1 = UNKNOWN)
    key_stall: torch.Tensor  # uint8
    val: torch.Tensor        # int64 view of uint64
    n_keys: torch.Tensor     # int64[1]
    total: torch.Tensor
    unknown: torch.Tensor
    n_ctx: int
    n_stall: int
    capacity: int
    n_nodes: int = 0

    def c(self) -> hpa_profile:
        return hpa_profile(self.capacity, _ptr(self.key_ctx), _ptr(self.key_node), _ptr(self.key_stall),
                           _ptr(self.val), _ptr(self.n_keys), _ptr(self.total), _ptr(self.unknown),
                           self.n_ctx, self.n_stall, self.n_nodes, 0)

    def count(self) -> int:
        return int(self.n_keys.item())

    def numpy(self):
        k = min(self.count(), self.capacity)
        return (self.key_ctx[:k].cpu().numpy().view(np.uint32), self.key_node[:k].cpu().numpy().view(np.uint32),
                self.key_stall[:k].cpu().numpy(), self.val[:k].cpu().numpy().view(np.uint64))

    def save(self, path: str):
        """Host dump of the sorted keys, totals and shape (.npz) -- a debugging
        aid; load_profile() puts it back on a device."""
        ctx, node, stall, val = self.numpy()
        np.savez(path, key_ctx=ctx, key_node=node, key_stall=stall, val=val,
                 total=self.total[: self.n_stall].cpu().numpy().view(np.uint64),
                 unknown=self.unknown[: self.n_stall].cpu().numpy().view(np.uint64),
                 shape=np.array([self.n_ctx, self.n_stall, self.n_nodes], np.int64))


def load_profile(path: str, device) -> Profile:
    """A profile written by Profile.save, on `device`."""
    z = np.load(path)
    n_ctx, n_stall, n_nodes = (int(x) for x in z["shape"])
    k = int(z["val"].shape[0])
    p = new_profile(max(1, k), n_stall, device)
    if k:
        p.key_ctx[:k] = torch.from_numpy(z["key_ctx"].view(np.int32))
        p.key_node[:k] = torch.from_numpy(z["key_node"].view(np.int32))
        p.key_stall[:k] = torch.from_numpy(z["key_stall"])
        p.val[:k] = torch.from_numpy(z["val"].view(np.int64))
    p.n_keys.fill_(k)
    p.total[:n_stall] = torch.from_numpy(z["total"].view(np.int64))
    p.unknown[:n_stall] = torch.from_numpy(z["unknown"].view(np.int64))
    p.n_ctx, p.n_nodes = n_ctx, n_nodes
    return p


def new_profile(capacity: int, n_stall: int, device) -> Profile:
    cap = max(1, int(capacity))
    z = lambda n, dt: torch.empty(n, dtype=dt, device=device)
    return Profile(z(cap, torch.int32), z(cap, torch.int32), z(cap, torch.uint8), z(cap, torch.int64),
                   torch.zeros(1, dtype=torch.int64, device=device), torch.zeros(HPA_MAX_STALL, dtype=torch.int64, device=device),
                   torch.zeros(HPA_MAX_STALL, dtype=torch.int64, device=device), 0, n_stall, cap)


def _structure(b):
    """hpa_structure over host copies of b's tables (returned to keep them alive)."""
    arrs = dict(
        range_lo=np.ascontiguousarray(b.range_lo, np.uint64), range_hi=np.ascontiguousarray(b.range_hi, np.uint64),
        range_node=np.ascontiguousarray(b.range_node, np.uint32),
        node_parent=np.ascontiguousarray(b.node_parent, np.uint32),
        node_kind=np.ascontiguousarray(b.node_kind, np.uint8), node_func=np.ascontiguousarray(b.node_func, np.uint32),
        cs_caller=np.ascontiguousarray(b.cs_caller, np.uint32), cs_callee=np.ascontiguousarray(b.cs_callee, np.uint32),
        cs_node=np.ascontiguousarray(b.cs_node, np.uint32))
    s = hpa_structure(arrs["range_lo"].shape[0], _ptr(arrs["range_lo"]), _ptr(arrs["range_hi"]),
                      _ptr(arrs["range_node"]), arrs["node_parent"].shape[0], _ptr(arrs["node_parent"]),
                      _ptr(arrs["node_kind"]), _ptr(arrs["node_func"]), int(b.n_funcs), arrs["cs_caller"].shape[0],
                      _ptr(arrs["cs_caller"]), _ptr(arrs["cs_callee"]), _ptr(arrs["cs_node"]))
    return s, arrs


def validate_structure(b):
    """hpa_validate_structure: (status, reason) of b's tables, on the host."""
    L = lib()
    s, _keep = _structure(b)
    msg = C.create_string_buffer(256)
    st = int(L.hpa_validate_structure(C.byref(s), msg, C.c_size_t(256)))
    return st, msg.value.decode()


class Hpa:
    """One library handle bound to a CUDA device and stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None, issued_mask: int = 1,
                 leaf_capacity: int = 0, cursor_shift: int | None = None,
                 sort_mode: int | None = None, partition: bool = True, small_leaves: int = 0,
                 leaf_hash: int = 0, timeout_iters: int = 0, leaf_emit: int = 0, checked: bool | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("hpa needs a CUDA device; there is no CPU implementation")
        self.L = lib(checked=checked)
        self.device = torch.device("cuda", device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.h = C.c_void_p()
        opt = hpa_options(issued_mask, leaf_capacity, timeout_iters)
        if cursor_shift is not None:
            opt.cursor_pad = cursor_shift + 1
        if sort_mode is not None:
            opt.leaf_ranking = sort_mode
        if not partition:
            opt.grouping = 1
        opt.small_leaves = small_leaves
        opt.leaf_hash = leaf_hash
        opt.leaf_emit = leaf_emit
        st = self.L.hpa_create(C.byref(self.h), device, C.c_void_p(self.stream.cuda_stream), C.byref(opt))
        if st:
            raise HpaError(st, "hpa_create failed")
        self._keep = []
        self._depth = {}

    def close(self):
        if self.h:
            self.L.hpa_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st):
        if st:
            raise HpaError(st, self.L.hpa_last_error(self.h).decode())

    def sync(self):
        bad = C.c_uint64(0)
        st = self.L.hpa_sync(self.h, C.byref(bad))
        if st:
            raise HpaError(st, self.L.hpa_last_error(self.h).decode())
        return int(bad.value)

    def sync_status(self):
        """(status, bad) without raising."""
        bad = C.c_uint64(0)
        st = self.L.hpa_sync(self.h, C.byref(bad))
        return int(st), int(bad.value)

    def wait_flag(self, flag: torch.Tensor, value: int):
        """hpa_wait_flag: the handle's stream waits (bounded) for flag[0] == value."""
        self.check(self.L.hpa_wait_flag(self.h, _ptr(flag), C.c_uint32(value)))

    def launches(self) -> int:
        return int(self.L.hpa_kernel_launches(self.h))

    def set_phase_timing(self, on: bool):
        self.check(self.L.hpa_set_phase_timing(self.h, 1 if on else 0))

    def phase_times(self):
        """{phase name: total ms} and the number of timed calls."""
        ms = np.zeros(8, np.float64)
        calls = C.c_uint64()
        n = C.c_uint32()
        self.check(self.L.hpa_phase_times(self.h, 8, _ptr(ms), C.byref(calls), C.byref(n)))
        return {PHASES[i]: float(ms[i]) for i in range(n.value)}, int(calls.value)

    def reserve(self, max_samples: int, max_groups: int):
        self.check(self.L.hpa_reserve(self.h, max_samples, max_groups))

    # ---- structure
    def load_structure(self, b) -> int:
        """b: an object with numpy arrays range_lo/hi/node, node_parent/kind/func, cs_* (see synth.Binary)."""
        s, arrs = _structure(b)
        bid = C.c_uint32(0)
        self.check(self.L.hpa_load_structure(self.h, C.byref(s), C.byref(bid)))
        # the structure-tree depth (computed by the library at load) bounds the inclusive expansion
        info = hpa_binary_info()
        self.check(self.L.hpa_binary_info_get(self.h, bid, C.byref(info), None))
        self._depth[int(bid.value)] = int(info.max_depth)
        return int(bid.value)

    def unload_structure(self, bid: int):
        self.check(self.L.hpa_unload_structure(self.h, bid))

    def binary_info(self, bid: int):
        info = hpa_binary_info()
        F = C.c_uint32()
        self.check(self.L.hpa_binary_info_get(self.h, bid, C.byref(info), None))
        cof = np.zeros(info.n_funcs, np.uint32)
        self.check(self.L.hpa_binary_info_get(self.h, bid, C.byref(info), _ptr(cof)))
        return info, cof

    # ---- samples
    @staticmethod
    def samples_c(pc, ctx, stall, count, n_ctx, n_stall) -> hpa_samples:
        return hpa_samples(int(pc.shape[0]), _ptr(pc), _ptr(ctx), _ptr(stall), _ptr(count), int(n_ctx), int(n_stall))

    def attribute_samples(self, bid: int, s, out: Profile | None = None, capacity: int | None = None) -> Profile:
        """s: synth.Samples-like with device tensors pc (int64), ctx (int32), stall (uint8), count (int32|None)."""
        if out is None:
            out = new_profile(s.n if capacity is None else capacity, s.n_stall, self.device)
        ci = self.samples_c(s.pc, s.ctx, s.stall, s.count, s.n_ctx, s.n_stall)
        co = out.c()
        self.check(self.L.hpa_attribute_samples(self.h, bid, C.byref(ci), C.byref(co)))
        out.n_ctx, out.n_stall, out.n_nodes = s.n_ctx, s.n_stall, co.n_nodes
        return out

    def attribute_samples_noalloc(self, bid: int, s, out: Profile) -> Profile:
        """hpa_attribute_samples_noalloc: no device allocation during the call (static scratch)."""
        ci = self.samples_c(s.pc, s.ctx, s.stall, s.count, s.n_ctx, s.n_stall)
        co = out.c()
        self.check(self.L.hpa_attribute_samples_noalloc(self.h, bid, C.byref(ci), C.byref(co)))
        out.n_ctx, out.n_stall, out.n_nodes = s.n_ctx, s.n_stall, co.n_nodes
        return out

    def attribute_samples_host(self, bid: int, pc, ctx, stall, count, n_ctx, n_stall, capacity=None, out=None):
        """Host arrays in, host arrays out (numpy arrays or CPU tensors, pinned for full speed).
        out: optional dict of preallocated host arrays ctx, node, stall, val, n, total, unknown."""
        n = int(pc.shape[0])
        cap = n if capacity is None else capacity
        if out is None:
            out = dict(ctx=np.empty(cap, np.uint32), node=np.empty(cap, np.uint32), stall=np.empty(cap, np.uint8),
                       val=np.empty(cap, np.uint64), n=np.zeros(1, np.uint64), total=np.zeros(HPA_MAX_STALL, np.uint64),
                       unknown=np.zeros(HPA_MAX_STALL, np.uint64))
        ci = self.samples_c(pc, ctx, stall, count, n_ctx, n_stall)
        co = hpa_profile(cap, _ptr(out["ctx"]), _ptr(out["node"]), _ptr(out["stall"]), _ptr(out["val"]),
                         _ptr(out["n"]), _ptr(out["total"]), _ptr(out["unknown"]), 0, 0)
        self.check(self.L.hpa_attribute_samples_host(self.h, bid, C.byref(ci), C.byref(co)))
        return out

    def propagate_inclusive(self, bid: int, p: Profile, tree: bool = True, cct_parent: torch.Tensor | None = None,
                            tree_capacity: int | None = None):
        """Inclusive metrics (Section 6.1).  Returns (tree Profile or None, cct tensor [n_cct, n_stall] or None).
        The input profile's key count bounds the expansion, so it is read first."""
        k = p.count()
        pin = p.c()
        pin.capacity = k
        tree_out = None
        tc = None
        if tree:
            info, _ = self.binary_info(bid)
            cap = tree_capacity if tree_capacity is not None else max(1, k * (self.max_depth(bid) + 1))
            tree_out = new_profile(cap, p.n_stall, self.device)
            tc = tree_out.c()
        cct_out = None
        cc = None
        if cct_parent is not None:
            n = int(cct_parent.shape[0])
            cct_out = torch.empty((n, p.n_stall), dtype=torch.int64, device=self.device)
            cc = hpa_cct(n, _ptr(cct_parent))
        self.check(self.L.hpa_propagate_inclusive(self.h, bid, C.byref(pin), C.byref(tc) if tc is not None else None,
                                                  C.byref(cc) if cc is not None else None,
                                                  _ptr(cct_out) if cct_out is not None else None))
        if tree_out is not None:
            tree_out.n_ctx, tree_out.n_stall, tree_out.n_nodes = p.n_ctx, p.n_stall, p.n_nodes
        return tree_out, cct_out

    def apportion_callgraph(self, bid: int, p: Profile, req_ctx):
        """GPU calling context trees (Section 6.3) of the requested contexts.
        Returns (incl [n_req, V, S+1] f32, a [n_req, E, S+1] f32, flags [n_req, E] u8)."""
        info, _ = self.binary_info(bid)
        req = torch.as_tensor(np.asarray(req_ctx, np.uint32).view(np.int32), device=self.device)
        n = int(req.shape[0])
        M = p.n_stall + 1
        incl = torch.empty((n, info.n_cnodes, M), dtype=torch.float32, device=self.device)
        a = torch.empty((n, info.n_calls, M), dtype=torch.float32, device=self.device)
        flags = torch.empty((n, info.n_calls), dtype=torch.uint8, device=self.device)
        g = hpa_gpucct(n, _ptr(req), _ptr(incl), _ptr(a), _ptr(flags))
        pc = p.c()
        self.check(self.L.hpa_apportion_callgraph(self.h, bid, C.byref(pc), C.byref(g)))
        self._keep = [req]
        return incl, a, flags

    def apportion_all(self, bid: int, p: Profile, shares: bool = False, caps=None, out=None):
        """hpa_apportion_all: GPU calling context trees of every context of p as
        sparse rows.  Two calls: the first (capacities 0) asks for the row
        counts, the second fills arrays of that size (caps=(nodes, edges) skips
        the first).  Returns a dict of device tensors: node_off, node_id,
        incl [rows, S+1], edge_off, edge_id, ratio, flags, a (with shares) and
        counts."""
        d = self.device
        M = p.n_stall + 1
        pc = p.c()
        if out is not None:                        # the arrays of an earlier call, reused
            shares = out["a"] is not None
            g = hpa_gpucct_all(out["caps"][0], out["caps"][1], _ptr(out["node_off"]), _ptr(out["node_id"]),
                               _ptr(out["incl"]), _ptr(out["edge_off"]), _ptr(out["edge_id"]), _ptr(out["ratio"]),
                               _ptr(out["a"]) if shares else None, _ptr(out["flags"]), _ptr(out["counts"]))
            self.check(self.L.hpa_apportion_all(self.h, bid, C.byref(pc), C.byref(g)))
            return out
        counts = torch.zeros(2, dtype=torch.int64, device=d)
        if caps is None:
            g = hpa_gpucct_all(0, 0, None, None, None, None, None, None, None, None, _ptr(counts))
            self.check(self.L.hpa_apportion_all(self.h, bid, C.byref(pc), C.byref(g)))
            self.sync()
            caps = tuple(int(x) for x in counts.tolist())
        cn, ce = caps
        out = dict(node_off=torch.empty(p.n_ctx + 1, dtype=torch.int64, device=d),
                   node_id=torch.empty(max(cn, 1), dtype=torch.int32, device=d),
                   incl=torch.empty((max(cn, 1), M), dtype=torch.float32, device=d),
                   edge_off=torch.empty(p.n_ctx + 1, dtype=torch.int64, device=d),
                   edge_id=torch.empty(max(ce, 1), dtype=torch.int32, device=d),
                   ratio=torch.empty(max(ce, 1), dtype=torch.float32, device=d),
                   flags=torch.empty(max(ce, 1), dtype=torch.uint8, device=d),
                   a=torch.empty((max(ce, 1), M), dtype=torch.float32, device=d) if shares else None,
                   counts=counts, caps=(cn, ce))
        g = hpa_gpucct_all(cn, ce, _ptr(out["node_off"]), _ptr(out["node_id"]), _ptr(out["incl"]),
                           _ptr(out["edge_off"]), _ptr(out["edge_id"]), _ptr(out["ratio"]),
                           _ptr(out["a"]) if shares else None, _ptr(out["flags"]), _ptr(counts))
        self.check(self.L.hpa_apportion_all(self.h, bid, C.byref(pc), C.byref(g)))
        return out

    def issue_by_function(self, bid: int, p: Profile, capacity: int | None = None):
        """hpa_issue_by_function: warp issue rate and stall shares per (context,
        function).  Returns a dict of device tensors (ctx, func, S, S_issued,
        W, frac [rows, S], n_rows); capacity defaults to the key count."""
        d = self.device
        cap = p.capacity if capacity is None else capacity
        out = dict(ctx=torch.empty(max(cap, 1), dtype=torch.int32, device=d),
                   func=torch.empty(max(cap, 1), dtype=torch.int32, device=d),
                   S=torch.empty(max(cap, 1), dtype=torch.int64, device=d),
                   S_issued=torch.empty(max(cap, 1), dtype=torch.int64, device=d),
                   W=torch.empty(max(cap, 1), dtype=torch.float32, device=d),
                   frac=torch.empty((max(cap, 1), p.n_stall), dtype=torch.float32, device=d),
                   n_rows=torch.zeros(1, dtype=torch.int64, device=d))
        o = hpa_issue_rows(cap, *[_ptr(out[k]) for k in ("ctx", "func", "S", "S_issued", "W", "frac", "n_rows")])
        pc = p.c()
        self.check(self.L.hpa_issue_by_function(self.h, bid, C.byref(pc), C.byref(o)))
        return out

    def expand_gpucct(self, bid: int, res, req_ctx, n_stall: int, q: int, budget: int):
        """hpa_expand_gpucct on an apportion_callgraph result `res` = (incl, a, flags)
        for the requested contexts req_ctx: context q's GPU CCT as a tree."""
        incl, a, flags = res
        req = torch.as_tensor(np.asarray(req_ctx, np.uint32).view(np.int32), device=self.device)
        g = hpa_gpucct(int(req.shape[0]), _ptr(req), _ptr(incl), _ptr(a), _ptr(flags))
        d = self.device
        out = dict(parent=torch.empty(budget, dtype=torch.int32, device=d), cnode=torch.empty(budget, dtype=torch.int32, device=d),
                   edge=torch.empty(budget, dtype=torch.int32, device=d), scale=torch.empty(budget, dtype=torch.float32, device=d),
                   incl=torch.empty((budget, n_stall + 1), dtype=torch.float32, device=d),
                   n=torch.zeros(1, dtype=torch.int64, device=d), truncated=torch.zeros(1, dtype=torch.int32, device=d))
        t = hpa_cct_tree(budget, _ptr(out["parent"]), _ptr(out["cnode"]), _ptr(out["edge"]), _ptr(out["scale"]),
                         _ptr(out["incl"]), _ptr(out["n"]), _ptr(out["truncated"]))
        self.check(self.L.hpa_expand_gpucct(self.h, bid, C.byref(g), n_stall, q, C.byref(t)))
        self._keep = [req]
        return out

    def bottom_up(self, bid: int, p: Profile, cct, levels: int, cap_nodes: int | None = None,
                  cap_values: int | None = None):
        """hpa_bottom_up_view: cct = (parent, module, offset) device tensors
        (int32 / int16 / int64).  Without capacities, a first call sizes the
        output.  Returns the node arrays, level_off, the (node, stall, val)
        values and the counts tensor (nodes, values needed)."""
        d = self.device
        pin = p.c()
        pin.capacity = max(1, p.count())
        desc = hpa_cct_nodes(int(cct[0].shape[0]), _ptr(cct[0]), _ptr(cct[1]), _ptr(cct[2]))
        if cap_nodes is None or cap_values is None:
            counts = torch.zeros(2, dtype=torch.int64, device=d)
            o = hpa_bottom_up(levels, 0, 0, None, None, None, None, None, None, None, None, _ptr(counts))
            self.check(self.L.hpa_bottom_up_view(self.h, bid, C.byref(pin), C.byref(desc), C.byref(o)))
            st, _ = self.sync_status()
            if st not in (HPA_OK, HPA_E_CAPACITY):
                raise HpaError(st, self.L.hpa_last_error(self.h).decode())
            n = counts.tolist()
            cap_nodes = n[0] if cap_nodes is None else cap_nodes
            cap_values = n[1] if cap_values is None else cap_values
        e = lambda n, dt: torch.empty(max(1, n), dtype=dt, device=d)
        out = dict(parent=e(cap_nodes, torch.int32), func=e(cap_nodes, torch.int32), module=e(cap_nodes, torch.int16),
                   offset=e(cap_nodes, torch.int64), level_off=e(levels + 2, torch.int64),
                   val_node=e(cap_values, torch.int32), val_stall=e(cap_values, torch.uint8),
                   val=e(cap_values, torch.int64), counts=torch.zeros(2, dtype=torch.int64, device=d))
        o = hpa_bottom_up(levels, cap_nodes, cap_values, *[_ptr(out[k]) for k in
                          ("parent", "func", "module", "offset", "level_off", "val_node", "val_stall", "val", "counts")])
        self.check(self.L.hpa_bottom_up_view(self.h, bid, C.byref(pin), C.byref(desc), C.byref(o)))
        self._keep = [p, cct, out]
        return out

    def unify_ccts(self, ccts, capacity: int | None = None):
        """hpa_unify_ccts: ccts = [(parent, module, offset)] device tensors per
        profile (int32 / int16 / int64).  Returns uid per input node and the
        merged tree's parent / module / offset and size."""
        N = sum(int(c[0].shape[0]) for c in ccts)
        cap = N if capacity is None else capacity
        d = self.device
        out = dict(uid=torch.empty(N, dtype=torch.int32, device=d), parent=torch.empty(cap, dtype=torch.int32, device=d),
                   module=torch.empty(cap, dtype=torch.int16, device=d), offset=torch.empty(cap, dtype=torch.int64, device=d),
                   n=torch.zeros(1, dtype=torch.int64, device=d))
        desc = (hpa_cct_nodes * len(ccts))(*[hpa_cct_nodes(int(c[0].shape[0]), _ptr(c[0]), _ptr(c[1]), _ptr(c[2]))
                                             for c in ccts])
        o = hpa_cct_unified(cap, _ptr(out["uid"]), _ptr(out["parent"]), _ptr(out["module"]), _ptr(out["offset"]),
                            _ptr(out["n"]))
        self.check(self.L.hpa_unify_ccts(self.h, desc, len(ccts), C.byref(o)))
        self._keep = [ccts, desc]
        return out

    def _profile_array(self, profiles):
        cps = [p.c() for p in profiles]
        for c, p in zip(cps, profiles):
            c.capacity = p.count()
        return cps, (C.POINTER(hpa_profile) * len(cps))(*[C.pointer(c) for c in cps])

    def build_cms(self, profiles):
        """hpa_build_cms: context-major sparse layout (Section 6.2) of the profiles."""
        total = sum(p.count() for p in profiles)
        d, n = self.device, max(1, total)
        t = lambda m, dt: torch.empty(m, dtype=dt, device=d)
        out = dict(plane_ctx=t(n, torch.int32), plane_node=t(n, torch.int32), plane_off=t(n + 1, torch.int64),
                   metric_id=t(n, torch.uint8), metric_off=t(n + 1, torch.int64), pid=t(n, torch.int32),
                   val=t(n, torch.int64), counts=torch.zeros(3, dtype=torch.int64, device=d))
        o = hpa_cms(n, n, n, *[_ptr(out[k]) for k in ("plane_ctx", "plane_node", "plane_off", "metric_id",
                                                        "metric_off", "pid", "val", "counts")])
        cps, arr = self._profile_array(profiles)
        self.check(self.L.hpa_build_cms(self.h, arr, len(cps), C.byref(o)))
        self._keep = [cps, arr]
        return out

    def build_pms(self, profiles):
        """hpa_build_pms: profile-major sparse layout (Section 6.2) of the profiles."""
        total = sum(p.count() for p in profiles)
        d, n = self.device, max(1, total)
        t = lambda m, dt: torch.empty(m, dtype=dt, device=d)
        out = dict(prof_off=t(len(profiles) + 1, torch.int64), plane_ctx=t(n, torch.int32), plane_node=t(n, torch.int32),
                   plane_off=t(n + 1, torch.int64), metric_id=t(n, torch.uint8), val=t(n, torch.int64),
                   counts=torch.zeros(2, dtype=torch.int64, device=d))
        o = hpa_pms(n, n, *[_ptr(out[k]) for k in ("prof_off", "plane_ctx", "plane_node", "plane_off", "metric_id",
                                                    "val", "counts")])
        cps, arr = self._profile_array(profiles)
        self.check(self.L.hpa_build_pms(self.h, arr, len(cps), C.byref(o)))
        self._keep = [cps, arr]
        return out

    def flat_profile(self, bid: int, p: Profile, capacity: int | None = None) -> Profile:
        """hpa_flat_profile: the profile summed over contexts, keys (0, node, stall)."""
        k = p.count()
        pin = p.c()
        pin.capacity = k
        out = new_profile(max(1, k if capacity is None else capacity), p.n_stall, self.device)
        co = out.c()
        self.check(self.L.hpa_flat_profile(self.h, bid, C.byref(pin), C.byref(co)))
        out.n_ctx, out.n_stall, out.n_nodes = 1, p.n_stall, co.n_nodes
        return out

    def derive_metrics(self, profiles, n_ctx: int | None = None, capacity: int | None = None):
        """Cross-profile statistics (Section 4.5) and per-context warp issue rate (Section 7)."""
        P = len(profiles)
        n_ctx = n_ctx or max(p.n_ctx for p in profiles)
        S = max(p.n_stall for p in profiles)
        cap = capacity if capacity is not None else max(1, sum(p.count() for p in profiles))
        d = self.device
        out = dict(ctx=torch.empty(cap, dtype=torch.int32, device=d), node=torch.empty(cap, dtype=torch.int32, device=d),
                   stall=torch.empty(cap, dtype=torch.uint8, device=d), sum=torch.empty(cap, dtype=torch.int64, device=d),
                   min=torch.empty(cap, dtype=torch.int64, device=d), max=torch.empty(cap, dtype=torch.int64, device=d),
                   mean=torch.empty(cap, dtype=torch.float32, device=d), std=torch.empty(cap, dtype=torch.float32, device=d),
                   cov=torch.empty(cap, dtype=torch.float32, device=d), n=torch.zeros(1, dtype=torch.int64, device=d),
                   S=torch.empty(n_ctx, dtype=torch.int64, device=d), S_issued=torch.empty(n_ctx, dtype=torch.int64, device=d),
                   W=torch.empty(n_ctx, dtype=torch.float32, device=d),
                   frac=torch.empty((n_ctx, S), dtype=torch.float32, device=d))
        o = hpa_derived(cap, _ptr(out["ctx"]), _ptr(out["node"]), _ptr(out["stall"]), _ptr(out["sum"]),
                        _ptr(out["min"]), _ptr(out["max"]), _ptr(out["mean"]), _ptr(out["std"]), _ptr(out["cov"]),
                        _ptr(out["n"]), n_ctx, _ptr(out["S"]), _ptr(out["S_issued"]), _ptr(out["W"]), _ptr(out["frac"]))
        cps = [p.c() for p in profiles]
        for c, p in zip(cps, profiles):
            c.capacity = p.count()
        arr = (C.POINTER(hpa_profile) * P)(*[C.pointer(c) for c in cps])
        self.check(self.L.hpa_derive_metrics(self.h, arr, P, C.byref(o)))
        self._keep = [cps, arr]
        return out

    def ratio_of_sums(self, bid: int, num, den, capacity: int | None = None):
        """hpa_ratio_of_sums: per key, the numerator profiles' sum over the
        denominator profiles' sum (Section 4.5).  Returns a dict of device
        tensors (ctx, node, stall, num, den, ratio, n); capacity defaults to
        the profiles' key counts added up."""
        num, den = list(num), list(den)
        cap = capacity if capacity is not None else max(1, sum(p.count() for p in num + den))
        d = self.device
        out = dict(ctx=torch.empty(cap, dtype=torch.int32, device=d), node=torch.empty(cap, dtype=torch.int32, device=d),
                   stall=torch.empty(cap, dtype=torch.uint8, device=d), num=torch.empty(cap, dtype=torch.int64, device=d),
                   den=torch.empty(cap, dtype=torch.int64, device=d), ratio=torch.empty(cap, dtype=torch.float32, device=d),
                   n=torch.zeros(1, dtype=torch.int64, device=d))
        o = hpa_ratio_rows(cap, *[_ptr(out[k]) for k in ("ctx", "node", "stall", "num", "den", "ratio", "n")])
        groups = []
        for ps in (num, den):
            cps = [p.c() for p in ps]
            for c, p in zip(cps, ps):
                c.capacity = p.count()
            groups.append((cps, (C.POINTER(hpa_profile) * max(1, len(cps)))(*[C.pointer(c) for c in cps])))
        self.check(self.L.hpa_ratio_of_sums(self.h, bid, groups[0][1], len(num), groups[1][1], len(den), C.byref(o)))
        self._keep = groups
        return out

    def max_depth(self, bid: int) -> int:
        return self._depth.get(bid, 16)

    def tune(self, bid: int, s, out: Profile | None = None, reps: int = 2):
        """hpa_tune: time every candidate configuration on this buffer and keep
        the fastest for the calls that follow.  Returns (chosen options as a
        dict, per-candidate ms)."""
        if out is None:
            out = new_profile(s.n, s.n_stall, self.device)
        ci = self.samples_c(s.pc, s.ctx, s.stall, s.count, s.n_ctx, s.n_stall)
        co = out.c()
        best = hpa_options()
        ms = np.zeros(HPA_TUNE_CANDIDATES, np.float32)
        self.check(self.L.hpa_tune(self.h, bid, C.byref(ci), C.byref(co), reps, C.byref(best), _ptr(ms)))
        chosen = {"leaf_capacity": best.leaf_capacity, "grouping": best.grouping, "leaf_hash": best.leaf_hash,
                  "leaf_ranking": best.leaf_ranking}
        return chosen, ms.tolist()

    def attribute_batch(self, bids, samples, outs=None):
        n = len(samples)
        if outs is None:
            outs = [new_profile(s.n, s.n_stall, self.device) for s in samples]
        ins = (hpa_samples * n)(*[self.samples_c(s.pc, s.ctx, s.stall, s.count, s.n_ctx, s.n_stall) for s in samples])
        cos = (hpa_profile * n)(*[o.c() for o in outs])
        ids = (C.c_uint32 * n)(*bids)
        self.check(self.L.hpa_attribute_batch(self.h, n, ids, ins, cos))
        for o, s, c in zip(outs, samples, cos):
            o.n_ctx, o.n_stall, o.n_nodes = s.n_ctx, s.n_stall, c.n_nodes
        return outs


class Server:
    """Request loop over host sample buffers (hpa_server_*)."""

    def __init__(self, h: Hpa, mem_cap_bytes: int = 0, max_batch: int = 0, max_inflight: int = 0):
        self.h = h
        self.s = C.c_void_p()
        opt = hpa_server_options(mem_cap_bytes, max_batch, max_inflight)
        h.check(h.L.hpa_server_create(h.h, C.byref(opt), C.byref(self.s)))
        self._live = {}

    def submit(self, bid: int, pc, ctx, stall, count, n_ctx: int, n_stall: int, capacity: int | None = None,
               out: dict | None = None):
        """Host arrays (pinned CPU tensors for full speed).  Returns a ticket; the
        result lands in self.result(ticket) once poll() reports completion.
        out: optional preallocated host arrays ctx, node, stall, val (capacity
        entries each), n (1), total and unknown (HPA_MAX_STALL each)."""
        n = int(pc.shape[0])
        if out is None:
            cap = max(1, n if capacity is None else capacity)
            out = dict(ctx=torch.empty(cap, dtype=torch.int32).pin_memory(),
                       node=torch.empty(cap, dtype=torch.int32).pin_memory(),
                       stall=torch.empty(cap, dtype=torch.uint8).pin_memory(),
                       val=torch.empty(cap, dtype=torch.int64).pin_memory(),
                       n=torch.zeros(1, dtype=torch.int64), total=torch.zeros(HPA_MAX_STALL, dtype=torch.int64).pin_memory(),
                       unknown=torch.zeros(HPA_MAX_STALL, dtype=torch.int64).pin_memory())
        else:
            cap = int(out["ctx"].shape[0])
        ci = Hpa.samples_c(pc, ctx, stall, count, n_ctx, n_stall)
        co = hpa_profile(cap, _ptr(out["ctx"]), _ptr(out["node"]), _ptr(out["stall"]), _ptr(out["val"]),
                         _ptr(out["n"]), _ptr(out["total"]), _ptr(out["unknown"]), 0, 0, 0, 0)
        t = C.c_uint64()
        self.h.check(self.h.L.hpa_server_submit(self.s, bid, C.byref(ci), C.byref(co), C.byref(t)))
        self._live[t.value] = (out, (pc, ctx, stall, count))
        return int(t.value)

    def poll(self, ticket: int, wait_ms: int = 0) -> int:
        return int(self.h.L.hpa_server_poll(self.s, ticket, wait_ms))

    def result(self, ticket: int):
        out, _ = self._live.pop(ticket)
        return out

    def stats(self):
        st = hpa_server_stats()
        self.h.check(self.h.L.hpa_server_stats_get(self.s, C.byref(st)))
        return {f: getattr(st, f) for f, _ in hpa_server_stats._fields_}

    def close(self):
        if self.s:
            self.h.L.hpa_server_destroy(self.s)
            self.s = C.c_void_p()
