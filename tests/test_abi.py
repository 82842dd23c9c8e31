"""The C-ABI library builds, loads without a GPU, and exports every entry
point declared in include/hpa.h; the binding refuses to run without CUDA."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "hpa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hpa_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ["hpa_load_structure", "hpa_attribute_samples", "hpa_apportion_callgraph",
                 "hpa_propagate_inclusive", "hpa_derive_metrics", "hpa_attribute_batch", "hpa_sync"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2109_06931_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (hpa_[a-z_]+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_bounds_checked_flavour_exports_the_same_symbols():
    """libhpa_checked.so (-DHPA_CHECKED) is the same boundary with index
    checks compiled in; hpa_build_flags tells the two apart."""
    from paper_2109_06931_gb300 import build
    from paper_2109_06931_gb300 import hpa as H
    lib = build.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (hpa_[a-z_]+)", out))
    assert not [n for n in declared() if n not in exported]
    assert H.lib(checked=True).hpa_build_flags() == H.HPA_BUILD_CHECKED
    assert H.lib(checked=False).hpa_build_flags() == 0


def test_library_loads_and_binding_types():
    import ctypes
    from paper_2109_06931_gb300 import hpa as H
    L = H.lib()
    for n in declared():
        assert hasattr(L, n)
    # without a device the handle cannot be created, and the binding says so
    import torch
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        assert L.hpa_create(ctypes.byref(h), 0, None, None) == H.HPA_E_CUDA
        with pytest.raises(RuntimeError):
            H.Hpa(0)


@pytest.mark.parametrize("field,value", [("leaf_capacity", 5000), ("leaf_ranking", 4), ("grouping", 2),
                                         ("cursor_pad", 8), ("small_leaves", 3), ("leaf_hash", 2),
                                         ("leaf_emit", 2)])
def test_create_rejects_invalid_options(field, value):
    """Option checks come before any device call, so they hold without a GPU."""
    import ctypes
    from paper_2109_06931_gb300 import hpa as H
    L = H.lib()
    opt = H.hpa_options()
    setattr(opt, field, value)
    h = ctypes.c_void_p()
    assert L.hpa_create(ctypes.byref(h), 0, None, ctypes.byref(opt)) == H.HPA_E_INVALID_ARG
    assert not h.value


def test_struct_layouts_match_header():
    """ctypes mirrors of the C structs have the sizes the C compiler gives."""
    import ctypes
    from paper_2109_06931_gb300 import hpa as H
    src = r'''
#include <stdio.h>
#include "hpa.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(hpa_options), sizeof(hpa_structure), sizeof(hpa_samples),
         sizeof(hpa_profile), sizeof(hpa_gpucct), sizeof(hpa_cct), sizeof(hpa_derived), sizeof(hpa_binary_info),
         sizeof(hpa_gpucct_all), sizeof(hpa_issue_rows), sizeof(hpa_ratio_rows));
  return 0;
}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    mine = [ctypes.sizeof(t) for t in (H.hpa_options, H.hpa_structure, H.hpa_samples, H.hpa_profile, H.hpa_gpucct,
                                       H.hpa_cct, H.hpa_derived, H.hpa_binary_info, H.hpa_gpucct_all, H.hpa_issue_rows,
                                       H.hpa_ratio_rows)]
    assert sizes == mine
