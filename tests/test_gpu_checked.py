"""The bounds-checked build (libhpa_checked.so, -DHPA_CHECKED): every index
that a kernel computes from counters, scans or data is checked against the
array it indexes, and a violation makes the call fail with HPA_E_INTERNAL
instead of touching memory out of range.  The GPU parity suites of the hot
path run again, in a child process, against that build; they pass only if
no check fires and every result still equals the oracle's."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SUITES = ["tests/test_gpu_attribution.py", "tests/test_gpu_derive.py", "tests/test_gpu_gpucct.py",
          "tests/test_gpu_inclusive.py", "tests/test_zz_no_alloc.py"]


def test_checked_flavour_is_the_one_loaded():
    from paper_2109_06931_gb300 import hpa
    assert hpa.lib(checked=True).hpa_build_flags() & hpa.HPA_BUILD_CHECKED
    assert not hpa.lib(checked=False).hpa_build_flags() & hpa.HPA_BUILD_CHECKED


def test_parity_suites_under_bounds_checks():
    from paper_2109_06931_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, HPA_CHECKED="1")
    # the headline-regime case spends most of its time in the oracle: the
    # other cases cover the same kernels
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-k", "not headline", "-p",
                        "no:cacheprovider"] + SUITES, cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
