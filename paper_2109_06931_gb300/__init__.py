"""GPU PC-sample analysis on GB300: a CUDA library (libhpa.so, C ABI in
include/hpa.h) and its Python binding (paper_2109_06931_gb300.hpa).

Operations follow "Measurement and Analysis of GPU-accelerated Applications
with HPCToolkit" (arXiv 2109.06931): attribution of PC samples to program
structure (Sections 4.2, 5), raw-metric aggregation (Section 4.5), the
approximate GPU calling context tree (Section 6.3), inclusive propagation
(Section 6.1) and derived metrics (Sections 4.5, 7).
"""
from . import build  # noqa: F401
