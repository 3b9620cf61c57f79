"""GB300-native online solver of the nested polarized-traces method for the
2D Helmholtz equation (Zepeda-Nunez & Demanet, arXiv 1510.01831).

The numerical path is libhz (CUDA, sm_103a) behind the C ABI of
include/hz.h; this package holds its build script and a thin ctypes binding
(``paper_1510_01831_gb300.hz``) with the same entry-point names.  PyTorch is
used only for device memory when a context is created with
``device_ptrs=True``.
"""
from .build import build as build_lib  # noqa: F401

__all__ = ["build_lib"]
