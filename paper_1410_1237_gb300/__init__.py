"""GB300 implementation of the parallel Louvain method of arXiv 1410.1237.

The computation lives in ``liblv.so`` (CUDA for sm_103a, C ABI declared in
``include/lv.h``); :mod:`paper_1410_1237_gb300.lv` is its ctypes binding.
"""
from . import lv  # noqa: F401
from .lv import LVError, Result, make_params, run  # noqa: F401

__all__ = ["lv", "run", "make_params", "LVError", "Result"]
