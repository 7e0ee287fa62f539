"""GB300-native Fullwave 2 time stepper (arXiv 2106.11476).

The compute path is ``libfw2.so`` (hand-written sm_103a CUDA behind the C ABI
of ``include/fw2.h``); ``paper_2106_11476_gb300.fw2`` is its ctypes binding.
Build the library with ``paper_2106_11476_gb300._build.build()``.
"""
from . import fw2  # noqa: F401

__all__ = ["fw2"]
