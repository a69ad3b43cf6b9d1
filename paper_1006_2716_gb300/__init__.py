"""GB300-native (sm_103a) Hirsch-Fye QMC based real-space DMFT for the trapped Hubbard model.

Method: Bluemer & Gorelik, arXiv:1006.2716.  The compute path is the CUDA library built from
``csrc/`` (C ABI in ``include/hf.h``); ``hf`` is its Python binding.
"""
from . import workloads  # noqa: F401

__all__ = ["hf", "workloads", "build"]
