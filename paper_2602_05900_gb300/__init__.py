"""GB300-native HOTRG coarse-graining for 2D classical lattice models.

The compute path lives in ``libhotrg.so`` (CUDA, sm_103a); this package is its
thin ctypes binding.  See ``include/hotrg.h`` for the C ABI.
"""
from .capi import (DIR_X, DIR_Y, PRECISIONS, STAGES, Hotrg, HotrgBatch, HotrgError, StepInfo,
                   dgemm_emu, header_symbols, ising_tensor, load, potts_tensor, status_string)

__all__ = ["DIR_X", "DIR_Y", "PRECISIONS", "STAGES", "Hotrg", "HotrgBatch", "HotrgError", "StepInfo",
           "dgemm_emu", "header_symbols", "ising_tensor", "load", "potts_tensor", "status_string"]
