"""GB300-native HOTRG coarse-graining for 2D classical lattice models and
quantum spin chains (through their imaginary-time networks), and iTEBD ground
states of those chains.

The compute path lives in ``libhotrg.so`` (CUDA, sm_103a); this package is its
thin ctypes binding.  See ``include/hotrg.h`` for the C ABI.
"""
from .capi import (DIR_X, DIR_Y, PRECISIONS, STAGES, Hotrg, HotrgBatch, HotrgError, Itebd, StepInfo,
                   dgemm_emu, header_symbols, ising_tensor, load, potts_tensor, status_string,
                   xxz_tensor)

__all__ = ["DIR_X", "DIR_Y", "PRECISIONS", "STAGES", "Hotrg", "HotrgBatch", "HotrgError", "Itebd", "StepInfo",
           "dgemm_emu", "header_symbols", "ising_tensor", "load", "potts_tensor", "status_string",
           "xxz_tensor"]
