"""CPU-side checks of the C ABI: the library loads, exports every function the
header declares, validates arguments without a GPU, and its host-side initial
tensors match the oracle's (closed-form square root vs. eigendecomposition)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import hotrg as ref

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_05900_gb300 import build as b
    b.build()
    import paper_2602_05900_gb300 as pkg
    return pkg.load()


def test_header_declares_the_boundary():
    from paper_2602_05900_gb300.capi import header_symbols
    names = header_symbols()
    for required in ["hotrg_create", "hotrg_step", "hotrg_free_energy", "hotrg_destroy",
                     "hotrg_log_z_per_site", "hotrg_spectrum", "hotrg_step_info"]:
        assert required in names


def test_library_exports_every_header_symbol(lib):
    from paper_2602_05900_gb300.capi import LIB_PATH, header_symbols
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [s for s in header_symbols() if s not in exported]
    assert not missing, missing
    for s in header_symbols():
        assert hasattr(lib, s)


@pytest.mark.parametrize("beta,h", [(0.4406867935097715, 0.0), (0.44, 0.01), (0.3, -0.25), (1.3, 0.2)])
def test_ising_tensor_matches_oracle(lib, beta, h):
    import paper_2602_05900_gb300 as pkg
    assert np.allclose(pkg.ising_tensor(beta, h), ref.ising_initial_tensor(beta, h),
                       rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("q,beta", [(2, 0.7), (3, 1.0050525696307162), (4, 0.5), (5, 1.2)])
def test_potts_tensor_matches_oracle(lib, q, beta):
    import paper_2602_05900_gb300 as pkg
    assert np.allclose(pkg.potts_tensor(q, beta), ref.potts_initial_tensor(q, beta),
                       rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("Jxy,Jz,tau", [(1.0, 1.0, 0.1), (1.0, 0.0, 1 / 32), (0.0, 1.0, 0.3),
                                         (0.7, -0.3, 0.05), (-1.0, -1.0, 0.2), (1.0, 1.0, 2.0)])
def test_xxz_tensor_matches_oracle(lib, Jxy, Jz, tau):
    import paper_2602_05900_gb300 as pkg
    from oracle import heisenberg
    assert np.allclose(pkg.xxz_tensor(Jxy, Jz, tau), heisenberg.cell_tensor(Jxy, Jz, tau),
                       rtol=0, atol=1e-13)


def test_xxz_argument_validation(lib):
    from paper_2602_05900_gb300.capi import HOTRG_EINVAL
    buf = np.zeros(256)
    dp = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.hotrg_xxz_tensor(1.0, 1.0, 0.0, dp) == HOTRG_EINVAL
    assert lib.hotrg_xxz_tensor(1.0, 1.0, -0.1, dp) == HOTRG_EINVAL
    assert lib.hotrg_xxz_tensor(float("nan"), 1.0, 0.1, dp) == HOTRG_EINVAL
    assert lib.hotrg_xxz_tensor(1.0, float("inf"), 0.1, dp) == HOTRG_EINVAL
    assert lib.hotrg_xxz_tensor(1.0, 1.0, 0.1, None) == HOTRG_EINVAL
    assert lib.hotrg_trace_y(None) == HOTRG_EINVAL


def test_itebd_argument_validation(lib):
    from paper_2602_05900_gb300.capi import HOTRG_EINVAL
    cp = np.array([1.0, 1.0, 0.05])
    dp = cp.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    bad = [(0, dp, 8, 1), (1, None, 8, 1), (1, dp, 0, 1), (1, dp, 49, 1), (1, dp, 8, 2), (1, dp, 8, 0)]
    for n, c, Db, D0 in bad:      # rejected before any device work
        assert lib.hotrg_itebd_create(n, c, Db, D0, None, None, None, None, ctypes.byref(h)) == HOTRG_EINVAL
        assert h.value is None
    for vals in ([1.0, 1.0, 0.0], [1.0, 1.0, -0.1], [float("nan"), 1.0, 0.1], [1.0, float("inf"), 0.1]):
        cb = np.array(vals)
        assert lib.hotrg_itebd_create(1, cb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 8, 1,
                                      None, None, None, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert lib.hotrg_itebd_create(1, dp, 8, 1, None, None, None, None, None) == HOTRG_EINVAL
    assert lib.hotrg_itebd_step(None, 1) == HOTRG_EINVAL
    assert lib.hotrg_itebd_energy(None, dp) == HOTRG_EINVAL
    lib.hotrg_itebd_destroy(None)   # NULL-safe


def test_host_argument_validation(lib):
    import paper_2602_05900_gb300 as pkg
    from paper_2602_05900_gb300.capi import HOTRG_EINVAL
    buf = np.zeros(16)
    dp = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.hotrg_ising_tensor(-1.0, 0.0, dp) == HOTRG_EINVAL
    assert lib.hotrg_ising_tensor(0.4, 0.0, None) == HOTRG_EINVAL
    assert lib.hotrg_potts_tensor(1, 0.4, dp) == HOTRG_EINVAL
    assert lib.hotrg_potts_tensor(17, 0.4, dp) == HOTRG_EINVAL
    h = ctypes.c_void_p()
    # invalid sizes and precisions are rejected before any device work
    assert lib.hotrg_create(dp, 0, 8, 0, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert lib.hotrg_create(dp, 2, 65, 0, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert lib.hotrg_create(dp, 2, 8, 9, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert lib.hotrg_create(None, 2, 8, 0, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert h.value is None
    assert lib.hotrg_step(None, 0) == HOTRG_EINVAL
    lib.hotrg_destroy(None)   # NULL-safe
    assert pkg.status_string(HOTRG_EINVAL) == "HOTRG_EINVAL"


def test_batch_argument_validation(lib):
    from paper_2602_05900_gb300.capi import HOTRG_EINVAL
    bufs = [np.zeros(16), np.zeros(16)]
    dp = ctypes.POINTER(ctypes.c_double)
    ptrs = (dp * 2)(*[b.ctypes.data_as(dp) for b in bufs])
    d0 = (ctypes.c_int * 2)(2, 2)
    h = ctypes.c_void_p()
    # rejected before any device work: count, NULL arrays, sizes, precision
    assert lib.hotrg_batch_create(0, ptrs, d0, (ctypes.c_int * 2)(8, 8), 1, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert lib.hotrg_batch_create(4097, ptrs, d0, (ctypes.c_int * 2)(8, 8), 1, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert lib.hotrg_batch_create(2, None, d0, (ctypes.c_int * 2)(8, 8), 1, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert lib.hotrg_batch_create(2, ptrs, d0, (ctypes.c_int * 2)(8, 65), 1, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert lib.hotrg_batch_create(2, ptrs, (ctypes.c_int * 2)(2, 0), (ctypes.c_int * 2)(8, 8), 1, None,
                                  ctypes.byref(h)) == HOTRG_EINVAL
    assert lib.hotrg_batch_create(2, ptrs, d0, (ctypes.c_int * 2)(8, 8), 7, None, ctypes.byref(h)) == HOTRG_EINVAL
    nullptrs = (dp * 2)(bufs[0].ctypes.data_as(dp), dp())
    assert lib.hotrg_batch_create(2, nullptrs, d0, (ctypes.c_int * 2)(8, 8), 1, None, ctypes.byref(h)) == HOTRG_EINVAL
    assert h.value is None
    n = ctypes.c_int()
    assert lib.hotrg_batch_size(None, ctypes.byref(n)) == HOTRG_EINVAL
    assert lib.hotrg_batch_step(None, 0) == HOTRG_EINVAL
    assert lib.hotrg_batch_log_z(None, None) == HOTRG_EINVAL


def test_option_and_emulated_gemm_argument_validation(lib):
    from paper_2602_05900_gb300.capi import HOTRG_EINVAL
    # no context: rejected before any device work
    assert lib.hotrg_set_option(None, 0, 1) == HOTRG_EINVAL
    # hotrg_dgemm_emu validates sizes, strides, pointers and digit count first
    p = ctypes.c_void_p(16)
    assert lib.hotrg_dgemm_emu(4, 4, 0, p, 4, p, 4, p, 4, 7, None) == HOTRG_EINVAL     # K < 1
    assert lib.hotrg_dgemm_emu(4, 4, 8, p, 4, p, 8, p, 4, 7, None) == HOTRG_EINVAL     # lda < K
    assert lib.hotrg_dgemm_emu(4, 4, 8, p, 8, p, 8, p, 2, 7, None) == HOTRG_EINVAL     # ldc < N
    assert lib.hotrg_dgemm_emu(4, 4, 8, None, 8, p, 8, p, 4, 7, None) == HOTRG_EINVAL  # NULL A
    assert lib.hotrg_dgemm_emu(4, 4, 8, p, 8, p, 8, p, 4, 3, None) == HOTRG_EINVAL     # digits < 4
    assert lib.hotrg_dgemm_emu(4, 4, 8, p, 8, p, 8, p, 4, 9, None) == HOTRG_EINVAL     # digits > 8
    assert lib.hotrg_dgemm_emu(-1, 4, 8, p, 8, p, 8, p, 4, 7, None) == HOTRG_EINVAL
    assert lib.hotrg_dgemm_emu(0, 4, 8, p, 8, p, 8, p, 4, 7, None) == 0                # empty: nothing to do


def test_binding_constants_match_the_header():
    """Every status code and option number the binding uses is the header's."""
    import re
    from paper_2602_05900_gb300 import capi
    text = open(os.path.join(ROOT, "include", "hotrg.h")).read()
    enums = {name: int(val) for name, val in re.findall(r"\b(HOTRG_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    for name in ["HOTRG_OK", "HOTRG_EINVAL", "HOTRG_ENOMEM", "HOTRG_ECUDA", "HOTRG_EEIG",
                 "HOTRG_ENONFINITE", "HOTRG_ETIMEOUT", "HOTRG_ESTATE", "HOTRG_EBOUNDS"]:
        assert getattr(capi, name) == enums[name], name
    opts = {k: v for k, v in enums.items() if k.startswith("HOTRG_OPT_")}
    assert opts, "no options in the header"
    for name, val in opts.items():
        assert getattr(capi, name[len("HOTRG_"):]) == val, name
