"""GPU test of hotrg_rescale_noalloc, the allocation-free max-norm rescale.

It is meant for callers that cannot allocate device memory (a framework that
owns all device memory through its own pool, a process whose quota that pool
already holds, a loop that cannot afford cudaMalloc's synchronisation).  The
test gives it device buffers it did not allocate and compares what it returns
with what the allocating path -- hotrg_create, which rescales the initial
tensor by its max-norm in context-owned scratch -- returns for the same
tensor, on two calls in a row (the second one also checks that the shared
scratch left over from the first call does not leak into the result).

This file is collected last so that a failure here stops a `-x` run only after
every other test has run.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the FP64 path's parity tolerance


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_05900_gb300 as pkg
    return torch, pkg, pkg.load()


def reference(pkg, T0):
    """Existing entry point: the normalised tensor and ln c0 of hotrg_create."""
    with pkg.Hotrg(T0, 8, "fp64") as h:
        T_ref = h.tensor()
        lz0 = h.ln_z_per_site()          # ln c0 + ln Tr(T0 / c0) after zero steps
    return T_ref, lz0 - math.log(np.einsum("aabb->", T_ref))


def call(torch, lib, T0, logsum0, weight):
    T = torch.tensor(np.ascontiguousarray(T0).ravel(), dtype=torch.float64, device="cuda")
    ls = torch.tensor([logsum0], dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.hotrg_rescale_noalloc(ctypes.c_void_p(T.data_ptr()), T.numel(), weight,
                                   ctypes.c_void_p(ls.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return st, T.cpu().numpy().reshape(T0.shape), float(ls.item())


def test_noalloc_rescale_matches_allocating_path_twice(env):
    torch, pkg, lib = env
    rng = np.random.default_rng(20260205)
    cases = [(pkg.ising_tensor(0.44, 0.01), 0.0, 1.0),                 # 16 elements
             (rng.random((7, 7, 7, 7)) * 3.0 + 0.01, 0.25, 0.125)]      # 2401 elements, one ragged block
    for T0, logsum0, weight in cases:
        T_ref, ln_c0 = reference(pkg, T0)
        st, T_got, ls = call(torch, lib, T0, logsum0, weight)
        assert st == 0
        np.testing.assert_allclose(T_got, T_ref, rtol=TOL, atol=0)
        assert abs(ls - (logsum0 + weight * ln_c0)) <= TOL * max(1.0, abs(ls))


def test_noalloc_rescale_rejects_bad_input(env):
    torch, pkg, lib = env
    T = torch.zeros(64, dtype=torch.float64, device="cuda")
    ls = torch.zeros(1, dtype=torch.float64, device="cuda")
    p, q = ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(ls.data_ptr())
    assert lib.hotrg_rescale_noalloc(p, (1 << 26) + 1, 1.0, q, None) == 1   # beyond the limit
    assert lib.hotrg_rescale_noalloc(p, 0, 1.0, q, None) == 1
    assert lib.hotrg_rescale_noalloc(None, 64, 1.0, q, None) == 1
    torch.cuda.synchronize()
    assert lib.hotrg_rescale_noalloc(p, 64, 1.0, q, None) == 5              # zero norm
    assert float(ls.item()) == 0.0
