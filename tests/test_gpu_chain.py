"""GPU parity of the fused a6 -> a7 projection kernel (TF32, Dx = Dy in {16, 32},
D' <= 32; Sec. II.B, Eq. 3: Q = P T is contracted with U on chip and never
written to device memory).

* One steady-state step from the same input with the fused kernel and with
  the two-GEMM chain: identical isometry (the eigensolver runs before the
  projection on identical environments) and T' equal up to the order of the
  FP32 sums over (x1', x2').
* Whole jobs (single context and a batch with two cut groups) against the
  FP64 oracle within the TF32 bound.
* The kernel's timeout path: a launch that issues no copies reports
  HOTRG_ETIMEOUT and leaves the device usable.

The sampled element check of T' against its definition at D_cut = 32 (TF32,
which takes the fused kernel) is in test_gpu_fullsize.py.
"""
import numpy as np
import pytest

from oracle import hotrg as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_05900_gb300 as p
    p.load()
    return p


def steady_input(pkg, beta, h, D_cut):
    """The normalised input tensor of the first step with Dx = Dy = D_cut."""
    with pkg.Hotrg(pkg.ising_tensor(beta, h), D_cut, "tf32") as h0:
        d = "x"
        while True:
            dx, dy, _ = h0.dims()
            if dx == D_cut and dy == D_cut:
                return h0.tensor()
            h0.step(d)
            d = "y" if d == "x" else "x"


@pytest.mark.parametrize("D_cut", [16, 32])
@pytest.mark.parametrize("direction", ["x", "y"])
def test_fused_step_matches_two_gemm_chain(pkg, D_cut, direction):
    """Both paths round Q to TF32 and accumulate T' in FP32 over the same D^2
    products; only the order of that sum differs ((x2', x1') against
    (x1', x2')), so |T'_fused - T'_chain| stays at FP32 accumulation level
    (D^2 2^-24 of the summed magnitudes, ~6e-5 at D = 32), far below the TF32
    error of T' itself (~2e-3, the bound of the sampled element test)."""
    from paper_2602_05900_gb300.capi import OPT_FUSED_CHAIN
    T_in = steady_input(pkg, 0.44, 0.01, D_cut)
    out = {}
    for fuse in (1, 0):
        with pkg.Hotrg(T_in, D_cut, "tf32") as h:
            h.set_option(OPT_FUSED_CHAIN, fuse)
            h.step(direction)
            info = h.step_info(0)
            out[fuse] = (h.tensor() * np.exp(info.ln_c), h.isometry())
    (Tf, Uf), (Tc, Uc) = out[1], out[0]
    assert np.array_equal(Uf, Uc)
    scale = np.abs(Tc).max()
    err = np.abs(Tf - Tc).max() / scale
    print(f"D={D_cut} {direction}: max |T'_fused - T'_chain| / max |T'| = {err:.2e}")
    assert err < 1e-4
    assert err > 0          # the fused kernel ran: its sums end in other last bits


@pytest.mark.parametrize("D_cut,nsteps", [(16, 16), (32, 12)])
def test_fused_job_vs_oracle(pkg, D_cut, nsteps):
    from paper_2602_05900_gb300.capi import OPT_FUSED_CHAIN
    want = ref.run(ref.ising_initial_tensor(0.44, 0.01), D_cut, nsteps).ln_z_per_site
    got = {}
    for fuse in (1, 0):
        with pkg.Hotrg(pkg.ising_tensor(0.44, 0.01), D_cut, "tf32") as h:
            h.set_option(OPT_FUSED_CHAIN, fuse)
            got[fuse] = h.run(nsteps).ln_z_per_site()
    err = abs(got[1] / want - 1)
    print(f"D={D_cut}: fused {err:.2e}, two-GEMM chain {abs(got[0] / want - 1):.2e}")
    assert err < 5e-4
    # both runs differ only at FP32 accumulation level per step (see above)
    assert abs(got[1] / got[0] - 1) < 1e-5


def test_fused_batch_vs_oracle(pkg):
    """Three instances in two cut groups (16, 16, 12): the D_cut = 16 group
    takes the fused kernel as one launch over its instances, the other the
    two-GEMM chain."""
    from paper_2602_05900_gb300.capi import OPT_FUSED_CHAIN
    betas, cuts, nsteps = [0.42, 0.45, 0.44], [16, 16, 12], 12
    with pkg.HotrgBatch([pkg.ising_tensor(b) for b in betas], cuts, "tf32") as bt:
        bt.set_option(OPT_FUSED_CHAIN, 1)
        lz = bt.run(nsteps).ln_z_per_site()
    for b, D, v in zip(betas, cuts, lz):
        want = ref.run(ref.ising_initial_tensor(b), D, nsteps).ln_z_per_site
        assert abs(v / want - 1) < 5e-4, (b, D, v, want)


def test_fused_kernel_timeout_is_reported(pkg):
    """A fused launch whose producer issues nothing: its MMA and epilogue
    waits run out, the kernel releases its tensor memory and returns, and the
    step reports HOTRG_ETIMEOUT; a new context afterwards matches the oracle."""
    from paper_2602_05900_gb300.capi import (HOTRG_ETIMEOUT, OPT_FUSED_CHAIN, OPT_TEST_STALL,
                                             OPT_WAIT_CYCLES, WAIT_CYCLES_DEFAULT)
    T_in = steady_input(pkg, 0.44, 0.01, 16)
    try:
        with pkg.Hotrg(T_in, 16, "tf32") as h:
            h.set_option(OPT_FUSED_CHAIN, 1)
            h.set_option(OPT_WAIT_CYCLES, 200_000)    # ~0.1 ms
            h.set_option(OPT_TEST_STALL, 2)
            with pytest.raises(pkg.HotrgError) as e:
                h.step("x")
            assert e.value.status == HOTRG_ETIMEOUT
    finally:
        with pkg.Hotrg(T_in, 16, "tf32") as h2:
            h2.set_option(OPT_WAIT_CYCLES, WAIT_CYCLES_DEFAULT)
    want = ref.run(ref.ising_initial_tensor(0.44, 0.01), 16, 8).ln_z_per_site
    with pkg.Hotrg(pkg.ising_tensor(0.44, 0.01), 16, "tf32") as h:
        assert abs(h.run(8).ln_z_per_site() / want - 1) < 5e-4
