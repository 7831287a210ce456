"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Compared quantities are gauge-invariant (Sec. II.A leaves the eigenvector
signs and degenerate rotations free): ln Z / N, the normalised spectra of the
chosen environment at steps whose cut is not degenerate, the discarded weights
and the step bookkeeping.  FP64 path: <= 1e-12 relative.  Mixed precision:
the error against the oracle is measured and bounded by the tolerances below
(each mode's operand rounding -- TF32 keeps 10 mantissa bits, a two-term BF16
split about 16 -- damped by the 1/2^n weights of the later steps).
"""
import math

import numpy as np
import pytest

from oracle import exact, hotrg as ref, onsager
from workloads import BETA_C_ISING, BETA_C_POTTS3, random_tensor

pytestmark = pytest.mark.gpu

GAP_TOL = 1e-9   # steps with a smaller relative gap at the cut are not compared element-wise
MIXED_TOL = {"tf32": 2e-4, "bf16x3": 5e-5, "bf16x6": 2e-6, "bf16xs": 1e-10}


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_05900_gb300 as p
    p.load()
    return p


def run_gpu(pkg, T0, D_cut, nsteps, prec="fp64", first="x"):
    h = pkg.Hotrg(T0, D_cut, prec)
    h.run(nsteps, first)
    return h


def compare_steps(h, r, tol):
    for i, s in enumerate(r.steps):
        info = h.step_info(i)
        assert (info.Dx, info.Dy, info.Dn) == (s.Dx, s.Dy, s.Dn)
        assert info.dir == (0 if s.direction == "x" else 1)
        if s.side >= 0:
            # the side choice is gauge-invariant unless both sides discard the same weight
            if abs(s.eps_L - s.eps_R) > 1e-8 * s.trace_G:
                assert info.side == s.side, (i, info.side, s.side)
        assert abs(info.trace_G / s.trace_G - 1) < tol
        if s.cut_gap > GAP_TOL:
            spec = h.spectrum(i)
            n = min(s.Dn, spec.size)
            assert np.allclose(spec[:n], s.spectrum[:n], rtol=0, atol=tol), i


@pytest.mark.parametrize("D_cut,nsteps", [(8, 20), (12, 12), (7, 10)])
def test_fp64_ising_critical_vs_oracle(pkg, D_cut, nsteps):
    T0 = pkg.ising_tensor(BETA_C_ISING)
    r = ref.run(ref.ising_initial_tensor(BETA_C_ISING), D_cut, nsteps)
    with run_gpu(pkg, T0, D_cut, nsteps) as h:
        assert abs(h.ln_z_per_site() / r.ln_z_per_site - 1) < 1e-12
        compare_steps(h, r, 1e-11)
        assert h.dims() == (r.T.shape[0], r.T.shape[2], nsteps)


def test_fp64_onsager_d8_20_steps(pkg):
    with run_gpu(pkg, pkg.ising_tensor(BETA_C_ISING), 8, 20) as h:
        f = h.free_energy(BETA_C_ISING)
    fo = onsager.ising_free_energy(BETA_C_ISING)
    assert abs(f / fo - 1) < 2e-5


@pytest.mark.parametrize("model,L,D_cut", [("ising_bc", 4, 16), ("ising_h", 4, 16), ("potts3", 2, 9)])
def test_fp64_no_truncation_is_exact(pkg, model, L, D_cut):
    """With D_cut at least the largest fused dimension nothing is cut and the
    result is the exact partition function of the L x L torus."""
    if model == "potts3":
        T0, B, w = pkg.potts_tensor(3, BETA_C_POTTS3), np.exp(BETA_C_POTTS3 * np.eye(3)), np.ones(3)
    else:
        beta, hf = (BETA_C_ISING, 0.0) if model == "ising_bc" else (0.44, 0.01)
        s = np.array([1.0, -1.0])
        T0, B, w = pkg.ising_tensor(beta, hf), np.exp(beta * np.outer(s, s)), np.exp(beta * hf * s)
    nsteps = 2 * int(round(math.log2(L)))
    with run_gpu(pkg, T0, D_cut, nsteps) as h:
        lz = h.ln_z_per_site() * L * L
        assert all(h.step_info(i).side == -1 for i in range(nsteps))
    assert abs(lz - exact.transfer_matrix_ln_z(B, w, L, L)) < 1e-11


@pytest.mark.parametrize("D0,D_cut,nsteps,first,seed", [(3, 5, 6, "x", 1), (4, 7, 5, "y", 2),
                                                          (2, 3, 7, "x", 3), (5, 13, 3, "y", 4)])
def test_fp64_random_tensor_vs_oracle(pkg, D0, D_cut, nsteps, first, seed):
    T0 = random_tensor(D0, seed=seed)
    r = ref.run(T0, D_cut, nsteps, first=first)
    with run_gpu(pkg, T0, D_cut, nsteps, first=first) as h:
        assert abs(h.ln_z_per_site() / r.ln_z_per_site - 1) < 1e-12
        compare_steps(h, r, 1e-10)


def test_fp64_potts3_vs_oracle(pkg):
    T0 = pkg.potts_tensor(3, BETA_C_POTTS3)
    r = ref.run(ref.potts_initial_tensor(3, BETA_C_POTTS3), 9, 10)
    with run_gpu(pkg, T0, 9, 10) as h:
        assert abs(h.ln_z_per_site() / r.ln_z_per_site - 1) < 1e-12


def test_fp64_tensor_and_isometry_after_step(pkg):
    """One truncating step element by element after fixing U's column signs."""
    T0 = random_tensor(3, seed=17)
    with pkg.Hotrg(T0, 4, "fp64") as h:
        h.step("y")
        Tg = h.tensor()
        Ug = h.isometry()
    Tn, c, U, info = ref.y_step(T0 / np.max(np.abs(T0)), 4)
    assert Ug.shape == U.shape
    sg = np.sign(np.sum(Ug * U, axis=0))          # per-column sign relating the two gauges
    assert np.allclose(np.abs(np.sum(Ug * U, axis=0)), 1.0, atol=1e-10)
    assert np.allclose(Ug * sg, U, atol=1e-10)
    assert np.allclose(np.einsum("abyz,a,b->abyz", Tg, sg, sg), Tn, atol=1e-12)


@pytest.mark.parametrize("prec", ["tf32", "bf16x3", "bf16x6", "bf16xs"])
@pytest.mark.parametrize("D_cut,nsteps", [(8, 14), (16, 12)])
def test_mixed_precision_vs_oracle(pkg, prec, D_cut, nsteps):
    T0 = pkg.ising_tensor(0.44, 0.01)
    r = ref.run(ref.ising_initial_tensor(0.44, 0.01), D_cut, nsteps)
    with run_gpu(pkg, T0, D_cut, nsteps, prec) as h:
        err = abs(h.ln_z_per_site() / r.ln_z_per_site - 1)
    print(f"{prec} D_cut={D_cut}: relative lnZ/N error vs FP64 oracle = {err:.3e}")
    assert err < MIXED_TOL[prec]


@pytest.mark.parametrize("prec", ["tf32", "bf16x3", "bf16xs"])
def test_mixed_precision_random_tensor(pkg, prec):
    T0 = random_tensor(4, seed=5)
    r = ref.run(T0, 11, 6, first="y")
    with run_gpu(pkg, T0, 11, 6, prec, first="y") as h:
        err = abs(h.ln_z_per_site() / r.ln_z_per_site - 1)
    assert err < MIXED_TOL[prec]


def test_nonfinite_initial_tensor_is_rejected(pkg):
    T0 = np.ones((2, 2, 2, 2))
    T0[0, 1, 0, 1] = np.nan
    with pytest.raises(pkg.HotrgError) as e:
        pkg.Hotrg(T0, 8)
    assert e.value.status == 5


def test_zero_tensor_is_rejected(pkg):
    with pytest.raises(pkg.HotrgError) as e:
        pkg.Hotrg(np.zeros((2, 2, 2, 2)), 8)
    assert e.value.status == 5


@pytest.mark.parametrize("D_cut,nsteps,paths", [(8, 10, {0, 1}), (12, 12, {0, 1, 2}), (16, 10, {0, 2})])
def test_eigensolver_paths_and_residuals(pkg, D_cut, nsteps, paths):
    """The own FP64 eigensolver serves every cut (no library fallback) and
    meets its residual target; spectra agree with LAPACK's through the oracle."""
    T0 = pkg.ising_tensor(0.44)
    r = ref.run(ref.ising_initial_tensor(0.44), D_cut, nsteps)
    with run_gpu(pkg, T0, D_cut, nsteps) as h:
        seen = set()
        for i, s in enumerate(r.steps):
            info = h.step_info(i)
            seen.add(info.eig_path)
            assert info.eig_path != 3, f"step {i} fell back to the library eigensolver"
            if info.eig_path == 2:
                assert info.eig_residual <= 1e-12
                assert 1 <= info.eig_iters <= 80
        assert seen <= paths and 0 in seen
        compare_steps(h, r, 1e-11)
        assert abs(h.ln_z_per_site() / r.ln_z_per_site - 1) < 1e-12


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_graph_replay_matches_eager(pkg, prec):
    """Contraction segments replayed from CUDA graphs (a non-NULL stream is
    needed for capture) give bit-identical results to eager launches."""
    torch = pytest.importorskip("torch")
    from paper_2602_05900_gb300.capi import OPT_GRAPHS
    stream = torch.cuda.Stream()
    T0 = pkg.ising_tensor(0.44, 0.01)
    out = {}
    for graphs in (1, 0):
        with pkg.Hotrg(T0, 16, prec, stream) as h:
            h.set_option(OPT_GRAPHS, graphs)
            h.run(16)
            out[graphs] = (h.ln_z_per_site(), h.tensor())
    assert out[1][0] == out[0][0]
    assert np.array_equal(out[1][1], out[0][1])


def test_eigensolver_iteration_cap_gives_eeig(pkg):
    """A solve that cannot reach its residual bound within the iteration cap
    fails the step with HOTRG_EEIG (no library fallback); the error is latched
    and a fresh context is unaffected."""
    from paper_2602_05900_gb300.capi import HOTRG_EEIG, OPT_EIG_MAX_ITERS
    T0 = pkg.ising_tensor(0.44)
    with pkg.Hotrg(T0, 12, "fp64") as h:
        h.set_option(OPT_EIG_MAX_ITERS, 1)
        with pytest.raises(pkg.HotrgError) as e:
            h.run(8)                     # step 4 (Dx = 16 > D_cut) needs the subspace iteration
        assert e.value.status == HOTRG_EEIG
        with pytest.raises(pkg.HotrgError) as e2:
            h.step("x")                  # latched
        assert e2.value.status == HOTRG_EEIG
    r = ref.run(ref.ising_initial_tensor(0.44), 12, 8)
    with run_gpu(pkg, T0, 12, 8) as h:
        assert abs(h.ln_z_per_site() / r.ln_z_per_site - 1) < 1e-12


@pytest.mark.parametrize("prec", ["tf32", "bf16xs"])
def test_bounded_wait_timeout_is_reported(pkg, prec):
    """The timeout path of the tensor-core kernels (tcgen05 GEMM, exact-slice
    GEMM): a launch whose producer issues nothing leaves its consumers waiting
    on a barrier nothing arrives at; with a short wait bound the kernel gives
    up, records the failure, releases its tensor memory and returns, and the
    step reports HOTRG_ETIMEOUT.  The device stays usable: a new context with
    the default bound reproduces the oracle."""
    from paper_2602_05900_gb300.capi import (HOTRG_ETIMEOUT, OPT_TEST_STALL, OPT_WAIT_CYCLES,
                                             WAIT_CYCLES_DEFAULT)
    T0 = pkg.ising_tensor(0.44, 0.01)
    try:
        with pkg.Hotrg(T0, 8, prec) as h:
            h.run(2)                                  # D = 4: the contractions are tensor-core GEMMs
            h.set_option(OPT_WAIT_CYCLES, 200_000)    # ~0.1 ms
            h.set_option(OPT_TEST_STALL, 1)
            with pytest.raises(pkg.HotrgError) as e:
                h.step("x")
            assert e.value.status == HOTRG_ETIMEOUT
    finally:
        with pkg.Hotrg(T0, 8, prec) as h2:
            h2.set_option(OPT_WAIT_CYCLES, WAIT_CYCLES_DEFAULT)
    r = ref.run(ref.ising_initial_tensor(0.44, 0.01), 8, 8)
    with run_gpu(pkg, T0, 8, 8, prec) as h:
        assert abs(h.ln_z_per_site() / r.ln_z_per_site - 1) < MIXED_TOL[prec]
