"""GPU parity of quantum HOTRG for the XXZ chain (Sec. II.A-B): the cell tensor
built by the C ABI, n_t Y steps along imaginary time, the time trace
(``hotrg_trace_y``) and X steps along the chain, against the FP64 oracle run
on the same schedule, and against the pinned exact results (free fermions
at Jz = 0, the classical Ising chain at Jxy = 0, dense rings).

Compared quantities are gauge-invariant: ln Z / N_cells, the step bookkeeping,
the normalised spectra at steps whose cut is not degenerate (the SU(2)
multiplets of the Heisenberg point make many cuts degenerate) and the
normalised spectrum of the final column matrix.
"""
import math

import numpy as np
import pytest

from oracle import heisenberg as hz

pytestmark = pytest.mark.gpu

GAP_TOL = 1e-9
# Relative error of ln Z / N_cells against the FP64 oracle, per precision mode.
# Operand rounding u perturbs every ln c_j by O(u) in absolute terms, while
# ln Z / N_cells is only about 2 tau |f| (0.044 at tau = 1/32, beta = 4): the
# relative error is amplified by 1 / (2 tau |f|) ~ 23 against a classical model.
# Bounds: 23 u with TF32 u = 2^-11 and split-BF16 u ~ 2^-16 (measured 3.6e-3
# and 2.0e-5); the exact-slice mode (six digits) measured 6.0e-11.
QTOL = {"fp64": 1e-12, "bf16xs": 3e-10, "bf16x3": 4e-4, "tf32": 1.2e-2}


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_05900_gb300 as p
    p.load()
    return p


def compare_steps(h, r, tol):
    """Step bookkeeping and the normalised spectra at non-degenerate cuts.  The
    environment traces are not compared: they scale with the max-norm of the
    previous tensor, which depends on the rotation chosen inside a kept
    degenerate multiplet (a gauge freedom; ln Z does not depend on it)."""
    mirrored = False   # a tie of the two sides was broken: later L / R may be swapped
    for i, s in enumerate(r.steps):
        info = h.step_info(i)
        assert (info.Dx, info.Dy, info.Dn) == (s.Dx, s.Dy, s.Dn), i
        assert info.dir == (0 if s.direction == "x" else 1)
        if s.side >= 0:
            # discarded weights relative to Tr G (free of the max-norm scale), unordered
            want = sorted([s.eps_L / s.trace_G, s.eps_R / s.trace_G])
            got = sorted([info.eps_L / info.trace_G, info.eps_R / info.trace_G])
            assert np.allclose(got, want, rtol=1e-6, atol=1e-13), i
            if abs(s.eps_L - s.eps_R) <= 1e-8 * s.trace_G:
                mirrored = True
            elif not mirrored:
                assert info.side == s.side, (i, info.side, s.side)
        if s.cut_gap > GAP_TOL:
            spec = h.spectrum(i)
            n = min(s.Dn, spec.size)
            assert np.allclose(spec[:n], s.spectrum[:n], rtol=0, atol=tol), i


def column_spectrum(T, k=6):
    """Leading |eigenvalues| of the closed column matrix, over the largest: invariant
    under the similarity gauge of the x legs and under the max-norm scale."""
    w = np.sort(np.abs(np.linalg.eigvals(T[:, :, 0, 0])))[::-1]
    return w[:k] / w[0]


# D_cut values whose every cut falls in a gap of the spectrum (> 1e-7 relative):
# at the SU(2) point most cuts split a degenerate multiplet, which makes the
# kept subspace depend on the eigensolver (see test_fp64_degenerate_cuts)
@pytest.mark.parametrize("Jxy,Jz,tau,D_cut,nt,nx", [
    (1.0, 1.0, 1 / 32, 16, 5, 12),     # Heisenberg, beta = 1
    (1.0, 1.0, 1 / 16, 16, 6, 12),     # Heisenberg, beta = 4
    (1.0, 0.0, 1 / 32, 16, 4, 12),     # XX chain
    (0.7, -0.3, 0.05, 18, 4, 10),      # anisotropic, ferromagnetic Jz
])
def test_fp64_quantum_run_vs_oracle(pkg, Jxy, Jz, tau, D_cut, nt, nx):
    r = hz.run(hz.cell_tensor(Jxy, Jz, tau), D_cut, nt, nx)
    with pkg.Hotrg(pkg.xxz_tensor(Jxy, Jz, tau), D_cut, "fp64") as h:
        h.run_quantum(nt, nx)
        assert abs(h.ln_z_per_site() / r.ln_z_per_site - 1) < 1e-12
        compare_steps(h, r, 1e-11)
        assert h.dims() == (r.T.shape[0], 1, nt + nx)
        T = h.tensor()
        assert T.shape == r.T.shape
        assert np.allclose(column_spectrum(T), column_spectrum(r.T), rtol=0, atol=1e-10)


def test_fp64_degenerate_cuts(pkg):
    """Heisenberg at D_cut = 24: the cuts split SU(2) multiplets, so which
    vectors of a split multiplet are kept is the eigensolver's choice.  ln Z
    then agrees to the truncation error (about 1e-8 relative here, measured
    on the oracle as D_cut = 24 against 32), not to rounding."""
    tau, nt, nx = 1 / 32, 5, 12
    r = hz.run(hz.cell_tensor(1.0, 1.0, tau), 24, nt, nx)
    with pkg.Hotrg(pkg.xxz_tensor(1.0, 1.0, tau), 24, "fp64") as h:
        h.run_quantum(nt, nx)
        assert abs(h.ln_z_per_site() / r.ln_z_per_site - 1) < 5e-8


@pytest.mark.parametrize("nt", [0, 1])
def test_fp64_trace_y_untruncated_is_dense_trotter(pkg, nt):
    """Nothing is cut (D_cut = 16 >= every fused dimension): ln Z of the ring
    of 2^(nx+1) sites over 2^nt periods equals the dense Trotter trace."""
    Jxy, Jz, tau, nx = 1.0, 1.0, 0.1, 2
    with pkg.Hotrg(pkg.xxz_tensor(Jxy, Jz, tau), 16, "fp64") as h:
        h.run_quantum(nt, nx)
        assert all(h.step_info(i).Dn == h.step_info(i).Dx ** 2 for i in range(nt + nx))
        lnz = h.ln_z_per_site() * 2 ** (nt + nx)
    assert abs(lnz - hz.trotter_ln_z(2 ** (nx + 1), Jxy, Jz, tau, 2 ** nt)) < 1e-11


def test_fp64_xx_free_fermions(pkg):
    tau, nt = 1 / 32, 3
    with pkg.Hotrg(pkg.xxz_tensor(1.0, 0.0, tau), 16, "fp64") as h:
        h.run_quantum(nt, 30)
        v = h.ln_z_per_site()
    assert abs(v - hz.xx_trotter_ln_z_per_cell(1.0, tau, 2 ** nt)) < 1e-11


@pytest.mark.parametrize("Jz", [1.0, -2.0])
def test_fp64_ising_chain_limit(pkg, Jz):
    tau, nt = 0.1, 4
    with pkg.Hotrg(pkg.xxz_tensor(0.0, Jz, tau), 16, "fp64") as h:
        h.run_quantum(nt, 30)
        v = h.ln_z_per_site()
    assert abs(v - hz.ising_chain_ln_z_per_cell(Jz, tau * 2 ** nt, 2 ** nt)) < 1e-13


@pytest.mark.parametrize("prec", ["tf32", "bf16x3", "bf16xs"])
def test_mixed_precision_heisenberg_vs_oracle(pkg, prec):
    Jxy, Jz, tau, D_cut, nt, nx = 1.0, 1.0, 1 / 32, 16, 7, 16
    r = hz.run(hz.cell_tensor(Jxy, Jz, tau), D_cut, nt, nx)
    with pkg.Hotrg(pkg.xxz_tensor(Jxy, Jz, tau), D_cut, prec) as h:
        h.run_quantum(nt, nx)
        v = h.ln_z_per_site()
        f = h.free_energy(2 * tau)
    err = abs(v / r.ln_z_per_site - 1)
    print(f"{prec}: rel err ln Z {err:.3e}, f {f:.12f} oracle "
          f"{hz.free_energy_per_site(r.ln_z_per_site, tau):.12f}")
    assert err < QTOL[prec]


def test_batch_of_couplings(pkg):
    """One context, several chains of the same cut: every instance matches its
    own oracle run, and the time trace closes all of them at once."""
    cases = [(1.0, 1.0, 1 / 32), (1.0, 0.0, 1 / 32), (0.0, 1.0, 0.1)]
    D_cut, nt, nx = 16, 5, 10
    T0s = [pkg.xxz_tensor(*c) for c in cases]
    with pkg.HotrgBatch(T0s, [D_cut] * len(cases), "fp64") as b:
        b.run_quantum(nt, nx)
        got = b.ln_z_per_site()
    for c, v in zip(cases, got):
        want = hz.run(hz.cell_tensor(*c), D_cut, nt, nx).ln_z_per_site
        assert abs(v / want - 1) < 1e-12, c


def test_batch_two_cut_groups(pkg):
    """Chains with different cuts form separate groups of one context; the time
    trace closes every group.  (Heisenberg at D_cut 16 cuts in spectral gaps; the
    Ising chain's cut at 12 only drops exact zeros.)"""
    cases = [((1.0, 1.0, 1 / 32), 16), ((0.0, 1.0, 0.1), 12), ((1.0, 1.0, 1 / 32), 16)]
    nt, nx = 5, 8
    with pkg.HotrgBatch([pkg.xxz_tensor(*c) for c, _ in cases], [d for _, d in cases], "fp64") as b:
        b.run_quantum(nt, nx)
        got = b.ln_z_per_site()
    for (c, d), v in zip(cases, got):
        want = hz.run(hz.cell_tensor(*c), d, nt, nx).ln_z_per_site
        assert abs(v / want - 1) < 1e-12, (c, d)


def test_free_energy_low_temperature(pkg):
    """beta = 16 at D_cut = 32 on the FP64 path: f approaches the Bethe-ansatz
    ground-state energy 1/4 - ln 2 with the T^2 / 3 correction of the chain."""
    tau, nt = 1 / 32, 9
    with pkg.Hotrg(pkg.xxz_tensor(1.0, 1.0, tau), 32, "fp64") as h:
        h.run_quantum(nt, 30)
        f = h.free_energy(2 * tau)
    e0 = 0.25 - math.log(2.0)
    assert abs(f - (e0 - (1 / 16) ** 2 / 3)) < 2e-3
