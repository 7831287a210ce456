"""GPU parity of iTEBD (Sec. II.A, Eq. 1) through the C ABI against the FP64
oracle: Schmidt values and bond energies after every update from a seeded
random state, a 400-update run whose cuts stay non-degenerate, the Heisenberg
and XX chains against the oracle and the exact ground-state energies, the
Ising fixed point, and batches against single chains."""
import numpy as np
import pytest

from oracle import heisenberg as hz
from oracle import itebd as it
from workloads import random_mps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_05900_gb300 as p
    p.load()
    return p


@pytest.mark.parametrize("Jxy,Jz,tau,D0,D_b", [(1.0, 1.0, 0.05, 4, 8), (1.0, 0.4, 0.1, 6, 10),
                                                (0.8, -0.5, 0.2, 3, 6)])
def test_fp64_updates_vs_oracle(pkg, Jxy, Jz, tau, D0, D_b):
    P, Q, lam = random_mps(D0, seed=5)
    h = hz.bond_hamiltonian(Jxy, Jz)
    g = hz.bond_gate(Jxy, Jz, tau)
    st = it.ItebdRun(P, Q, lam, np.ones(D0) / np.sqrt(D0))
    with pkg.Itebd([(Jxy, Jz, tau)], D_b, init=[(P, Q, lam)]) as c:
        assert abs(c.energy()[0] - it.site_energy(st, h)) < 1e-13
        for k in range(12):
            old = st.lam
            st.P, st.Q, st.lam, disc = it.update(st.P, st.Q, st.lam, g, D_b)
            st.lam_other = old
            c.step(1)
            lam_gpu = c.lam(0)
            assert c.dims()[:2] == (st.lam.size, old.size)
            assert np.allclose(lam_gpu, st.lam, rtol=0, atol=1e-10), k
            assert abs(c.discarded(0) - disc) < 1e-12
            assert abs(c.energy()[0] - it.site_energy(st, h)) < 1e-11, k


def test_fp64_long_run_vs_oracle(pkg):
    """400 updates from a seeded random state of an anisotropic chain whose cut
    stays in a gap of the Schmidt spectrum all along (checked on the oracle run):
    the truncation is unique, so the two sides agree to rounding."""
    Jxy, Jz, tau, D0, D_b, n = 1.0, 0.5, 0.1, 6, 12, 400
    P, Q, lam = random_mps(D0, seed=5)
    g = hz.bond_gate(Jxy, Jz, tau)
    st = it.ItebdRun(P, Q, lam, np.ones(D0) / np.sqrt(D0))
    min_gap = 1.0
    for _ in range(n):
        Dl, Dr = st.P.shape[0], st.Q.shape[2]
        phit = np.einsum("ABab,iabm->iABm", g.reshape(2, 2, 2, 2), np.einsum("iaj,jbm->iabm", st.P, st.Q))
        sv = np.linalg.svd((st.lam[:, None, None, None] * phit).reshape(2 * Dl, 2 * Dr), compute_uv=False)
        if D_b < sv.size:
            min_gap = min(min_gap, (sv[D_b - 1] - sv[D_b]) / sv[0])
        old = st.lam
        st.P, st.Q, st.lam, _ = it.update(st.P, st.Q, st.lam, g, D_b)
        st.lam_other = old
    assert min_gap > 1e-5
    with pkg.Itebd([(Jxy, Jz, tau)], D_b, init=[(P, Q, lam)]) as c:
        c.step(n)
        assert abs(c.energy()[0] - it.site_energy(st, hz.bond_hamiltonian(Jxy, Jz))) < 1e-9
        assert np.allclose(c.lam(0), st.lam, rtol=0, atol=1e-8)


def test_fp64_heisenberg_from_neel(pkg):
    """Neel start, 1500 updates at D_b = 16.  The first updates cut exactly
    degenerate (SU(2)) Schmidt multiplets, where which vectors are kept is the
    eigensolver's choice; imaginary-time convergence of the gapless chain is
    slow (the oracle's own energy still moves by ~5e-6 between 1000 and 1500
    updates), so the two runs agree to that transient level and both lie just
    above the Bethe energy."""
    tau, D_b, n = 0.05, 16, 1500
    ref = it.site_energy(it.run(1.0, 1.0, tau, D_b, n), hz.bond_hamiltonian(1.0, 1.0))
    with pkg.Itebd([(1.0, 1.0, tau)], D_b) as c:
        e = c.step(n).energy()[0]
    assert abs(e - ref) < 2e-5
    e0 = it.heisenberg_ground_energy(1.0)
    assert 0.0 < e - e0 < 4e-3


def test_fp64_xx_ground_energy_extrapolation(pkg):
    """Two step sizes in one batch; the fixed point's error is linear in tau."""
    with pkg.Itebd([(1.0, 0.0, 0.04), (1.0, 0.0, 0.02)], 16) as c:
        e = c.step(5000).energy()
    ex = 2 * e[1] - e[0]
    assert abs(ex - it.xx_ground_energy(1.0)) < 1e-4


def test_fp64_long_run_stays_normalised(pkg):
    """20000 updates at tau = 0.05 (an unnormalised state would grow by ~e^750):
    finite, and at D_b = 4 (no degenerate cut after the transient) equal to the
    oracle's energy."""
    ref = it.site_energy(it.run(1.0, 1.0, 0.05, 4, 20000), hz.bond_hamiltonian(1.0, 1.0))
    with pkg.Itebd([(1.0, 1.0, 0.05)], 4) as c:
        e = c.step(20000).energy()[0]
    assert np.isfinite(e) and abs(e - ref) < 1e-6


@pytest.mark.parametrize("Jz", [1.0, 2.5])
def test_fp64_ising_limit(pkg, Jz):
    with pkg.Itebd([(0.0, Jz, 0.1)], 4) as c:
        c.step(40)
        assert abs(c.energy()[0] + Jz / 4) < 1e-14
        lam = c.lam(0)
        assert abs(lam[0] - 1.0) < 1e-14 and np.all(np.abs(lam[1:]) < 1e-7)


def test_batch_equals_single_chains(pkg):
    cps = [(1.0, 1.0, 0.05), (1.0, 0.0, 0.1), (0.7, 1.3, 0.08), (1.0, -0.5, 0.05)]
    with pkg.Itebd(cps, 12) as c:
        eb = c.step(60).energy()
        lb = [c.lam(i) for i in range(len(cps))]
    for i, cp in enumerate(cps):
        with pkg.Itebd([cp], 12) as c1:
            e1 = c1.step(60).energy()[0]
            assert e1 == eb[i]
            assert np.array_equal(c1.lam(0), lb[i])
