"""Pins of the iTEBD oracle against routes independent of it (CPU only):
exact identities of one update without truncation, the closed-form Schmidt
values of one gate on a Neel pair, the Ising-limit fixed point, and the exact
ground-state energies of the XX (free fermions) and Heisenberg (Bethe ansatz)
chains, approached as D_b grows and tau -> 0."""
import math

import numpy as np
import pytest

from oracle import heisenberg as hz
from oracle import itebd as it
from workloads import random_mps


def test_update_without_truncation_is_exact():
    P, Q, lam = random_mps(3, seed=11)
    g = hz.bond_gate(1.0, 0.7, 0.1)
    Qn, Pn, sn, disc = it.update(P, Q, lam, g, D_b=6)          # d D = 6: nothing cut
    phi = np.einsum("iaj,jbm->iabm", P, Q)
    phit = np.einsum("ABab,iabm->iABm", g.reshape(2, 2, 2, 2), phi).reshape(6, 6)
    assert disc == 0.0 or disc < 1e-28
    s_full = np.linalg.svd((lam[:, None, None] * phit.reshape(3, 2, 6)).reshape(6, 6), compute_uv=False)
    norm = np.linalg.norm(s_full)                                # the state is renormalised
    assert np.allclose(Pn.reshape(6, -1) @ Qn.reshape(Qn.shape[0], -1) * norm, phit, rtol=0, atol=1e-13)
    Qm = Qn.reshape(Qn.shape[0], -1)
    assert np.allclose(Qm @ Qm.T, np.eye(Qm.shape[0]), rtol=0, atol=1e-14)   # right-canonical
    assert abs(np.sum(sn * sn) - 1.0) < 1e-15 and np.all(np.diff(sn) <= 0)
    # the Schmidt values are the singular values of the lam-weighted gated pair
    assert np.allclose(sn, s_full / norm, rtol=0, atol=1e-14)


@pytest.mark.parametrize("Jxy,Jz,tau", [(1.0, 1.0, 0.1), (1.0, 0.0, 0.3), (0.7, -0.3, 0.2)])
def test_neel_pair_schmidt_values(Jxy, Jz, tau):
    # U |up down> = u |up down> + v |down up>, u, v from the spectrum of h on the Sz = 0 pair
    es = math.exp(-tau * (Jxy / 2 - Jz / 4))
    ea = math.exp(-tau * (-Jxy / 2 - Jz / 4))
    u, v = (es + ea) / 2, (es - ea) / 2
    want = np.sort(np.abs([u, v]))[::-1] / math.hypot(u, v)
    P, Q, lam = it.neel_state()
    _, _, sn, _ = it.update(P, Q, lam, hz.bond_gate(Jxy, Jz, tau), D_b=4)
    assert np.allclose(sn[:2], want, rtol=0, atol=1e-15)
    assert np.all(np.abs(sn[2:]) < 1e-15)


@pytest.mark.parametrize("Jxy", [0.0, 1.0, -0.4])
def test_bond_energy_of_neel_pair(Jxy):
    P, Q, lam = it.neel_state()
    for Jz in (1.0, -2.0):
        assert abs(it.bond_energy(P, Q, lam, hz.bond_hamiltonian(Jxy, Jz)) + Jz / 4) < 1e-15


@pytest.mark.parametrize("Jz", [1.0, 2.5])
def test_ising_limit_neel_is_fixed_point(Jz):
    st = it.run(0.0, Jz, 0.1, 4, 40)
    assert abs(it.site_energy(st, hz.bond_hamiltonian(0.0, Jz)) + Jz / 4) < 1e-14
    assert abs(st.lam[0] - 1.0) < 1e-14 and np.all(np.abs(st.lam[1:]) < 1e-14)


def extrapolated(Jxy, Jz, D):
    h = hz.bond_hamiltonian(Jxy, Jz)
    e1 = it.site_energy(it.run(Jxy, Jz, 0.04, D, 2500), h)
    e2 = it.site_energy(it.run(Jxy, Jz, 0.02, D, 5000), h)
    return e1, e2, 2 * e2 - e1          # the fixed point's error is linear in tau


@pytest.mark.parametrize("Jxy,Jz,exact", [(1.0, 1.0, it.heisenberg_ground_energy(1.0)),
                                           (1.0, 0.0, it.xx_ground_energy(1.0))])
def test_ground_energy_limits(Jxy, Jz, exact):
    e1, e2, ex8 = extrapolated(Jxy, Jz, 8)
    _, _, ex16 = extrapolated(Jxy, Jz, 16)
    assert exact < e2 < e1                          # above the ground state, falling with tau
    assert abs(ex8 - exact) < 6e-4
    assert abs(ex16 - exact) < 1e-4 and abs(ex16 - exact) < abs(ex8 - exact)


def test_state_stays_normalised_over_long_runs():
    # 20000 updates at tau = 0.05 would scale an unnormalised state by ~exp(750)
    st = it.run(1.0, 1.0, 0.05, 4, 20000)
    assert np.all(np.isfinite(st.P)) and np.all(np.isfinite(st.Q))
    assert 1e-3 < np.linalg.norm(st.P) < 1e3


def _update_via_density_matrix(P, Q, lam, g, D_b):
    """The same update with the SVD taken from the eigendecomposition of theta^T theta
    (the bond's right density matrix: the Hermitian route of the GPU path)."""
    Dl, d, _ = P.shape
    Dr = Q.shape[2]
    phit = np.einsum("ABab,iabm->iABm", g.reshape(d, d, d, d), np.einsum("iaj,jbm->iabm", P, Q))
    theta = (lam[:, None, None, None] * phit).reshape(Dl * d, d * Dr)
    w, V = np.linalg.eigh(theta.T @ theta)
    w, V = np.maximum(w[::-1], 0.0), V[:, ::-1]
    Dn = min(D_b, w.size)
    s = np.sqrt(w[:Dn])
    norm = np.linalg.norm(s)
    Y = V[:, :Dn]
    return (Y.T.reshape(Dn, d, Dr), (phit.reshape(Dl * d, d * Dr) @ Y).reshape(Dl, d, Dn) / norm,
            s / norm)


def test_density_matrix_route_matches_svd_route():
    # 1500 updates from the Neel state at D_b = 16: the two routes to the Schmidt
    # decomposition give the same energy to well below the truncation level
    g = hz.bond_gate(1.0, 1.0, 0.05)
    h = hz.bond_hamiltonian(1.0, 1.0)
    st = it.run(1.0, 1.0, 0.05, 16, 1500)
    P, Q, lam = it.neel_state()
    other = np.ones(1)
    for _ in range(1500):
        old = lam
        P, Q, lam = _update_via_density_matrix(P, Q, lam, g, 16)
        other = old
    e_gram = 0.5 * (it.bond_energy(P, Q, lam, h) + it.bond_energy(Q, P, other, h))
    assert abs(e_gram - it.site_energy(st, h)) < 1e-8


def test_energy_falls_with_bond_dimension():
    h = hz.bond_hamiltonian(1.0, 1.0)
    es = [it.site_energy(it.run(1.0, 1.0, 0.05, D, 1500), h) for D in (2, 4, 8, 16)]
    assert all(a > b for a, b in zip(es, es[1:]))
    assert es[-1] > it.heisenberg_ground_energy(1.0)
