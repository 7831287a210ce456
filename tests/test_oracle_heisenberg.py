"""Pins of the quantum (XXZ chain) oracle against routes independent of it (CPU only).

Closed-form spectra of the bond Hamiltonian and of small rings, dense 2^L
Trotter products built site by site, exact diagonalisation, the free-fermion
solution of the Trotterised XX chain, the classical Ising chain and the
high-temperature cumulant series.
"""
import math

import numpy as np
import pytest

from oracle import exact, hotrg
from oracle import heisenberg as hz
from workloads import random_tensor

BIG = 10 ** 9  # D_cut that disables truncation
COUPLINGS = [(1.0, 1.0), (1.0, 0.0), (0.0, 1.0), (0.7, -0.3), (-1.0, -1.0)]


# ---------------------------------------------------------------- bond gate

@pytest.mark.parametrize("Jxy,Jz", COUPLINGS)
def test_bond_hamiltonian_spectrum(Jxy, Jz):
    # |uu>, |dd>: Jz/4; (|ud> +- |du>)/sqrt2: +-Jxy/2 - Jz/4
    want = sorted([Jz / 4, Jz / 4, Jxy / 2 - Jz / 4, -Jxy / 2 - Jz / 4])
    assert np.allclose(np.linalg.eigvalsh(hz.bond_hamiltonian(Jxy, Jz)), want, atol=1e-15)


@pytest.mark.parametrize("Jxy,Jz", COUPLINGS)
def test_bond_gate_closed_form_and_semigroup(Jxy, Jz):
    tau = 0.23
    ep = math.exp(-tau * (Jxy / 2 - Jz / 4))    # symmetric Sz = 0 state
    em = math.exp(-tau * (-Jxy / 2 - Jz / 4))   # antisymmetric (singlet) state
    p = math.exp(-tau * Jz / 4)
    want = np.zeros((4, 4))
    want[0, 0] = want[3, 3] = p
    want[1, 1] = want[2, 2] = (ep + em) / 2
    want[1, 2] = want[2, 1] = (ep - em) / 2
    g = hz.bond_gate(Jxy, Jz, tau)
    assert np.allclose(g, want, rtol=0, atol=1e-15)
    assert np.allclose(hz.bond_gate(Jxy, Jz, 0.1) @ hz.bond_gate(Jxy, Jz, 0.13), g,
                       rtol=0, atol=1e-13)


def test_one_site_basis_is_pauli():
    P = hz.one_site_basis()
    sx, sy, sz = hz.spin_operators()
    assert np.array_equal(P[0], np.eye(2))
    assert np.allclose(P[1], 2 * sx) and np.allclose(P[3], 2 * sz)
    assert np.allclose(P[2], 2j * sy)
    # orthogonal under Tr(A^T B) with norm 2
    gram = np.einsum("kab,lab->kl", P, P)
    assert np.array_equal(gram, 2 * np.eye(4))


@pytest.mark.parametrize("Jxy,Jz", COUPLINGS)
def test_gate_factors(Jxy, Jz):
    tau = 0.17
    A, B = hz.gate_factors(Jxy, Jz, tau)
    g = hz.bond_gate(Jxy, Jz, tau)
    assert np.allclose(sum(np.kron(A[k], B[k]) for k in range(4)), g, rtol=0, atol=1e-15)
    # coefficients of I I, X X, E E, Z Z from the gate's closed form
    ep = math.exp(-tau * (Jxy / 2 - Jz / 4))
    em = math.exp(-tau * (-Jxy / 2 - Jz / 4))
    p, u, v = math.exp(-tau * Jz / 4), (ep + em) / 2, (ep - em) / 2
    c = np.array([(p + u) / 2, v / 2, -v / 2, (p - u) / 2])
    P = hz.one_site_basis()
    assert np.allclose(A, np.sqrt(np.abs(c))[:, None, None] * P, rtol=0, atol=1e-13)
    assert np.allclose(B, (np.sign(c) * np.sqrt(np.abs(c)))[:, None, None] * P,
                       rtol=0, atol=1e-13)


# ---------------------------------------------------------------- small rings

def test_ring_ground_states():
    # four- and six-site Heisenberg rings: E0 = -2 J and -(1 + sqrt(13) / 2) J
    for L, e0 in ((4, -2.0), (6, -(1 + math.sqrt(13) / 2))):
        He, Ho = hz.chain_hamiltonians(L, 1.0, 1.0)
        assert abs(np.linalg.eigvalsh(He + Ho).min() - e0) < 1e-13
        assert np.allclose(He @ He @ Ho, He @ (He @ Ho))  # well-formed
    # commuting bonds: H_e is a sum of disjoint bonds, its spectrum is additive
    He, _ = hz.chain_hamiltonians(6, 1.0, 1.0)
    lam = np.linalg.eigvalsh(He)
    assert abs(lam.min() - 3 * (-0.75)) < 1e-13 and abs(lam.max() - 3 * 0.25) < 1e-13


@pytest.mark.parametrize("Jxy,Jz", COUPLINGS)
@pytest.mark.parametrize("L", [2, 4, 6])
def test_cell_network_equals_dense_trotter(Jxy, Jz, L):
    tau = 0.1
    T = hz.cell_tensor(Jxy, Jz, tau)
    for M in (1, 2, 3):
        lnz, sign = exact.network_ln_abs_z(T, L // 2, M)
        assert sign > 0
        assert abs(lnz - hz.trotter_ln_z(L, Jxy, Jz, tau, M)) < 1e-12


def test_trotter_error_is_second_order():
    ex = hz.exact_ln_z(6, 1.0, 1.0, 1.0)
    err = [hz.trotter_ln_z(6, 1.0, 1.0, 1.0 / M, M) - ex for M in (8, 16, 32)]
    assert 3.9 < err[0] / err[1] < 4.1 and 3.9 < err[1] / err[2] < 4.1
    assert abs(err[2]) < 1e-4


# ---------------------------------------------------------------- HOTRG runs

def test_trace_y_closes_the_columns():
    T = random_tensor(3, seed=7, Dy=2)
    Tx, c = hotrg.trace_y(T)
    loop = np.zeros((3, 3))
    for y in range(2):
        loop += T[:, :, y, y]
    assert Tx.shape == (3, 3, 1, 1)
    assert np.allclose(Tx[:, :, 0, 0] * c, loop, rtol=0, atol=1e-15)
    # a ring of Lx closed columns is the Lx x 1 periodic network
    for Lx in (1, 2, 3):
        lnz, _ = exact.network_ln_abs_z(T, Lx, 1)
        P = np.linalg.matrix_power(loop, Lx)
        assert abs(lnz - math.log(abs(np.trace(P)))) < 1e-12


@pytest.mark.parametrize("n_time,n_space", [(2, 1), (1, 2), (0, 2)])
def test_untruncated_run_equals_dense_trotter(n_time, n_space):
    Jxy, Jz, tau = 1.0, 1.0, 0.1
    r = hz.run(hz.cell_tensor(Jxy, Jz, tau), BIG, n_time, n_space)
    L, M = 2 * 2 ** n_space, 2 ** n_time
    ncell = 2 ** (n_time + n_space)
    assert abs(r.ln_z_per_site * ncell - hz.trotter_ln_z(L, Jxy, Jz, tau, M)) < 1e-11


def test_xx_free_fermion_reference():
    # continuum limit tau -> 0 at beta = 1: ln Z / L = (1/2pi) int ln(1 + e^{-beta cos k})
    k = 2 * np.pi * np.arange(4096) / 4096
    cont = 2 * np.mean(np.log1p(np.exp(-np.cos(k))))
    err = [hz.xx_trotter_ln_z_per_cell(1.0, 1.0 / M, M) * M - cont for M in (16, 32)]
    assert 3.9 < err[0] / err[1] < 4.1 and abs(err[1]) < 5e-6
    # a 12-site ring is within finite-size corrections of the infinite chain
    tau, M = 1 / 32, 32
    d = hz.trotter_ln_z(12, 1.0, 0.0, tau, M) / (6 * M)
    assert abs(d - hz.xx_trotter_ln_z_per_cell(1.0, tau, M)) < 2e-9


@pytest.mark.parametrize("n_time,D_cut,tol", [(1, 16, 1e-13), (2, 16, 1e-13), (3, 16, 1e-11)])
def test_xx_chain_thermodynamic_limit(n_time, D_cut, tol):
    tau = 1 / 32
    r = hz.run(hz.cell_tensor(1.0, 0.0, tau), D_cut, n_time, 30)
    assert abs(r.ln_z_per_site - hz.xx_trotter_ln_z_per_cell(1.0, tau, 2 ** n_time)) < tol


def test_open_time_legs_lose_the_entropy():
    """Why the time direction is closed before the chain steps: X steps taken with
    the time legs open truncate the time-boundary states, and for the Ising chain
    (Jxy = 0, beta Jz / 4 = 0.4) only the ground-state term survives,
    ln Z / L = beta Jz / 4 instead of ln(2 cosh(beta Jz / 4))."""
    tau, nt, nx = 0.1, 4, 24
    T0 = hz.cell_tensor(0.0, 1.0, tau)
    opened = hotrg.run(T0, 16, nt + nx, dirs=["y"] * nt + ["x"] * nx).ln_z_per_site
    closed = hz.run(T0, 16, nt, nx).ln_z_per_site
    beta, M = tau * 2 ** nt, 2 ** nt
    assert abs(closed - hz.ising_chain_ln_z_per_cell(1.0, beta, M)) < 1e-13
    assert abs(opened * M / 2 - beta / 4) < 1e-6            # per site: ground state only
    assert closed - opened > 0.04                            # the missing entropy per cell


@pytest.mark.parametrize("Jz", [1.0, -1.0, 2.5])
def test_ising_chain_limit(Jz):
    tau, nt = 0.1, 4
    r = hz.run(hz.cell_tensor(0.0, Jz, tau), 16, nt, 30)
    want = hz.ising_chain_ln_z_per_cell(Jz, tau * 2 ** nt, 2 ** nt)
    assert abs(r.ln_z_per_site - want) < 1e-13


def test_high_t_cumulants_from_dense_traces():
    He, Ho = hz.chain_hamiltonians(8, 1.0, 1.0)
    H = He + Ho
    d, L = 2 ** 8, 8
    H2 = H @ H
    m2, m3, m4 = np.trace(H2) / d, np.trace(H2 @ H) / d, np.trace(H2 @ H2) / d
    assert abs(np.trace(H) / d) < 1e-15
    assert abs(m2 / L - 3 / 16) < 1e-14
    assert abs(m3 / L + 3 / 32) < 1e-14
    assert abs((m4 - 3 * m2 * m2) / L + 15 / 128) < 1e-13


@pytest.mark.parametrize("beta", [0.05, 0.1, 0.2])
def test_heisenberg_high_t_series(beta):
    nt = 6
    tau = beta / 2 ** nt
    r = hz.run(hz.cell_tensor(1.0, 1.0, tau), 16, nt, 30)
    per_site = r.ln_z_per_site / (2 * tau) * beta          # (ln Z / N_cells) M / 2
    assert abs(per_site - hz.heisenberg_high_t_ln_z_per_site(1.0, beta)) < 0.01 * beta ** 5


def test_heisenberg_matches_dense_ring():
    tau, nt = 1 / 32, 4
    r = hz.run(hz.cell_tensor(1.0, 1.0, tau), 24, nt, 30)
    d = hz.trotter_ln_z(12, 1.0, 1.0, tau, 2 ** nt) / (6 * 2 ** nt)
    assert abs(r.ln_z_per_site - d) < 1e-8


def test_heisenberg_low_t_energy():
    # f -> e0 = 1/4 - ln 2 (Bethe ansatz) as T -> 0, with f - e0 = -T^2/3 + ...
    tau, nt = 1 / 32, 9                                      # beta = 16
    r = hz.run(hz.cell_tensor(1.0, 1.0, tau), 24, nt, 30)
    f = hz.free_energy_per_site(r.ln_z_per_site, tau)
    e0 = 0.25 - math.log(2.0)
    assert abs(f - (e0 - (1 / 16) ** 2 / 3)) < 2e-3
