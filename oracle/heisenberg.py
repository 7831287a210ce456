"""Quantum HOTRG for the spin-1/2 XXZ (Heisenberg) chain -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What is computed
----------------
The finite-temperature partition function Z = Tr exp(-beta H) of the chain

    H = sum_i h_{i,i+1},   h = Jxy (Sx Sx + Sy Sy) + Jz Sz Sz

(Jxy = Jz = J > 0: the antiferromagnetic Heisenberg chain of Sec. II.A; the
paper notes that other models follow by changing H) is mapped onto a 2D
classical network with an extra imaginary-time direction (Sec. II.B): the
bonds are split into even and odd ones, H = H_e + H_o, and the checkerboard
Trotter product

    Z_M = Tr (exp(-tau H_o) exp(-tau H_e))^M,   beta = M tau,

is written as the contraction of a periodic network of identical cell tensors,
one cell being two neighbouring sites (even site e, odd site o) over one period
of imaginary time.  HOTRG steps along the time direction (Y) compose the
imaginary-time evolution; once beta is reached the time direction is closed by
a trace over its leg pair, and steps along the chain (X) then take the
product of column matrices to the thermodynamic limit.

Cell tensor (conventions shared with the CUDA library's initial tensor, each
side computing it on its own):

* Spin states s = 0 (Sz = +1/2), 1 (Sz = -1/2); a two-site state of sites (a, b)
  has index 2 s_a + s_b.  The bond gate is g = exp(-tau h) as a 4 x 4 matrix
  g[out, in].
* g is expanded in products of the real one-site basis
  P = (I, X, E, Z) with X = sigma_x, E = [[0, 1], [-1, 0]] (= i sigma_y),
  Z = sigma_z:  g = sum_k c_k P_k (x) P_k, the coefficients
  c_k = Tr((P_k (x) P_k)^T g) / 4 of the Hilbert-Schmidt projection (the
  U(1) x Z2 symmetry of h makes all mixed products P_k (x) P_l, k != l, vanish).
  The left site of a bond receives A_k = sqrt|c_k| P_k and the right site
  B_k = sign(c_k) sqrt|c_k| P_k, joined by a virtual bond k of dimension 4.
* T[x, x', y, y'] with y = 2 e + o the two spins at the start of the period and
  y' at its end: the even-bond gate acts first inside the cell, then the two
  odd bonds that leave the cell act through B_x on e (left leg) and A_x' on o
  (right leg):

      T[x, x', (e0 o0), (e2 o2)] = sum_{e1, o1} g[(e1 o1), (e0 o0)] B_x[e2, e1] A_x'[o2, o1]

  The x' leg of a cell contracted with the x leg of its right neighbour gives
  sum_k A_k[o2, o1] B_k[e2', e1'] = g[(o2 e2'), (o1 e1')], the odd-bond gate.

A network of Lx x Ly cells (periodic both ways) is Z_M of a periodic chain of
L = 2 Lx sites with M = Ly.  After n_t Y steps, the time trace and n_x X
steps, ln Z / N_cells comes out of ``hotrg.HotrgRun.ln_z_per_site`` unchanged;
per site and with beta = 2^n_t tau, f = -(ln Z / N_cells) / (2 tau).

Pins (tests/test_oracle_heisenberg.py): the gate against the singlet / triplet
spectrum of h and the semigroup law; the cell network against dense 2^L
Trotter products built from Kronecker products; the Trotter limit against
exact diagonalisation (error O(tau^2)); untruncated HOTRG on a finite torus
against the network; truncated HOTRG in the thermodynamic limit against the
free-fermion solution of the Trotterised XX chain (Jz = 0), the classical
Ising chain (Jxy = 0) and the high-temperature series of the Heisenberg chain.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import hotrg

__all__ = [
    "one_site_basis", "spin_operators", "bond_hamiltonian", "bond_gate",
    "gate_coefficients", "gate_factors", "cell_tensor", "chain_hamiltonians",
    "trotter_ln_z", "exact_ln_z", "run", "free_energy_per_site",
    "xx_trotter_ln_z_per_cell", "ising_chain_ln_z_per_cell",
    "heisenberg_high_t_ln_z_per_site",
]


def one_site_basis() -> np.ndarray:
    """(I, X, E, Z): the real one-site operator basis, shape (4, 2, 2)."""
    return np.array([
        [[1.0, 0.0], [0.0, 1.0]],
        [[0.0, 1.0], [1.0, 0.0]],
        [[0.0, 1.0], [-1.0, 0.0]],
        [[1.0, 0.0], [0.0, -1.0]],
    ])


def spin_operators():
    """Complex spin-1/2 operators (Sx, Sy, Sz) in the basis (up, down)."""
    sx = np.array([[0, 1], [1, 0]], dtype=complex) / 2
    sy = np.array([[0, -1j], [1j, 0]], dtype=complex) / 2
    sz = np.array([[1, 0], [0, -1]], dtype=complex) / 2
    return sx, sy, sz


def bond_hamiltonian(Jxy: float, Jz: float) -> np.ndarray:
    """h = Jxy (Sx Sx + Sy Sy) + Jz Sz Sz on two sites (4 x 4, real)."""
    sx, sy, sz = spin_operators()
    h = Jxy * (np.kron(sx, sx) + np.kron(sy, sy)) + Jz * np.kron(sz, sz)
    assert np.max(np.abs(h.imag)) == 0.0
    return h.real.copy()


def bond_gate(Jxy: float, Jz: float, tau: float) -> np.ndarray:
    """g = exp(-tau h), from the eigendecomposition of the symmetric h."""
    lam, V = np.linalg.eigh(bond_hamiltonian(Jxy, Jz))
    return (V * np.exp(-tau * lam)) @ V.T


def gate_coefficients(g: np.ndarray) -> np.ndarray:
    """C[k, l] = Tr((P_k (x) P_l)^T g) / 4 over the real basis (I, X, E, Z)."""
    P = one_site_basis()
    C = np.empty((4, 4))
    for k in range(4):
        for l in range(4):
            C[k, l] = np.trace(np.kron(P[k], P[l]).T @ g) / 4.0
    return C


def gate_factors(Jxy: float, Jz: float, tau: float):
    """(A, B), each (4, 2, 2): g = sum_k A_k (x) B_k with the sign on B."""
    C = gate_coefficients(bond_gate(Jxy, Jz, tau))
    off = C - np.diag(np.diag(C))
    if np.max(np.abs(off)) > 1e-14 * np.max(np.abs(C)):
        raise ValueError("gate has mixed products in the one-site basis")
    c = np.diag(C)
    P = one_site_basis()
    r = np.sqrt(np.abs(c))
    A = r[:, None, None] * P
    B = (np.sign(c) * r)[:, None, None] * P
    return A, B


def cell_tensor(Jxy: float, Jz: float, tau: float) -> np.ndarray:
    """T[x, x', y, y'] of one two-site cell over one Trotter period, (4, 4, 4, 4)."""
    g = bond_gate(Jxy, Jz, tau).reshape(2, 2, 2, 2)        # g[e1, o1, e0, o0]
    A, B = gate_factors(Jxy, Jz, tau)
    T = np.einsum("mnab,xcm,ydn->xyabcd", g, B, A)           # [x, x', e0, o0, e2, o2]
    return T.reshape(4, 4, 4, 4)


# --------------------------------------------------------------------------
# dense references for small chains
# --------------------------------------------------------------------------

def _bond_term(L: int, i: int, h: np.ndarray) -> np.ndarray:
    """h acting on sites (i, i+1 mod L) of an L-site chain (site 0 slowest)."""
    j = (i + 1) % L
    h4 = h.reshape(2, 2, 2, 2)
    out = np.zeros((2 ** L, 2 ** L))
    for col in range(2 ** L):
        bits = [(col >> (L - 1 - s)) & 1 for s in range(L)]
        for a in range(2):
            for b in range(2):
                v = h4[a, b, bits[i], bits[j]]
                if v != 0.0:
                    nb = list(bits)
                    nb[i], nb[j] = a, b
                    row = int("".join(map(str, nb)), 2)
                    out[row, col] += v
    return out


def chain_hamiltonians(L: int, Jxy: float, Jz: float):
    """(H_e, H_o) of the periodic L-site chain (L even): bonds (2m, 2m+1) and
    (2m+1, 2m+2 mod L)."""
    if L < 2 or L % 2:
        raise ValueError("L must be even and >= 2")
    h = bond_hamiltonian(Jxy, Jz)
    He = sum(_bond_term(L, i, h) for i in range(0, L, 2))
    Ho = sum(_bond_term(L, i, h) for i in range(1, L, 2))
    return He, Ho


def trotter_ln_z(L: int, Jxy: float, Jz: float, tau: float, M: int) -> float:
    """ln Tr (exp(-tau H_o) exp(-tau H_e))^M of the periodic L-site chain."""
    He, Ho = chain_hamiltonians(L, Jxy, Jz)
    V = scipy.linalg.expm(-tau * Ho) @ scipy.linalg.expm(-tau * He)
    s = np.max(np.abs(V))
    P = np.linalg.matrix_power(V / s, M)
    return float(M * np.log(s) + np.log(np.trace(P)))


def exact_ln_z(L: int, Jxy: float, Jz: float, beta: float) -> float:
    """ln Tr exp(-beta H) of the periodic L-site chain by exact diagonalisation."""
    He, Ho = chain_hamiltonians(L, Jxy, Jz)
    E = np.linalg.eigvalsh(He + Ho)
    e0 = E.min()
    return float(-beta * e0 + np.log(np.sum(np.exp(-beta * (E - e0)))))


# --------------------------------------------------------------------------
# HOTRG run and thermodynamics
# --------------------------------------------------------------------------

def run(T0: np.ndarray, D_cut: int, n_time: int, n_space: int) -> hotrg.HotrgRun:
    """n_time Y steps along imaginary time (beta = 2^n_time tau), then the time
    direction is closed by a trace (``hotrg.trace_y``: Z_M is a trace over the
    time-boundary states, which carry an extensive entropy at finite
    temperature and so cannot be truncated), then n_space X steps take the
    chain of column matrices to the thermodynamic limit (Tr T_x^(2^n_space))."""
    st = hotrg.run(T0, D_cut, n_time, dirs=["y"] * n_time)
    st.T, c = hotrg.trace_y(st.T)
    st.logsum += np.log(c) / 2.0 ** st.n
    for _ in range(n_space):
        st.T, c, _, info = hotrg.x_step(st.T, D_cut)
        st.n += 1
        st.logsum += np.log(c) / 2.0 ** st.n
        st.steps.append(info)
    return st


def free_energy_per_site(ln_z_per_cell: float, tau: float) -> float:
    """f = -ln Z / (beta L) = -(ln Z / N_cells) / (2 tau)."""
    return -ln_z_per_cell / (2.0 * tau)


def xx_trotter_ln_z_per_cell(Jxy: float, tau: float, M: int, nq: int = 4096) -> float:
    """Thermodynamic-limit ln Z_M / N_cells of the Trotterised XX chain (Jz = 0).

    Jordan-Wigner maps Jxy (Sx Sx + Sy Sy) to free fermions hopping with
    amplitude t = Jxy / 2; with a two-site cell of momentum q the even and odd
    bonds act on (a_q, b_q) as h_e = [[0, t], [t, 0]] and
    h_o = [[0, t e^{-iq}], [t e^{iq}, 0]].  The trace of a product of Gaussian
    operators is det(1 + product of their one-particle matrices), so
    ln Z_M / N_cells = (1 / M) (1 / 2 pi) int dq ln det(1 + V(q)^M),
    V = exp(-tau h_o) exp(-tau h_e).  The periodic integrand is integrated by
    the trapezoidal rule on nq points.
    """
    t = Jxy / 2.0
    acc = 0.0
    for q in 2.0 * np.pi * np.arange(nq) / nq:
        he = np.array([[0.0, t], [t, 0.0]], dtype=complex)
        ho = np.array([[0.0, t * np.exp(-1j * q)], [t * np.exp(1j * q), 0.0]])
        V = scipy.linalg.expm(-tau * ho) @ scipy.linalg.expm(-tau * he)
        mu = np.linalg.eigvals(V).real
        acc += float(np.sum(np.logaddexp(0.0, M * np.log(mu))))
    return acc / nq / M


def ising_chain_ln_z_per_cell(Jz: float, beta: float, M: int) -> float:
    """Jxy = 0: commuting Ising bonds Jz Sz Sz, so the Trotter product is exact
    and ln Z / L = ln(2 cosh(beta Jz / 4)) in the thermodynamic limit (transfer
    matrix of the classical chain with coupling beta Jz / 4); per cell that is
    2 ln(2 cosh(beta Jz / 4)) / M."""
    return 2.0 * np.log(2.0 * np.cosh(beta * Jz / 4.0)) / M


def heisenberg_high_t_ln_z_per_site(J: float, beta: float) -> float:
    """ln Z / L = ln 2 + (3/32) x^2 + (1/64) x^3 - (5/1024) x^4 + O(x^5), x = beta J,
    for the isotropic chain: the cumulant expansion of ln Tr exp(-beta H) about
    infinite temperature, sum_n kappa_n (-beta)^n / n!, with Tr over 2^L states.
    Per site, kappa_2 = <h^2> = 3 J^2 / 16 and kappa_3 = <h^3> = -3 J^3 / 32
    (h has eigenvalues J/4 (x3) and -3J/4; a product of different bonds with a
    site that appears once averages to zero), and kappa_4 = -15 J^4 / 128 (the
    connected products of up to four bonds, which span at most five sites, so
    that any ring of six or more sites gives the per-site value exactly)."""
    x = beta * J
    return float(np.log(2.0) + 3.0 * x * x / 32.0 + x ** 3 / 64.0 - 5.0 * x ** 4 / 1024.0)
