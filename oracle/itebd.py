"""iTEBD for the spin-1/2 XXZ (Heisenberg) chain -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What is computed
----------------
The ground state of the infinite chain H = sum_i h_{i,i+1},
h = Jxy (Sx Sx + Sy Sy) + Jz Sz Sz (the antiferromagnetic Heisenberg chain at
Jxy = Jz = 1, Sec. II.A), as a matrix-product state with a two-site unit cell
(Eq. 1: ... lambda_2 A lambda_1 B lambda_2 ...), reached by imaginary-time
evolution with the two-site gate U = exp(-tau h) applied alternately to the
two kinds of bond; after each gate the bond is cut back to D_b states by an
SVD whose singular values are the new lambda (Sec. II.A).

State and one update (conventions shared with the CUDA library, each side
implementing them on its own):

* The state is (P, Q, lam): P[i, a, j] and Q[j, b, m] are the site tensors of
  the bond being updated in right-canonical form (Gamma lambda), lam[i] the
  Schmidt values on P's left bond; the physical index a, b = 0 (Sz = +1/2) or
  1 (Sz = -1/2), and a two-site index is 2 a + b.
* phi[i, a, b, m] = sum_j P[i, a, j] Q[j, b, m];
  phit[i, a', b', m] = sum_{a b} g[(a' b'), (a b)] phi[i, a, b, m];
  theta = lam[i] phit, viewed as the (D_l d) x (d D_r) matrix M[(i a'), (b' m)].
* M = X S Y^T (SVD); D' = min(D_b, rank); the new Schmidt values are
  S[:D'] / |S[:D']|; Q' = Y[:, :D']^T viewed as [j, b', m]; P' = phit Y[:, :D'] / |S[:D']|
  viewed as [i, a', j] (= Gamma' lambda' without dividing by the old lambda; the
  division by |S[:D']| keeps the state normalised, which the non-unitary
  imaginary-time gate does not: its scale would drift by exp(-tau e) per update).
* The next update acts on the other kind of bond: (P, Q, lam) <- (Q', P', S').

Energy per bond: <theta|h|theta> / <theta|theta> with theta = lam[i] phi (the
bond's two-site wave function in the lambda environment); per site, the mean of
the two bonds' energies.

Pins (tests/test_oracle_itebd.py): exact reconstruction and right-orthonormality
without truncation; the Schmidt values of one gate on a Neel pair against the
gate's closed form; the Neel state as the exact fixed point of the Ising
limit; the ground-state energies of the XX chain (-Jxy / pi, free fermions)
and of the Heisenberg chain (1/4 - ln 2, Bethe ansatz) approached with
growing D_b and shrinking tau; the variational bound.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .heisenberg import bond_gate, bond_hamiltonian

__all__ = ["neel_state", "update", "bond_energy", "site_energy", "ItebdRun", "run",
           "xx_ground_energy", "heisenberg_ground_energy"]


def neel_state():
    """(P, Q, lam) of the Neel product state |up down up down ...> (D = 1)."""
    P = np.zeros((1, 2, 1))
    Q = np.zeros((1, 2, 1))
    P[0, 0, 0] = 1.0
    Q[0, 1, 0] = 1.0
    return P, Q, np.ones(1)


def update(P: np.ndarray, Q: np.ndarray, lam: np.ndarray, g: np.ndarray, D_b: int):
    """One gate on the (P, Q) bond; returns the next state (Q', P', S') and the
    discarded weight sum_{k >= D'} S_k^2 / sum_k S_k^2."""
    Dl, d, _ = P.shape
    Dr = Q.shape[2]
    phi = np.einsum("iaj,jbm->iabm", P, Q)
    phit = np.einsum("ABab,iabm->iABm", g.reshape(d, d, d, d), phi)
    theta = lam[:, None, None, None] * phit
    _, s, Yt = np.linalg.svd(theta.reshape(Dl * d, d * Dr), full_matrices=False)
    Dn = min(D_b, s.size)
    w = s * s
    disc = float(np.sum(w[Dn:]) / np.sum(w))
    Y = Yt[:Dn].T                                       # (d Dr, Dn)
    Qn = Yt[:Dn].reshape(Dn, d, Dr)
    norm = np.linalg.norm(s[:Dn])
    Pn = (phit.reshape(Dl * d, d * Dr) @ Y).reshape(Dl, d, Dn) / norm
    sn = s[:Dn] / norm
    return Qn, Pn, sn, disc


def bond_energy(P: np.ndarray, Q: np.ndarray, lam: np.ndarray, h: np.ndarray) -> float:
    """<theta|h|theta> / <theta|theta>, theta[i, a, b, m] = lam[i] sum_j P Q."""
    d = P.shape[1]
    theta = lam[:, None, None, None] * np.einsum("iaj,jbm->iabm", P, Q)
    htheta = np.einsum("ABab,iabm->iABm", h.reshape(d, d, d, d), theta)
    return float(np.sum(theta * htheta) / np.sum(theta * theta))


@dataclass
class ItebdRun:
    P: np.ndarray
    Q: np.ndarray
    lam: np.ndarray
    lam_other: np.ndarray
    n: int = 0
    disc: list = field(default_factory=list)


def site_energy(st: ItebdRun, h: np.ndarray) -> float:
    """Mean of the two bonds' energies: the current bond (P, Q) with lam, and the
    other bond (Q, P) with the other bond's Schmidt values."""
    return 0.5 * (bond_energy(st.P, st.Q, st.lam, h) + bond_energy(st.Q, st.P, st.lam_other, h))


def run(Jxy: float, Jz: float, tau: float, D_b: int, nsteps: int, state=None) -> ItebdRun:
    """nsteps gate updates from ``state`` (default: the Neel state)."""
    P, Q, lam = state if state is not None else neel_state()
    g = bond_gate(Jxy, Jz, tau)
    st = ItebdRun(P, Q, lam, np.ones(P.shape[2]) / np.sqrt(P.shape[2]))
    for _ in range(nsteps):
        old = st.lam
        Qn, Pn, sn, disc = update(st.P, st.Q, st.lam, g, D_b)
        st.P, st.Q, st.lam, st.lam_other = Qn, Pn, sn, old
        st.n += 1
        st.disc.append(disc)
    return st


def xx_ground_energy(Jxy: float) -> float:
    """Free fermions (Jordan-Wigner, hopping Jxy / 2): e0 = -|Jxy| / pi per site."""
    return -abs(Jxy) / np.pi


def heisenberg_ground_energy(J: float) -> float:
    """Bethe ansatz, isotropic antiferromagnet: e0 = J (1/4 - ln 2) per site."""
    return J * (0.25 - np.log(2.0))
