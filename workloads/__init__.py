"""Seeded synthetic workloads shared by the tests, ``smoke()`` and ``bench.py``.

This module holds only workload *parameters* and seeded random draws; it holds
none of the method's arithmetic (no initial-tensor construction, no
contraction), so that the oracle and the CUDA library, which both consume it,
stay independent of each other.

The five model configurations are the ones the benchmarks are quoted on:

* ``ising_bc_d8``     -- Ising, beta_c = ln(1+sqrt 2)/2, h = 0, D_cut = 8, 20 steps, FP64
* ``ising_044_d32``   -- Ising, beta = 0.44, h = 0, D_cut = 32, 30 steps (FP64 vs TF32)
* ``ising_044h_d48``  -- Ising, beta = 0.44, h = 0.01, D_cut = 48, 30 steps, split BF16
* ``sweep256``        -- 256 Ising instances, beta ~ U[0.35, 0.55], D_cut in
                         {16, 24, 32, 40} (64 each, shuffled), 25 steps, TF32
* ``potts3_d64``      -- q = 3 Potts, beta = ln(1 + sqrt 3), D_cut = 64, 30 steps, split BF16

All directions alternate starting with X.  Random draws use
``numpy.random.default_rng(SEED)``.

Quantum chains (``QUANTUM_CONFIGS``): the antiferromagnetic Heisenberg chain,
tau = 1/32, 7 imaginary-time steps (beta = 4), 16 chain steps, D_cut in
{8, 16, 32, 64}, exact-slice (FP64-grade) contractions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED = 20260205


@dataclass(frozen=True)
class Model:
    """One HOTRG instance: model family, coupling, field, cut and step count."""
    name: str
    family: str          # 'ising' or 'potts'
    beta: float
    h: float = 0.0
    q: int = 2
    D_cut: int = 8
    steps: int = 20
    precision: str = "fp64"   # 'fp64' | 'tf32' | 'bf16x3' | 'bf16x6'


BETA_C_ISING = 0.5 * math.log(1.0 + math.sqrt(2.0))
BETA_C_POTTS3 = math.log(1.0 + math.sqrt(3.0))

CONFIGS = {
    "ising_bc_d8": Model("ising_bc_d8", "ising", BETA_C_ISING, 0.0, 2, 8, 20, "fp64"),
    "ising_044_d32": Model("ising_044_d32", "ising", 0.44, 0.0, 2, 32, 30, "tf32"),
    "ising_044h_d48": Model("ising_044h_d48", "ising", 0.44, 0.01, 2, 48, 30, "bf16x3"),
    "potts3_d64": Model("potts3_d64", "potts", BETA_C_POTTS3, 0.0, 3, 64, 30, "bf16x3"),
}


@dataclass(frozen=True)
class QuantumChain:
    """Finite-temperature quantum HOTRG of the spin-1/2 XXZ chain: the
    Trotterised two-site cell tensor with step tau, n_time Y steps along
    imaginary time (beta = 2^n_time tau), the time trace, n_space X steps."""
    name: str
    Jxy: float
    Jz: float
    tau: float
    n_time: int
    n_space: int
    D_cut: int
    precision: str = "bf16xs"

    @property
    def beta(self) -> float:
        return self.tau * 2 ** self.n_time


# The antiferromagnetic Heisenberg chain (Jxy = Jz = 1) at beta = 4 with
# tau = 1/32; the update-step timings sweep the bond dimension D_cut.
QUANTUM_CONFIGS = {
    f"heisenberg_b4_d{D}": QuantumChain(f"heisenberg_b4_d{D}", 1.0, 1.0, 1 / 32, 7, 16, D, "bf16xs")
    for D in (8, 16, 32, 64)
}


def sweep256(seed: int = SEED, n: int = 256, cuts=(16, 24, 32, 40), steps: int = 25):
    """The batched beta sweep: n Ising instances with seeded beta and D_cut."""
    rng = np.random.default_rng(seed)
    betas = rng.uniform(0.35, 0.55, size=n)
    dcuts = np.repeat(np.asarray(cuts), n // len(cuts))
    rng.shuffle(dcuts)
    return [Model(f"sweep_{i}", "ising", float(b), 0.0, 2, int(d), steps, "tf32")
            for i, (b, d) in enumerate(zip(betas, dcuts))]


def sweep_subset(per_group: int = 4, seed: int = SEED):
    """The first `per_group` instances of every cut group of ``sweep256`` (in
    creation order): a seeded subset of the batched sweep small enough for the
    oracle, with all four cut groups."""
    seen = {}
    out = []
    for m in sweep256(seed):
        if seen.get(m.D_cut, 0) < per_group:
            seen[m.D_cut] = seen.get(m.D_cut, 0) + 1
            out.append(m)
    return out


def random_tensor(D0: int, seed: int = SEED, Dy: int | None = None) -> np.ndarray:
    """I.i.d. U[0,1) tensor T[x,x',y,y'] of shape (D0, D0, Dy, Dy) (stress input)."""
    rng = np.random.default_rng(seed)
    Dy = D0 if Dy is None else Dy
    return rng.random((D0, D0, Dy, Dy))


def random_mps(D: int, d: int = 2, seed: int = SEED):
    """Seeded random two-site-cell MPS state (P, Q, lam): P, Q i.i.d. N(0, 1) of
    shape (D, d, D), lam positive, descending, with sum lam^2 = 1."""
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((D, d, D))
    Q = rng.standard_normal((D, d, D))
    lam = np.sort(rng.uniform(0.1, 1.0, size=D))[::-1]
    return P, Q, lam / np.linalg.norm(lam)


def random_orthogonal(n: int, seed: int = SEED) -> np.ndarray:
    """Haar-random orthogonal matrix (QR of a Gaussian matrix, sign-fixed)."""
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))
