"""Exact partition functions of small periodic lattices (no truncation).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Two independent routes to Z = Tr T^N (Eq. 2, Sec. II.A) on an Lx x Ly torus in
which every site has four bonds (left, right, down, up; on a length-1 or
length-2 direction a site meets itself or the same neighbour twice, exactly as
the periodic tensor network does):

* ``transfer_matrix_ln_z(B, w, Lx, Ly)`` -- spins with bond matrix B and site
  weight w, by the row-to-row transfer matrix, Z = Tr V^Ly.
* ``network_ln_abs_z(T, Lx, Ly)`` -- any local tensor T[x,x',y,y'], by closing
  each row of Lx tensors into a ring and taking the trace of the Ly-th power
  of the resulting row matrix.

Both are exact up to rounding.  ``oracle/brute_force.c`` enumerates every spin
configuration and pins the first; the second is pinned against the first on
tensors built from (B, w).
"""
from __future__ import annotations

import itertools

import numpy as np


def transfer_matrix_ln_z(B: np.ndarray, w: np.ndarray, Lx: int, Ly: int) -> float:
    """ln Z of the Lx x Ly torus with bond weights B[s,s'] and site weights w[s]."""
    B = np.asarray(B, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    q = B.shape[0]
    rows = list(itertools.product(range(q), repeat=Lx))
    nr = len(rows)
    R = np.ones(nr)
    for r, sig in enumerate(rows):
        for i in range(Lx):
            R[r] *= w[sig[i]] * B[sig[i], sig[(i + 1) % Lx]]
    V = np.ones((nr, nr))
    for r, sig in enumerate(rows):
        for c, sig2 in enumerate(rows):
            for i in range(Lx):
                V[r, c] *= B[sig[i], sig2[i]]
    Tm = R[:, None] * V                       # weight of row r times its bonds to row c
    scale = np.max(np.abs(Tm))
    P = np.eye(nr)
    for _ in range(Ly):
        P = P @ (Tm / scale)
    return float(Ly * np.log(scale) + np.log(np.trace(P)))


def network_ln_abs_z(T: np.ndarray, Lx: int, Ly: int):
    """(ln|Z|, sign Z) of the Lx x Ly periodic network of copies of T[x,x',y,y'].

    Each row of Lx tensors is closed into a ring over its horizontal bonds,
    giving a row matrix from the Lx down legs to the Lx up legs; Z is the trace
    of the Ly-th power of that matrix.
    """
    T = np.asarray(T, dtype=np.float64)
    scale = np.max(np.abs(T))
    t = T / scale
    D, E = t.shape[0], t.shape[2]
    # R[h_first, h_last, down legs..., up legs...] for the first i+1 sites of a row
    R = t.reshape(D, D, E, E)
    for _ in range(1, Lx):
        R = np.einsum("ab...,bcuv->ac...uv", R, t)
    R = np.einsum("aa...->...", R)                     # close the ring (periodic in x)
    # axes are (v0, v0', v1, v1', ...): group the down legs, then the up legs
    perm = list(range(0, 2 * Lx, 2)) + list(range(1, 2 * Lx, 2))
    Rm = R.transpose(perm).reshape(E ** Lx, E ** Lx)
    P = np.eye(E ** Lx)
    for _ in range(Ly):
        P = P @ Rm
    Z = np.trace(P)
    return float(Lx * Ly * np.log(scale) + np.log(abs(Z))), float(np.sign(Z))
