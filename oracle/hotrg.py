"""Plain FP64 NumPy HOTRG -- the oracle for the CUDA path.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What the method computes
------------------------
The partition function of a 2D classical spin model is written as the full
contraction of N copies of a local tensor, Z = Tr T^N (Eq. 2, Sec. II.A).  HOTRG
coarse-grains that network: two neighbouring tensors are contracted along one
bond, the two parallel legs that result are fused, and each fused leg is cut
back to at most ``D_cut`` states by a higher-order SVD that reduces to the SVD of
a reshaped matrix (Sec. II.A) -- here the eigendecomposition of its Hermitian
Gram matrix ``M M^T`` (the Hermitian case of Eq. 5).  Repeating this along
alternating directions doubles the number of sites per step.

Conventions (also used by the CUDA library, each side implementing them on
its own):

* ``T[x, x', y, y']`` = legs (left, right, down, up); ``T.shape = (Dx, Dx, Dy, Dy)``.
* A **Y step** contracts the up leg of a lower tensor ``T1`` with the down leg of
  an upper tensor ``T2``::

      M[x1,x2,x1',x2',y,y'] = sum_k T[x1,x1',y,k] T[x2,x2',k,y']

  fuses (x1,x2) -> X and (x1',x2') -> X' with x1 the slower index, and projects
  both with the same isometry ``U`` (Dx^2 x D')::

      T'[a,b,y,y'] = sum U[(x1 x2),a] M[x1,x2,x1',x2',y,y'] U[(x1' x2'),b]

* ``U`` holds the leading D' = min(Dx^2, D_cut) eigenvectors of the left Gram
  matrix ``G_L = M_(X) M_(X)^T`` or of the right one ``G_R = M_(X') M_(X')^T``,
  whichever discards less weight ``eps = sum_{i > D'} lambda_i`` (ties -> left).
  When Dx^2 <= D_cut nothing is cut: ``U`` is the identity.
* An **X step** is a Y step on the view ``T[y, y', x, x']`` with the result viewed
  back; no other code path exists for it.
* After every step ``c = max |T'|``, ``T' /= c``; the initial tensor is scaled by
  ``c_0 = max |T0|`` as well.  With ``logsum = sum_j ln(c_j) / 2^j``,
  ``ln Z / N = logsum + ln(Tr T_n) / 2^n`` where ``Tr`` is the periodic trace over
  both leg pairs and ``N = 2^n`` sites.

Pins (tests/test_oracle_*.py): exact transfer-matrix and brute-force Z of small
tori with truncation switched off (also for random non-symmetric tensors, where
an independent ``einsum`` of the whole network is the reference); Onsager's
closed form at h = 0 with truncation on; the definition of the environment as
an SVD of the explicitly formed unfolding of M on small random tensors; the
Potts q = 2 / Ising mapping; W W = B for the initial tensor; f(h) = f(-h);
beta -> 0 limit; invariance under an invertible gauge of the legs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "sqrtm_psd", "initial_tensor", "ising_initial_tensor", "potts_initial_tensor",
    "gram_environments", "eigh_desc", "y_step", "x_step", "HotrgRun", "run",
    "periodic_trace", "trace_y", "directions",
]


# --------------------------------------------------------------------------
# a0: initial tensor
# --------------------------------------------------------------------------

def sqrtm_psd(B: np.ndarray) -> np.ndarray:
    """Symmetric square root of a symmetric positive definite matrix via eigh."""
    B = np.asarray(B, dtype=np.float64)
    lam, V = np.linalg.eigh(B)
    if lam.min() <= 0.0:
        raise ValueError("bond Boltzmann matrix is not positive definite")
    return (V * np.sqrt(lam)) @ V.T


def initial_tensor(B: np.ndarray, w: np.ndarray) -> np.ndarray:
    """T0[x,x',y,y'] = sum_s w_s W[s,x] W[s,x'] W[s,y] W[s,y'],  W = sqrt(B).

    Each bond weight B[s,s'] = sum_x W[s,x] W[x,s'] is split evenly between the
    two sites it joins, so that contracting the tensors of all sites (Eq. 2)
    gives Z = sum_config prod_sites w_s prod_bonds B[s_i, s_j].
    """
    W = sqrtm_psd(B)
    w = np.asarray(w, dtype=np.float64)
    return np.einsum("s,sa,sb,sc,sd->abcd", w, W, W, W, W)


def ising_initial_tensor(beta: float, h: float = 0.0) -> np.ndarray:
    """Ising model H = -sum_<ij> s_i s_j - h sum_i s_i (J = 1), s = +1, -1.

    Bond matrix B[s,s'] = exp(beta s s'), site weight w_s = exp(beta h s); index 0
    is s = +1 and index 1 is s = -1.
    """
    s = np.array([1.0, -1.0])
    return initial_tensor(np.exp(beta * np.outer(s, s)), np.exp(beta * h * s))


def potts_initial_tensor(q: int, beta: float) -> np.ndarray:
    """q-state Potts model H = -sum_<ij> delta(s_i, s_j) (J = 1), no field.

    Bond matrix B[s,s'] = exp(beta delta_{ss'}), site weight 1.
    """
    return initial_tensor(np.exp(beta * np.eye(q)), np.ones(q))


# --------------------------------------------------------------------------
# a2/a3: environments (Gram matrices of the two unfoldings of M)
# --------------------------------------------------------------------------

def gram_environments(T: np.ndarray):
    """Left and right Gram matrices of M for a Y step, each (Dx^2, Dx^2).

    G_L[(x1 x2),(u1 u2)] = sum_{x1',x2',y,y'} M[x1,x2,x1',x2',y,y'] M[u1,u2,x1',x2',y,y']
    G_R[(x1'x2'),(u1'u2')] = sum_{x1,x2,y,y'}  M[x1,x2,x1',x2',y,y'] M[x1,x2,u1',u2',y,y']

    Both are evaluated without forming M, by regrouping the sums:
    ``G_L = sum_{k,k'} A_L[x1,k,u1,k'] B_L[x2,k,u2,k']`` with
    ``A_L = sum_{x1',y} T[x1,x1',y,k] T[u1,x1',y,k']`` and
    ``B_L = sum_{x2',y'} T[x2,x2',k,y'] T[u2,x2',k',y']`` (and the same over the
    unprimed legs for the right side).  The regrouping is exact algebra; the
    tests check it against the SVD of the explicitly formed unfolding of M.
    """
    Dx = T.shape[0]
    A_L = np.tensordot(T, T, axes=([1, 2], [1, 2]))            # [x1,k,u1,k']
    B_L = np.tensordot(T, T, axes=([1, 3], [1, 3]))            # [x2,k,u2,k']
    G_L = np.tensordot(A_L, B_L, axes=([1, 3], [1, 3]))        # [x1,u1,x2,u2]
    G_L = G_L.transpose(0, 2, 1, 3).reshape(Dx * Dx, Dx * Dx)
    A_R = np.tensordot(T, T, axes=([0, 2], [0, 2]))            # [x1',k,u1',k']
    B_R = np.tensordot(T, T, axes=([0, 3], [0, 3]))            # [x2',k,u2',k']
    G_R = np.tensordot(A_R, B_R, axes=([1, 3], [1, 3]))        # [x1',u1',x2',u2']
    G_R = G_R.transpose(0, 2, 1, 3).reshape(Dx * Dx, Dx * Dx)
    return 0.5 * (G_L + G_L.T), 0.5 * (G_R + G_R.T)


def eigh_desc(G: np.ndarray):
    """Eigenpairs of a symmetric matrix, eigenvalues in descending order."""
    lam, V = np.linalg.eigh(G)
    return lam[::-1].copy(), V[:, ::-1].copy()


# --------------------------------------------------------------------------
# a4-a8: one coarse-graining step
# --------------------------------------------------------------------------

@dataclass
class StepInfo:
    direction: str          # 'x' or 'y'
    Dx: int                 # fused-leg bond dimension before the step (in the step's own view)
    Dy: int                 # contracted-leg bond dimension
    Dn: int                 # kept dimension D' = min(Dx^2, D_cut)
    ln_c: float             # ln max|T'| before rescale
    eps_L: float            # discarded weight of the left environment
    eps_R: float            # discarded weight of the right environment
    side: int               # 0 = left, 1 = right, -1 = no truncation (U = I)
    cut_gap: float          # (lam_{D'} - lam_{D'+1}) / lam_1 of the chosen side (inf if no cut)
    trace_G: float          # Tr G_L (= Tr G_R = ||M||_F^2)
    spectrum: np.ndarray = field(repr=False)  # eigenvalues of the chosen env / lam_1, descending


def y_step(T: np.ndarray, D_cut: int):
    """One Y coarse-graining step; returns (T' normalised, c, U, StepInfo)."""
    T = np.asarray(T, dtype=np.float64)
    Dx, Dx2, Dy, Dy2 = T.shape
    if Dx != Dx2 or Dy != Dy2:
        raise ValueError("T must have shape (Dx, Dx, Dy, Dy)")
    n = Dx * Dx
    Dn = min(n, D_cut)

    G_L, G_R = gram_environments(T)
    lam_L, V_L = eigh_desc(G_L)
    lam_R, V_R = eigh_desc(G_R)
    eps_L = float(np.sum(lam_L[Dn:]))
    eps_R = float(np.sum(lam_R[Dn:]))
    if n <= D_cut:
        side = -1
        U = np.eye(n)
        lam = lam_L
    elif eps_L <= eps_R:
        side, U, lam = 0, V_L[:, :Dn], lam_L
    else:
        side, U, lam = 1, V_R[:, :Dn], lam_R
    if Dn < n:
        cut_gap = float((lam[Dn - 1] - lam[Dn]) / lam[0])
    else:
        cut_gap = float("inf")

    Tn = project(T, U)
    c = float(np.max(np.abs(Tn)))
    if not np.isfinite(c) or c <= 0.0:
        raise FloatingPointError("coarse-grained tensor has no finite nonzero max-norm")
    info = StepInfo("y", Dx, Dy, Dn, float(np.log(c)), eps_L, eps_R, side, cut_gap,
                    float(np.trace(G_L)), lam / lam[0])
    return Tn / c, c, U, info


def project(T: np.ndarray, U: np.ndarray) -> np.ndarray:
    """T'[a,b,y,y'] = sum U[(x1 x2),a] T[x1,x1',y,k] T[x2,x2',k,y'] U[(x1'x2'),b].

    Evaluated as three pairwise contractions (U into the lower tensor, the
    upper tensor over (x2,k), then U over (x1',x2')), never forming M.
    """
    Dx = T.shape[0]
    U3 = U.reshape(Dx, Dx, U.shape[1])                         # [x1,x2,a]
    P = np.tensordot(U3, T, axes=([0], [0]))                   # [x2,a,x1',y,k]
    Q = np.tensordot(P, T, axes=([0, 4], [0, 2]))              # [a,x1',y,x2',y']
    del P
    Tn = np.tensordot(Q, U3, axes=([1, 3], [0, 1]))            # [a,y,y',b]
    return np.ascontiguousarray(Tn.transpose(0, 3, 1, 2))      # [a,b,y,y']


def x_step(T: np.ndarray, D_cut: int):
    """One X step: the Y step on the view T[y,y',x,x'], viewed back."""
    Tn, c, U, info = y_step(np.ascontiguousarray(np.transpose(T, (2, 3, 0, 1))), D_cut)
    info.direction = "x"
    return np.ascontiguousarray(np.transpose(Tn, (2, 3, 0, 1))), c, U, info


# --------------------------------------------------------------------------
# a9: whole run and free energy
# --------------------------------------------------------------------------

def periodic_trace(T: np.ndarray) -> float:
    """Tr_x Tr_y T = sum_{x,y} T[x,x,y,y] (both directions periodic)."""
    return float(np.einsum("aabb->", T))


def trace_y(T: np.ndarray):
    """Close the y direction: T_x[x, x', 0, 0] = sum_y T[x, x', y, y].

    Returns (T_x / c, c) with c = max |T_x|.  The y legs become trivial (size 1),
    so every later X step is a plain product of the (Dx x Dx) column matrices
    and Tr T_x^Lx is the periodic network of Lx columns.
    """
    T = np.asarray(T, dtype=np.float64)
    Tx = np.einsum("abyy->ab", T)[:, :, None, None]
    c = float(np.max(np.abs(Tx)))
    if not np.isfinite(c) or c <= 0.0:
        raise FloatingPointError("traced tensor has no finite nonzero max-norm")
    return Tx / c, c


def directions(nsteps: int, first: str = "x"):
    """Alternating step directions starting with ``first``."""
    other = "y" if first == "x" else "x"
    return [first if i % 2 == 0 else other for i in range(nsteps)]


@dataclass
class HotrgRun:
    T: np.ndarray
    n: int = 0
    logsum: float = 0.0
    steps: list = field(default_factory=list)

    @property
    def ln_z_per_site(self) -> float:
        tr = periodic_trace(self.T)
        if not tr > 0.0:
            raise FloatingPointError("periodic trace of the coarse-grained tensor is not positive")
        return self.logsum + np.log(tr) / 2.0 ** self.n

    def free_energy(self, beta: float) -> float:
        """f = -(1/beta) ln Z / N  (J = 1 units)."""
        return -self.ln_z_per_site / beta


def run(T0: np.ndarray, D_cut: int, nsteps: int, first: str = "x", dirs=None) -> HotrgRun:
    """Scale T0 by its max-norm, then apply ``nsteps`` alternating X/Y steps."""
    T0 = np.asarray(T0, dtype=np.float64)
    c0 = float(np.max(np.abs(T0)))
    if not np.isfinite(c0) or c0 <= 0.0:
        raise FloatingPointError("initial tensor has no finite nonzero max-norm")
    st = HotrgRun(T=T0 / c0, n=0, logsum=float(np.log(c0)))
    for d in (dirs if dirs is not None else directions(nsteps, first)):
        step = x_step if d == "x" else y_step
        st.T, c, _, info = step(st.T, D_cut)
        st.n += 1
        st.logsum += np.log(c) / 2.0 ** st.n
        st.steps.append(info)
    return st
