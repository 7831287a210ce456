"""Element-by-element evaluation of one coarse-graining step's outputs.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

At bond dimensions where the full oracle takes minutes per step, the GPU's own
input tensor T and isometry U of one step are read back and single elements of
the step's outputs are recomputed here straight from their definitions
(Sec. II.A: the contracted pair M of two tensors, its Gram matrices, and the
projection of its fused legs):

    M[x1,x2,x1',x2',y,y'] = sum_k T[x1,x1',y,k] T[x2,x2',k,y']
    G_L[(x1 x2),(u1 u2)]   = sum M[x1,x2,...] M[u1,u2,...]      (over x1',x2',y,y')
    G_R[(x1'x2'),(u1'u2')] = sum M[...,x1',x2',y,y'] M[...,u1',u2',y,y']
    T'[a,b,y,y']           = sum U[(x1 x2),a] M[x1,x2,x1',x2',y,y'] U[(x1'x2'),b]

Each routine forms only the slice of M that the requested element needs.
"""
from __future__ import annotations

import numpy as np


def m_slice_left(T: np.ndarray, x1: int, x2: int) -> np.ndarray:
    """M[x1,x2,:,:,:,:] as an array [x1',x2',y,y']."""
    return np.einsum("pyk,qkz->pqyz", T[x1], T[x2])


def m_slice_right(T: np.ndarray, x1p: int, x2p: int) -> np.ndarray:
    """M[:,:,x1',x2',:,:] as an array [x1,x2,y,y']."""
    return np.einsum("ayk,bkz->abyz", T[:, x1p], T[:, x2p])


def m_slice_yy(T: np.ndarray, y: int, yp: int) -> np.ndarray:
    """M[:,:,:,:,y,y'] as an array [x1,x2,x1',x2']."""
    return np.einsum("apk,bqk->abpq", T[:, :, y, :], T[:, :, :, yp])


def gram_element(T: np.ndarray, side: int, i: int, j: int) -> float:
    """G_L[i,j] (side 0) or G_R[i,j] (side 1) of a Y step on T."""
    Dx = T.shape[0]
    a1, a2 = divmod(i, Dx)
    b1, b2 = divmod(j, Dx)
    f = m_slice_left if side == 0 else m_slice_right
    return float(np.vdot(f(T, a1, a2), f(T, b1, b2)))


def projected_elements(T: np.ndarray, U: np.ndarray, samples):
    """T'[a,b,y,y'] (before rescale) for each (a, b, y, y') in ``samples``."""
    Dx = T.shape[0]
    out = []
    cache = {}
    for (a, b, y, yp) in samples:
        key = (y, yp)
        if key not in cache:
            cache[key] = m_slice_yy(T, y, yp)
        Mq = cache[key]
        ua = U[:, a].reshape(Dx, Dx)
        ub = U[:, b].reshape(Dx, Dx)
        out.append(float(np.einsum("ab,abpq,pq->", ua, Mq, ub)))
    return np.array(out)
