"""Pins of the FP64 oracle against things other than itself (CPU only).

Every check here uses a route independent of the function under test:
closed forms (Onsager, Catalan's constant), exact enumeration / transfer
matrices, the SVD of an explicitly formed unfolding, invariances that hold
exactly in the mathematics, and element-by-element definitions.
"""
import math

import numpy as np
import pytest

from oracle import brute, exact, hotrg, onsager, sampled
from workloads import BETA_C_ISING, BETA_C_POTTS3, random_orthogonal, random_tensor

BIG = 10 ** 9  # D_cut that disables truncation


def ising_Bw(beta, h=0.0):
    s = np.array([1.0, -1.0])
    return np.exp(beta * np.outer(s, s)), np.exp(beta * h * s)


def potts_Bw(q, beta):
    return np.exp(beta * np.eye(q)), np.ones(q)


# ---------------------------------------------------------------- Onsager

CATALAN = 0.915965594177219015054603514932384110774  # Catalan's constant G


def test_catalan_constant_literal():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    assert abs(float(mpmath.catalan) - CATALAN) < 1e-16


def test_onsager_critical_point_closed_form():
    # at beta_c the integral evaluates to 2G/pi + ln(2)/2
    assert abs(onsager.ising_ln_z_per_site(BETA_C_ISING) - (2 * CATALAN / math.pi + 0.5 * math.log(2))) < 1e-14


@pytest.mark.parametrize("beta", [0.3, 0.44, 0.6])
def test_onsager_single_vs_double_integral(beta):
    assert abs(onsager.ising_ln_z_per_site(beta) - onsager.ising_ln_z_per_site_double(beta)) < 1e-10


def test_onsager_high_temperature_limit():
    assert abs(onsager.ising_ln_z_per_site(1e-8) - math.log(2)) < 1e-12


# ---------------------------------------------------------------- initial tensor

@pytest.mark.parametrize("beta,h", [(BETA_C_ISING, 0.0), (0.44, 0.01), (0.3, -0.2)])
def test_ising_initial_tensor_structure(beta, h):
    B, w = ising_Bw(beta, h)
    W = hotrg.sqrtm_psd(B)
    assert np.allclose(W @ W, B, rtol=0, atol=1e-14)
    T0 = hotrg.ising_initial_tensor(beta, h)
    # 1x1 torus: the site meets itself through both bonds
    assert abs(hotrg.periodic_trace(T0) - float(np.sum(w * np.diag(B) ** 2))) < 1e-13
    # leg symmetries
    assert np.allclose(T0, T0.transpose(1, 0, 2, 3), atol=1e-15)
    assert np.allclose(T0, T0.transpose(0, 1, 3, 2), atol=1e-15)
    assert np.allclose(T0, T0.transpose(2, 3, 0, 1), atol=1e-15)


def test_ising_trace_at_beta_c_is_two_plus_two_sqrt2():
    assert abs(hotrg.periodic_trace(hotrg.ising_initial_tensor(BETA_C_ISING)) - (2 + 2 * math.sqrt(2))) < 1e-14


def test_ising_W_at_beta_c_closed_form():
    # eigen-decomposition of B in closed form: eigenvalues 2cosh(beta), 2sinh(beta)
    b = BETA_C_ISING
    lp, lm = math.sqrt(2 * math.cosh(b)), math.sqrt(2 * math.sinh(b))
    W = hotrg.sqrtm_psd(ising_Bw(b)[0])
    assert np.allclose(W, 0.5 * np.array([[lp + lm, lp - lm], [lp - lm, lp + lm]]), atol=1e-15)


# ---------------------------------------------------------------- exact small tori

@pytest.mark.parametrize("Lx,Ly", [(1, 1), (2, 1), (2, 2), (3, 2), (3, 3)])
def test_transfer_matrix_vs_brute_force_random_weights(Lx, Ly):
    rng = np.random.default_rng(7 + Lx * 10 + Ly)
    B = rng.uniform(0.2, 2.0, size=(3, 3))
    w = rng.uniform(0.5, 1.5, size=3)
    assert abs(exact.transfer_matrix_ln_z(B, w, Lx, Ly) - brute.brute_ln_z(B, w, Lx, Ly)) < 1e-12


def test_ising_4x4_at_beta_c_integer_partition_function():
    # at beta_c, e^{2 beta} = 1 + sqrt 2 and every energy is a multiple of 4, so Z is an integer
    B, w = ising_Bw(BETA_C_ISING)
    lnz = brute.brute_ln_z(B, w, 4, 4)
    assert abs(math.exp(lnz) - 5509120.0) < 1e-6


@pytest.mark.parametrize("model", ["ising_bc", "ising_044h", "potts3", "ising_random_field"])
def test_hotrg_no_truncation_equals_exact_4x4(model):
    if model == "ising_bc":
        B, w = ising_Bw(BETA_C_ISING)
    elif model == "ising_044h":
        B, w = ising_Bw(0.44, 0.01)
    elif model == "ising_random_field":
        B, w = ising_Bw(0.37, -0.3)
    else:
        B, w = potts_Bw(3, BETA_C_POTTS3)
    T0 = hotrg.initial_tensor(B, w)
    r = hotrg.run(T0, BIG, 4)
    lnz_tm = exact.transfer_matrix_ln_z(B, w, 4, 4)
    lnz_bf = brute.brute_ln_z(B, w, 4, 4)
    assert abs(lnz_tm - lnz_bf) < 1e-11
    assert abs(r.ln_z_per_site * 16 - lnz_bf) < 1e-11


def test_survey_anchor_values_4x4():
    # ln Z / 16 of the 4x4 torus, recomputed by enumeration
    cases = [(ising_Bw(BETA_C_ISING), 0.9701197161722049),
             (ising_Bw(0.44), 0.969045408669885),
             (ising_Bw(0.44, 0.01), 0.9691630142785459),
             (potts_Bw(3, BETA_C_POTTS3), 2.135788008614013)]
    for (B, w), ref in cases:
        assert abs(brute.brute_ln_z(B, w, 4, 4) / 16 - ref) < 1e-14


@pytest.mark.parametrize("dirs,Lx,Ly", [("x", 2, 1), ("y", 1, 2), ("xy", 2, 2), ("yx", 2, 2),
                                        ("xyx", 4, 2), ("yxy", 2, 4), ("xyxy", 4, 4)])
def test_hotrg_no_truncation_random_tensor_vs_network(dirs, Lx, Ly):
    T = random_tensor(3, seed=11, Dy=2)
    r = hotrg.run(T, BIG, len(dirs), dirs=list(dirs))
    lnz, sign = exact.network_ln_abs_z(T, Lx, Ly)
    assert sign > 0
    assert abs(r.ln_z_per_site * Lx * Ly - lnz) < 1e-11


@pytest.mark.parametrize("Lx,Ly", [(1, 1), (2, 2), (4, 2), (4, 4)])
def test_network_vs_transfer_matrix(Lx, Ly):
    B, w = potts_Bw(3, 0.7)
    T0 = hotrg.initial_tensor(B, w)
    assert abs(exact.network_ln_abs_z(T0, Lx, Ly)[0] - exact.transfer_matrix_ln_z(B, w, Lx, Ly)) < 1e-11


def test_invertible_gauge_leaves_exact_z_unchanged():
    # T -> T x_left G x_right G^{-T}: every contracted bond sees G^{-1} G = 1
    T = random_tensor(2, seed=3)
    rng = np.random.default_rng(5)
    Gx = np.eye(2) + 0.3 * rng.standard_normal((2, 2))
    Gy = np.eye(2) + 0.3 * rng.standard_normal((2, 2))
    Tg = np.einsum("abcd,ax,by,cz,dw->xyzw", T, Gx, np.linalg.inv(Gx).T, Gy, np.linalg.inv(Gy).T)
    r1 = hotrg.run(T, BIG, 4)
    r2 = hotrg.run(Tg, BIG, 4)
    assert abs(r1.ln_z_per_site - r2.ln_z_per_site) < 1e-12
    # the swapped gauge (G on the right leg) is not an invariance: it must change Z
    Tb = np.einsum("abcd,ax,by,cz,dw->xyzw", T, np.linalg.inv(Gx).T, np.linalg.inv(Gx).T, Gy, np.linalg.inv(Gy).T)
    assert abs(hotrg.run(Tb, BIG, 4).ln_z_per_site - r1.ln_z_per_site) > 1e-6


# ---------------------------------------------------------------- truncation vs definition

def definition_y_step(T, D_cut):
    """Y step by its definition: M formed explicitly, truncation from the SVDs of
    its two unfoldings (singular values squared are the Gram eigenvalues)."""
    Dx, _, Dy, _ = T.shape
    M = np.einsum("acyk,bdkz->abcdyz", T, T)       # [x1,x2,x1',x2',y,y']
    n = Dx * Dx
    Dn = min(n, D_cut)
    ML = M.reshape(n, -1)
    MR = M.transpose(2, 3, 0, 1, 4, 5).reshape(n, -1)
    UL, sL, _ = np.linalg.svd(ML, full_matrices=False)
    UR, sR, _ = np.linalg.svd(MR, full_matrices=False)
    lamL = np.concatenate([sL ** 2, np.zeros(n - sL.size)])
    lamR = np.concatenate([sR ** 2, np.zeros(n - sR.size)])
    epsL, epsR = lamL[Dn:].sum(), lamR[Dn:].sum()
    if epsL <= epsR:
        U, lam, side = UL[:, :Dn], lamL, 0
    else:
        U, lam, side = UR[:, :Dn], lamR, 1
    Tn = np.einsum("ia,ijyz,jb->abyz", U, M.reshape(n, n, Dy, Dy), U)
    return Tn, U, lam, epsL, epsR, side


def sign_fix(U):
    idx = np.argmax(np.abs(U), axis=0)
    return U * np.sign(U[idx, np.arange(U.shape[1])])


@pytest.mark.parametrize("shape,D_cut,seed", [((3, 3, 2, 2), 4, 1), ((3, 3, 3, 3), 5, 2),
                                              ((2, 2, 4, 4), 3, 3), ((4, 4, 2, 2), 7, 4)])
def test_truncated_y_step_matches_definition(shape, D_cut, seed):
    rng = np.random.default_rng(seed)
    T = rng.standard_normal(shape)
    Tn, c, U, info = hotrg.y_step(T, D_cut)
    Td, Ud, lam, epsL, epsR, side = definition_y_step(T, D_cut)
    assert info.side == side
    assert abs(info.eps_L - epsL) < 1e-12 * lam[0]
    assert abs(info.eps_R - epsR) < 1e-12 * lam[0]
    assert np.allclose(info.spectrum, lam / lam[0], rtol=0, atol=1e-12)
    # elementwise after fixing the eigenvector signs (non-degenerate random spectra)
    S1 = np.sign(U[np.argmax(np.abs(U), axis=0), np.arange(U.shape[1])])
    S2 = np.sign(Ud[np.argmax(np.abs(Ud), axis=0), np.arange(Ud.shape[1])])
    A = np.einsum("abyz,a,b->abyz", Tn * c, S1, S1)
    B = np.einsum("abyz,a,b->abyz", Td, S2, S2)
    assert np.allclose(A, B, rtol=0, atol=1e-12 * np.max(np.abs(B)))
    assert abs(c - np.max(np.abs(Td))) < 1e-12 * c


def test_x_step_is_y_step_on_transposed_view():
    T = random_tensor(3, seed=9, Dy=2)
    Tx, cx, _, ix = hotrg.x_step(T, 3)
    Td, _, lam, _, _, _ = definition_y_step(T.transpose(2, 3, 0, 1), 3)
    assert ix.direction == "x"
    assert np.allclose(ix.spectrum, lam / lam[0], atol=1e-12)
    assert Tx.shape == (3, 3, 3, 3)   # (Dx, Dx, Dy', Dy') with Dy' = min(2*2, 3)
    assert abs(cx - np.max(np.abs(Td))) < 1e-12 * cx


def test_gram_environments_vs_unfolding():
    T = np.random.default_rng(12).standard_normal((3, 3, 2, 2))
    G_L, G_R = hotrg.gram_environments(T)
    M = np.einsum("acyk,bdkz->abcdyz", T, T)
    ML = M.reshape(9, -1)
    MR = M.transpose(2, 3, 0, 1, 4, 5).reshape(9, -1)
    assert np.allclose(G_L, ML @ ML.T, atol=1e-12)
    assert np.allclose(G_R, MR @ MR.T, atol=1e-12)
    assert abs(np.trace(G_L) - np.trace(G_R)) < 1e-12


def test_sampled_elements_vs_full_step():
    T = np.random.default_rng(13).standard_normal((4, 4, 3, 3))
    G_L, G_R = hotrg.gram_environments(T)
    rng = np.random.default_rng(0)
    for _ in range(10):
        i, j = rng.integers(0, 16, size=2)
        assert abs(sampled.gram_element(T, 0, i, j) - G_L[i, j]) < 1e-12 * np.abs(G_L).max()
        assert abs(sampled.gram_element(T, 1, i, j) - G_R[i, j]) < 1e-12 * np.abs(G_R).max()
    Tn, c, U, _ = hotrg.y_step(T, 6)
    samples = [tuple(int(v) for v in rng.integers(0, [6, 6, 3, 3])) for _ in range(12)]
    vals = sampled.projected_elements(T, U, samples)
    ref = np.array([Tn[s] * c for s in samples])
    assert np.allclose(vals, ref, atol=1e-12 * c)


# ---------------------------------------------------------------- truncated runs vs closed forms

@pytest.mark.parametrize("D_cut,tol", [(8, 2e-5), (12, 2e-6), (16, 2e-7)])
def test_truncated_hotrg_vs_onsager_at_beta_c(D_cut, tol):
    r = hotrg.run(hotrg.ising_initial_tensor(BETA_C_ISING), D_cut, 20)
    exact_v = onsager.ising_ln_z_per_site(BETA_C_ISING)
    assert abs(r.ln_z_per_site / exact_v - 1) < tol


def test_truncated_hotrg_vs_onsager_off_critical():
    r = hotrg.run(hotrg.ising_initial_tensor(0.44), 12, 24)
    assert abs(r.ln_z_per_site / onsager.ising_ln_z_per_site(0.44) - 1) < 5e-6


def test_potts_q2_is_ising_at_half_coupling():
    bp = 0.9
    Tp = hotrg.potts_initial_tensor(2, bp)
    Ti = hotrg.ising_initial_tensor(bp / 2)
    assert np.allclose(Tp, math.exp(bp) * Ti, rtol=1e-14, atol=0)
    rp = hotrg.run(Tp, 10, 20)
    ri = hotrg.run(Ti, 10, 20)
    assert abs(rp.ln_z_per_site - (ri.ln_z_per_site + bp)) < 1e-12
    assert abs(rp.ln_z_per_site - bp - onsager.ising_ln_z_per_site(bp / 2)) < 1e-5


def test_field_reversal_symmetry():
    r1 = hotrg.run(hotrg.ising_initial_tensor(0.44, 0.05), 10, 16)
    r2 = hotrg.run(hotrg.ising_initial_tensor(0.44, -0.05), 10, 16)
    assert abs(r1.ln_z_per_site - r2.ln_z_per_site) < 1e-12


@pytest.mark.parametrize("q", [2, 3])
def test_infinite_temperature_limit(q):
    T0 = hotrg.potts_initial_tensor(q, 1e-10) if q == 3 else hotrg.ising_initial_tensor(1e-10)
    r = hotrg.run(T0, 8, 12)
    assert abs(r.ln_z_per_site - math.log(q)) < 1e-8


def test_orthogonal_gauge_invariance_with_truncation():
    T0 = hotrg.ising_initial_tensor(0.44, 0.01)
    # gauge the D0 = 2 legs with random orthogonal matrices (same O on both legs of a direction)
    Ox, Oy = random_orthogonal(2, seed=21), random_orthogonal(2, seed=22)
    Tg = np.einsum("abcd,ax,by,cz,dw->xyzw", T0, Ox, Ox, Oy, Oy)
    r1 = hotrg.run(T0, 8, 14)
    r2 = hotrg.run(Tg, 8, 14)
    assert abs(r1.ln_z_per_site - r2.ln_z_per_site) < 1e-12
    for a, b in zip(r1.steps, r2.steps):
        n = min(a.Dn + 1, a.spectrum.size)
        assert np.allclose(a.spectrum[:n], b.spectrum[:n], atol=1e-11)


def test_step_bookkeeping():
    r = hotrg.run(hotrg.ising_initial_tensor(BETA_C_ISING), 8, 6)
    dims = [(s.direction, s.Dx, s.Dy, s.Dn) for s in r.steps]
    # X: fuses y legs (2->4); Y: fuses x legs (2->4); X: 4->16 cut to 8; Y: 4->8; X: 8->8; Y: 8->8
    assert dims == [("x", 2, 2, 4), ("y", 2, 4, 4), ("x", 4, 4, 8), ("y", 4, 8, 8),
                    ("x", 8, 8, 8), ("y", 8, 8, 8)]
    assert r.T.shape == (8, 8, 8, 8)
    assert [s.side for s in r.steps[:2]] == [-1, -1]
