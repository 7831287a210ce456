"""GPU checks of hotrg_dgemm_emu, the exact-slice FP64-grade GEMM on the BF16
tensor cores, against FP64 / extended-precision products on the host.

Error model (stated in include/hotrg.h): per term about 2^-(6 S) relative to
the row maxima, so |C - AB^T|_ij <= c K max|A_i.| max|B_j.| 2^-(6S - 2).  The
digit sums are exact only if the tensor cores accumulate integer-valued FP32
sums below 2^24 without loss; the saturation cases drive those sums to their
bound at the largest K of one part (2336) and would show errors near 2^-24 if
they were not exact.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_05900_gb300 as p
    p.load()
    return torch, p


def ref_product(A, B):
    """A @ B.T with a long-double accumulation (at least 64-bit significand)."""
    return (A.astype(np.longdouble) @ B.T.astype(np.longdouble))


def run(env, A, B, slices):
    torch, p = env
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.zeros(A.shape[0], B.shape[0], dtype=torch.float64, device="cuda")
    p.dgemm_emu(dA, dB, dC, slices)
    return dC.cpu().numpy()


def scaled_error(C, A, B):
    ref = ref_product(A, B)
    bound = (np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :] * A.shape[1])
    return float(np.max(np.abs(C.astype(np.longdouble) - ref) / np.maximum(bound, 1e-300)))


@pytest.mark.parametrize("M,N,K", [(300, 77, 1000), (129, 96, 33), (1024, 72, 1024), (64, 200, 2304),
                                   (50, 40, 3000), (130, 33, 5000)])
def test_fp64_grade_random(env, M, N, K):
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-20, 20, size=(M, 1)))
    B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-20, 20, size=(N, 1)))
    for s, bound in ((7, 2.0 ** -41), (8, 2.0 ** -47)):
        err = scaled_error(run(env, A, B, s), A, B)
        print(f"M={M} N={N} K={K} slices={s}: max scaled error {err:.3e} (2^{np.log2(max(err, 1e-300)):.1f})")
        assert err < bound


@pytest.mark.parametrize("K", [2336, 2304, 4096])
def test_exact_digit_sums_at_saturation(env, K):
    # leading digit 63 (odd) in every entry and random lower digits, all of one
    # sign per row: the leading accumulator sums K * 63^2 ~ 2^23 with its low
    # bits set, the next ones their own largest sums; a lossy accumulation
    # would show errors near 2^-24 of the result
    M, N = 128, 96
    rng = np.random.default_rng(K)
    A = (63.0 + rng.uniform(-0.5, 0.5, size=(M, K))) / 64.0
    B = (63.0 + rng.uniform(-0.5, 0.5, size=(N, K))) / 64.0
    for s, bound in ((7, 2.0 ** -41), (8, 2.0 ** -47)):
        assert scaled_error(run(env, A, B, s), A, B) < bound
    A[1::2] *= -1.0
    for s, bound in ((7, 2.0 ** -41), (8, 2.0 ** -47)):
        assert scaled_error(run(env, A, B, s), A, B) < bound


def test_fewer_slices_follow_the_error_model(env):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((256, 512))
    B = rng.standard_normal((64, 512))
    errs = {s: scaled_error(run(env, A, B, s), A, B) for s in (4, 5, 6, 7, 8)}
    print(errs)
    for s, e in errs.items():
        assert e < 2.0 ** -(6 * s - 2), (s, e)
    assert errs[4] > errs[5] > errs[6] > errs[7]


def test_zero_and_nonfinite_rows(env):
    rng = np.random.default_rng(9)
    A = rng.standard_normal((40, 100))
    B = rng.standard_normal((30, 100))
    A[3] = 0.0
    A[7, 11] = np.nan
    C = run(env, A, B, 7)
    assert np.all(C[3] == 0.0)
    assert np.all(np.isnan(C[7]))
    ok = np.ones(40, bool)
    ok[7] = False
    assert scaled_error(C[ok], A[ok], B) < 2.0 ** -40


def test_argument_validation(env):
    torch, p = env
    from paper_2602_05900_gb300.capi import HOTRG_EINVAL
    A = torch.zeros(4, 8, dtype=torch.float64, device="cuda")
    C = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    for slices in (3, 9):
        with pytest.raises(p.HotrgError) as e:
            p.dgemm_emu(A, A, C, slices)
        assert e.value.status == HOTRG_EINVAL
