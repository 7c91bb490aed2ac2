"""Pins of the oracle's SRHT (Section 5) against what the definition and the
mathematics fix: the fast transform equals the Hadamard matrix of the
recursive definition (scipy.linalg.hadamard); the sketch equals the explicit
dense S = (1/sqrt(k)) P H D; E||S x||^2 = ||x||^2; the sampled rows are
uniform and the signs balanced; sketch-and-solve with it recovers b = A x and
keeps an O(1) distortion."""
import numpy as np
import pytest
import scipy.linalg

import inputs


@pytest.mark.parametrize("d", [1, 2, 4, 64, 1024])
def test_fwht_is_the_recursive_hadamard_matrix(orc, d):
    X = np.random.default_rng(d).integers(-9, 10, size=(d, 3)).astype(np.float64)
    assert np.array_equal(orc.fwht(X), scipy.linalg.hadamard(d).astype(np.float64) @ X)


def test_srht_is_the_explicit_dense_sketch(orc):
    d, n, k, seed = 256, 5, 40, 11
    A = np.random.default_rng(1).integers(-5, 6, size=(d, n)).astype(np.float64)
    b = np.random.default_rng(2).integers(-5, 6, size=d).astype(np.float64)
    D = np.diag(orc.srht_signs(seed, d).astype(np.float64))
    P = np.zeros((k, d))
    P[np.arange(k), orc.srht_rows(seed, k, d).astype(np.int64)] = 1.0
    H = scipy.linalg.hadamard(d).astype(np.float64)
    X = np.hstack([A, b[:, None]])
    # integer entries: every sum is exact, so both sides divide the same
    # integers by sqrt(k) once
    assert np.array_equal(orc.srht(A, k, seed, b=b), (P @ H @ D @ X) / np.sqrt(np.float64(k)))


def test_srht_preserves_norms_in_expectation(orc):
    # E ||S x||^2 = ||x||^2: H D x has squared norm d ||x||^2 spread evenly in
    # expectation over d rows; k rows sampled uniformly, divided by k
    d, k = 4096, 512
    X = np.random.default_rng(3).standard_normal((d, 4))
    r = [np.linalg.norm(orc.srht(X, k, sd)) ** 2 / np.linalg.norm(X) ** 2 for sd in range(8)]
    assert abs(np.mean(r) - 1.0) < 0.05


def test_srht_rows_uniform_and_signs_balanced(orc):
    d, k = 64, 64000
    j = orc.srht_rows(5, k, d)
    assert j.max() < d
    cnt = np.bincount(j, minlength=d)
    chi2 = ((cnt - k / d) ** 2 / (k / d)).sum()
    assert chi2 < 120  # 63 degrees of freedom: P(chi2 > 120) < 1e-5
    s = orc.srht_signs(6, 1 << 16)
    assert abs(int(s.astype(np.int64).sum())) < 5 * 256  # 5 sigma of 2^16 fair signs


def test_srht_sns_recovers_and_embeds(orc):
    d, n = 1 << 13, 8
    A, _, _ = inputs.ls_problem(d, n, -2, seed=51)
    A = A.numpy()
    x_true = np.arange(1, n + 1, dtype=np.float64)
    x, rel, _ = orc.sns_lstsq_srht(A, A @ x_true, 4 * n * n, 3)
    assert np.max(np.abs(x - x_true)) < 1e-11 * np.max(np.abs(x_true)) and rel < 1e-13
    A2, _, _ = inputs.ls_problem(d, n, -2, seed=52)
    b2 = inputs.noisy_rhs(A2, 0.0, 0.01, seed=53).numpy()
    A2 = A2.numpy()
    ro = orc.relres(A2, b2, orc.lstsq_exact(A2, b2))
    for sd in range(3):
        _, rs, _ = orc.sns_lstsq_srht(A2, b2, 4 * n * n, sd)
        assert ro * (1 - 1e-12) <= rs < 2.0 * ro
