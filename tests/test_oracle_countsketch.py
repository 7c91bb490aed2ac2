"""Pins of the oracle's CountSketch (Definition 3 and its row form, Section 4):
brute force against the explicitly formed dense S, exact integer sums, the
sum and column-sum invariants, and the embedding property of Section 1."""
import math

import numpy as np
import pytest
import torch

import inputs


def dense_S(orc, seed, d, k):
    h, s = orc.hash_rows(seed, 0, d, k)
    S = np.zeros((k, d))
    S[h.astype(np.int64), np.arange(d)] = s
    return S


@pytest.mark.parametrize("d,n,k", [(1000, 5, 37), (64, 1, 7), (3, 4, 5), (517, 3, 1)])
def test_bruteforce_dense_S(orc, d, n, k):
    A = inputs.normal_matrix(d, n, 3, torch.float64).numpy()
    Y = orc.countsketch(A, k, 99)
    S = dense_S(orc, 99, d, k)
    Ybf = S @ A
    tol = 64 * np.finfo(np.float64).eps * (np.abs(S) @ np.abs(A))
    assert Y.shape == (k, n)
    assert np.all(np.abs(Y - Ybf) <= tol + 1e-300)


def test_integer_sums_exact(orc):
    d, n, k = 5000, 6, 50
    A = inputs.integer_matrix(d, n, 5).numpy()
    S = dense_S(orc, 1234, d, k)
    assert np.array_equal(orc.countsketch(A, k, 1234), S @ A)


def test_extra_column_b(orc):
    d, n, k = 800, 4, 21
    A = inputs.normal_matrix(d, n, 8).numpy()
    b = inputs.normal_matrix(d, 1, 9).numpy()[:, 0]
    Y = orc.countsketch(A, k, 5, b=b)
    assert Y.shape == (k, n + 1)
    S = dense_S(orc, 5, d, k)
    assert np.allclose(Y[:, :n], orc.countsketch(A, k, 5), rtol=0, atol=0)
    assert np.allclose(Y[:, n], S @ b, rtol=1e-14, atol=1e-14)


def test_sum_and_column_sum_invariants(orc):
    d, n, k = 20000, 7, 512
    A = inputs.normal_matrix(d, n, 10).numpy()
    Y = orc.countsketch(A, k, 77)
    _, s = orc.hash_rows(77, 0, d, k)
    # sum of all entries of SA = sum_i s(i) rowsum(A_i)
    want = math.fsum((s.astype(np.float64)[:, None] * A).ravel())
    assert abs(math.fsum(Y.ravel()) - want) <= 1e-12 * np.abs(A).sum()
    # 1^T (S A) = s^T A, column by column
    for j in range(n):
        wj = math.fsum(s.astype(np.float64) * A[:, j])
        assert abs(math.fsum(Y[:, j]) - wj) <= 1e-13 * np.abs(A[:, j]).sum()


def test_float32_input_is_upcast_exactly(orc):
    d, n, k = 3000, 3, 97
    A32 = inputs.normal_matrix(d, n, 12, torch.float32).numpy()
    assert np.array_equal(orc.countsketch(A32, k, 4), orc.countsketch(A32.astype(np.float64), k, 4))


def test_bucket_subset_matches_full(orc):
    d, n, k = 4000, 5, 64
    A = inputs.normal_matrix(d, n, 13).numpy()
    b = inputs.normal_matrix(d, 1, 14).numpy()[:, 0]
    Y = orc.countsketch(A, k, 21, b=b)
    lst = np.array([0, 5, 63, 17])
    Yb, ab, cnt = orc.countsketch_buckets(A, k, 21, lst, b=b)
    assert np.array_equal(Yb, Y[lst])
    h, _ = orc.hash_rows(21, 0, d, k)
    assert np.array_equal(cnt, np.bincount(h, minlength=k)[lst])
    absum = orc.bucket_abs_sums(A, k, 21, b=b)
    assert np.allclose(ab, absum[lst], rtol=1e-14)


def test_empty_and_degenerate(orc):
    A = np.zeros((0, 3))
    assert np.array_equal(orc.countsketch(A, 5, 1), np.zeros((5, 3)))
    A1 = np.ones((10, 1))
    Y = orc.countsketch(A1, 1, 2)  # k = 1: every row in bucket 0
    _, s = orc.hash_rows(2, 0, 10, 1)
    assert Y[0, 0] == float(s.sum())


def test_norm_preservation_statistical(orc):
    # E ||S A x||^2 = ||A x||^2 for a CountSketch (the inner-product embedding
    # of Definition 1 in expectation); average over 200 seeds.
    d, n, k = 2000, 3, 64
    A = inputs.normal_matrix(d, n, 15).numpy()
    x = np.array([1.0, -2.0, 0.5])
    ax2 = float(np.dot(A @ x, A @ x))
    ratios = [float(np.sum((orc.countsketch(A, k, sd) @ x) ** 2)) / ax2 for sd in range(200)]
    # variance of the ratio is about 2/k per seed
    assert abs(np.mean(ratios) - 1.0) < 5 * math.sqrt(2.0 / k / 200)
