"""Pins of the oracle's operator v = A^T (A p) of the preconditioned normal
equations (Section 6.3), independent of its implementation: exact rational
arithmetic on small inputs, and a cancellation that plain FP64 sums lose."""
from fractions import Fraction

import numpy as np
import pytest


def _exact(A32, p):
    """w_i = round(sum_j a_ij p_j) exactly rounded to FP64, then v_j the same
    over i, by Fractions."""
    d, n = A32.shape
    Af = [[Fraction(float(A32[i, j])) for j in range(n)] for i in range(d)]
    pf = [Fraction(float(x)) for x in p]
    w = [float(sum(Af[i][j] * pf[j] for j in range(n))) for i in range(d)]
    wf = [Fraction(x) for x in w]
    return np.array([float(sum(Af[i][j] * wf[i] for i in range(d))) for j in range(n)])


@pytest.mark.parametrize("d,n,seed", [(1, 1, 0), (7, 3, 1), (13, 5, 2), (33, 8, 3)])
def test_normal_apply_equals_exact_rational(orc, d, n, seed):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((d, n)) * np.exp2(rng.integers(-20, 20, (d, n)))).astype(np.float32)
    p = rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))
    v = orc.normal_apply(A, p)
    assert np.array_equal(v, _exact(A, p))


def test_normal_apply_cancellation(orc):
    # w = 2^60 + 1 - 2^60 = 1 exactly, so v = (1, 1, 1); left-to-right FP64
    # sums lose the 1 and give v = 0
    A = np.array([[1.0, 1.0, 1.0]], dtype=np.float32)
    p = np.array([2.0 ** 60, 1.0, -(2.0 ** 60)])
    naive = A.astype(np.float64).T @ (A.astype(np.float64) @ p)
    assert np.array_equal(orc.normal_apply(A, p), np.ones(3))
    assert np.array_equal(_exact(A, p), np.ones(3))
    assert not np.array_equal(naive, np.ones(3))


def test_normal_apply_zero_and_transpose_identity(orc):
    rng = np.random.default_rng(9)
    A = rng.standard_normal((40, 6)).astype(np.float32)
    assert np.array_equal(orc.normal_apply(A, np.zeros(6)), np.zeros(6))
    # p = e_j gives column j of A^T A, which is symmetric
    M = np.stack([orc.normal_apply(A, np.eye(6)[j]) for j in range(6)], axis=1)
    assert np.allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
