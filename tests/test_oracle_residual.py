"""Pins of the oracle's residual (the relative residual ||b - A x|| / ||b|| by
which Section 6.3 scores every least-squares solve, and the gradient A^T r the
refinement uses) against what mathematics fixes on its own:

* integer problems whose residual is known exactly (b = A x + e with integer
  e, so r = e and ||r||^2, ||b||^2 are exact integers evaluated in Python's
  arbitrary-precision arithmetic): a squared norm, a dropped square root, a
  missing term, a sign slip in r or a constant factor all fail here;
* the special cases x = 0 (r = b, relres = 1) and b = A x (relres = 0);
* agreement with an independent FP64 evaluation (numpy's matrix product and
  norm) on random float64 and float32 problems, for r, g = A^T r and both
  norms;
* the orthogonality of the residual at the least-squares minimiser (LAPACK's
  lstsq): A^T r = 0 up to rounding.
"""
import math

import numpy as np
import pytest

EPS64 = np.finfo(np.float64).eps


def _int_problem(d, n, seed, dtype=np.float64):
    rng = np.random.default_rng(seed)
    A = rng.integers(-50, 51, size=(d, n)).astype(dtype)
    x = rng.integers(-9, 10, size=n).astype(np.float64)
    e = rng.integers(-20, 21, size=d).astype(np.float64)
    Ai = A.astype(np.int64)
    b_int = Ai @ x.astype(np.int64) + e.astype(np.int64)
    return A, x, e.astype(np.int64), b_int


@pytest.mark.parametrize("d,n,dtype", [(1, 1, np.float64), (7, 3, np.float64), (1000, 17, np.float64),
                                       (4099, 8, np.float32)])
def test_residual_exact_on_integer_problem(orc, d, n, dtype):
    A, x, e, b_int = _int_problem(d, n, 10 + d + n, dtype)
    b = b_int.astype(np.float64)
    rr_exact = sum(int(v) * int(v) for v in e)          # ||r||^2, r = e exactly
    bb_exact = sum(int(v) * int(v) for v in b_int)      # ||b||^2
    rn, bn = orc.residual(A, b, x)
    assert rn == math.sqrt(rr_exact)
    assert bn == math.sqrt(bb_exact)
    want = math.sqrt(rr_exact) / math.sqrt(bb_exact)
    assert abs(orc.relres(A, b, x) - want) <= 2 * EPS64 * want
    r, g, rn2, bn2 = orc.residual_and_gradient(A, b, x)
    assert np.array_equal(r, e.astype(np.float64))     # r = b - A x, not A x - b
    g_exact = A.astype(np.int64).T @ e                    # A^T r in integers
    assert np.array_equal(g, g_exact.astype(np.float64))
    assert rn2 == rn and bn2 == bn


def test_residual_special_cases(orc):
    A, x, _, b_int = _int_problem(300, 5, 3)
    b = b_int.astype(np.float64)
    # x = 0: r = b, relres exactly 1
    assert orc.relres(A, b, np.zeros(5)) == 1.0
    # b = A x exactly: zero residual
    b0 = (A.astype(np.int64) @ x.astype(np.int64)).astype(np.float64)
    r, g, rn, _ = orc.residual_and_gradient(A, b0, x)
    assert rn == 0.0 and not r.any() and not g.any()
    # the residual scales with b: relres of (A, 2b, 2x) equals relres of (A, b, x)
    assert orc.relres(A, 2 * b, 2 * x) == orc.relres(A, b, x)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_residual_matches_independent_fp64_evaluation(orc, dtype):
    rng = np.random.default_rng(7)
    d, n = 5000, 24
    A = rng.standard_normal((d, n)).astype(dtype)
    x = rng.standard_normal(n)
    b = rng.standard_normal(d)
    A64 = A.astype(np.float64)            # binary32 -> binary64 is exact
    r_np = b - A64 @ x
    g_np = A64.T @ r_np
    r, g, rn, bn = orc.residual_and_gradient(A, b, x)
    scale = np.abs(b) + np.abs(A64) @ np.abs(x)
    assert np.all(np.abs(r - r_np) <= 2 * (n + 2) * EPS64 * scale)
    gscale = np.abs(A64).T @ scale
    assert np.all(np.abs(g - g_np) <= 4 * (n + d + 2) * EPS64 * gscale)
    assert abs(rn - np.linalg.norm(r_np)) <= 1e-13 * rn
    assert abs(bn - np.linalg.norm(b)) <= 1e-13 * bn
    assert abs(orc.relres(A, b, x) - np.linalg.norm(r_np) / np.linalg.norm(b)) <= 1e-13 * rn / bn


def test_residual_orthogonal_at_minimiser(orc):
    rng = np.random.default_rng(11)
    d, n = 3000, 12
    A = rng.standard_normal((d, n))
    b = rng.standard_normal(d)
    xo = np.linalg.lstsq(A, b, rcond=None)[0]
    r, g, rn, bn = orc.residual_and_gradient(A, b, xo)
    # A^T r vanishes at the minimiser up to rounding of x (kappa(A) ~ 1 here)
    assert np.max(np.abs(g)) <= 1e3 * EPS64 * np.linalg.norm(A) * np.linalg.norm(b)
    # and the minimiser's residual is below any perturbed point's
    for t in (1e-3, 1e-6):
        assert orc.relres(A, b, xo + t * rng.standard_normal(n)) > rn / bn
