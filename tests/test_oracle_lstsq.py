"""Pins of the oracle's least-squares solvers against what the paper fixes:
exact recovery for b = A x, the sketch-and-solve distortion bound of Section 2,
agreement with the normal equations when well conditioned and their breakdown
for kappa > 1e8 (Section 6.3), and convergence of the refinement to the exact
least-squares minimiser."""
import math

import numpy as np
import pytest
import torch

import inputs


def test_sns_exact_recovery(orc):
    d, n = 1 << 13, 8
    A, _, _ = inputs.ls_problem(d, n, -2, seed=21)
    A = A.numpy()
    x_true = np.arange(1, n + 1, dtype=np.float64)
    b = A @ x_true
    x, rel, _ = orc.sns_lstsq(A, b, 2 * n * n, 4 * n, seed=5)
    # kappa(A) = 100: forward error O(kappa u)
    assert np.max(np.abs(x - x_true)) < 1e-11 * np.max(np.abs(x_true))
    assert rel < 1e-13


@pytest.mark.parametrize("mu,var", [(0.0, 0.01), (3.0, 2.0)])
def test_sns_distortion_bound(orc, mu, var):
    # Section 2: relres(x_sns)/relres(x_opt) in [1, sqrt((1+eps)/(1-eps))];
    # with k = 2n^2 and p = 4n the embedding is a modest-eps one: the ratio must
    # be >= 1 and O(1) (here below 2, i.e. eps < 0.6), over several seeds.
    d, n = 1 << 13, 8
    A, _, _ = inputs.ls_problem(d, n, -2, seed=22)
    b = inputs.noisy_rhs(A, mu, var, seed=23).numpy()
    A = A.numpy()
    xo = orc.lstsq_exact(A, b)
    ro = orc.relres(A, b, xo)
    for sd in range(5):
        _, rs, _ = orc.sns_lstsq(A, b, 2 * n * n, 4 * n, seed=sd)
        assert ro * (1 - 1e-12) <= rs < 2.0 * ro


def test_ne_agrees_when_well_conditioned(orc):
    d, n = 1 << 12, 10
    A, b, _ = inputs.ls_problem(d, n, -4, seed=24)
    A, b = A.numpy(), b.numpy()
    xn, info = orc.ne_lstsq(A, b)
    xq = orc.lstsq_exact(A, b)
    assert info == 0
    # kappa^2 u ~ 1e-8 relative
    assert np.max(np.abs(xn - xq)) < 1e-6 * np.max(np.abs(xq))


def test_ne_breaks_down_beyond_1e8_while_sns_does_not(orc):
    # Section 6.3, sensitivity experiment: d = 2^17, n = 16, b = A e.
    d, n = 1 << 17, 16
    e = np.ones(n)
    A, _, _ = inputs.ls_problem(d, n, -10, seed=25)
    A = A.numpy()
    b = A @ e
    xq = orc.lstsq_exact(A, b)
    rq = orc.relres(A, b, xq)
    xs, rs, _ = orc.sns_lstsq(A, b, 2 * n * n, 4 * n, seed=3)
    xn, info = orc.ne_lstsq(A, b)
    rn = orc.relres(A, b, xn) if info == 0 else math.inf
    assert rq < 1e-13 and rs < 1e-12   # QR and sketch-and-solve stay stable
    assert info > 0 or rn > 1e3 * max(rs, rq)   # the normal equations do not


def test_refinement_reaches_exact_minimiser(orc):
    d, n = 1 << 13, 12
    A, b, _ = inputs.ls_problem(d, n, -6, seed=26, dtype=torch.float32)
    A, b = A.numpy(), b.numpy()
    xo = orc.lstsq_exact(A, b)
    ro = orc.relres(A, b, xo)
    x0, rs, Rf = orc.sns_lstsq(A, b, 2 * n * n, 4 * n, seed=4)
    x, hist = orc.refine(A, b, Rf[:n, :n], x0, max_iter=100, tol=1e-13)
    assert abs(hist[-1] - ro) <= 1e-10 * ro
    assert np.allclose(x, xo, rtol=1e-6, atol=1e-6 * np.max(np.abs(xo)))
    # CG on the normal equations decreases ||r|| monotonically
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))
