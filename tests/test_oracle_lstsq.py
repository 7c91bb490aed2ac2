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


@pytest.mark.parametrize("lsig", [-2, -6])
def test_rand_cholqr_is_the_qr_of_A(orc, lsig):
    # Algorithm 4 returns a QR factorisation of A itself: Q^T Q = I, Q R = A,
    # R upper triangular; the QR of a full-rank A is unique up to the signs of
    # R's rows, so |R| and |Q| match LAPACK's (numpy.linalg.qr) to ~kappa u.
    d, n = 3000, 20
    A, _, _ = inputs.ls_problem(d, n, lsig, seed=31)
    A = A.numpy()
    Q, R, info = orc.rand_cholqr(A, 2 * n * n, 4 * n, seed=7)
    assert info == 0
    eps = np.finfo(np.float64).eps
    nA = np.linalg.norm(A, 2)
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 100 * n * eps
    assert np.abs(Q @ R - A).max() < 100 * n * eps * nA
    assert np.all(np.tril(R, -1) == 0.0)
    Ql, Rl = np.linalg.qr(A)
    kappa = 10.0 ** (-lsig)
    assert np.allclose(np.abs(R), np.abs(Rl), rtol=0, atol=100 * n * kappa * eps * nA)
    assert np.allclose(np.abs(Q), np.abs(Ql), rtol=0, atol=100 * n * kappa * eps)
    # R's diagonal carries the signs of the Householder R0 of the sketch
    Y, _, _ = orc.multisketch(A, 2 * n * n, 4 * n, 7)
    assert np.array_equal(np.sign(np.diag(R)), np.sign(np.diag(orc.householder_r(Y))))


@pytest.mark.parametrize("lsig", [-2, -6, -10])
def test_rand_cholqr_lstsq_is_the_exact_minimiser(orc, lsig):
    # Algorithm 5 solves the least-squares problem with no sketching
    # distortion, for kappa(A) < 1/u (Section 6.3): at 1e10, where the normal
    # equations fail, it still lands on the minimiser of the QR solver.
    d, n = 1 << 13, 12
    A, b, _ = inputs.ls_problem(d, n, lsig, seed=32)
    A, b = A.numpy(), b.numpy()
    x, info = orc.rand_cholqr_lstsq(A, b, 2 * n * n, 4 * n, seed=8)
    assert info == 0
    xo = orc.lstsq_exact(A, b)
    ro = orc.relres(A, b, xo)
    # within the 1e-8 relative bar (at kappa 1e10 the two solvers' own
    # O(kappa u) errors differ by ~1e-10 of relres)
    assert abs(orc.relres(A, b, x) - ro) <= 1e-8 * ro
    _, rs, _ = orc.sns_lstsq(A, b, 2 * n * n, 4 * n, seed=8)
    assert ro <= rs  # sketch-and-solve carries the distortion, Algorithm 5 does not
    if lsig == -10:
        xn, infon = orc.ne_lstsq(A, b)
        assert infon > 0 or orc.relres(A, b, xn) > 10 * ro


@pytest.mark.parametrize("kind", ["count", "gauss"])
def test_single_sketch_sns_recovers_and_embeds(orc, kind):
    # Algorithm 1 with the CountSketch alone or the Gaussian alone (the other
    # two sketch-and-solve variants Section 6.3 compares): exact recovery for
    # b = A x, and an O(1) distortion of the least-squares residual
    d, n = 1 << 13, 8
    A, _, _ = inputs.ls_problem(d, n, -2, seed=41)
    A = A.numpy()
    x_true = np.arange(1, n + 1, dtype=np.float64)
    run = (lambda A_, b_, sd: orc.sns_lstsq_count(A_, b_, 2 * n * n, sd)) if kind == "count" \
        else (lambda A_, b_, sd: orc.sns_lstsq_gauss(A_, b_, 4 * n, sd))
    x, rel, _ = run(A, A @ x_true, 3)
    assert np.max(np.abs(x - x_true)) < 1e-11 * np.max(np.abs(x_true)) and rel < 1e-13
    A2, _, _ = inputs.ls_problem(d, n, -2, seed=42)
    b2 = inputs.noisy_rhs(A2, 0.0, 0.01, seed=43).numpy()
    A2 = A2.numpy()
    ro = orc.relres(A2, b2, orc.lstsq_exact(A2, b2))
    for sd in range(3):
        _, rs, _ = run(A2, b2, sd)
        assert ro * (1 - 1e-12) <= rs < 2.0 * ro


def test_gaussian_sketch_preserves_norms_in_expectation(orc):
    # E ||G y||^2 = ||y||^2 for N(0, 1/p) entries: the Frobenius norm of G X
    # over X's columns concentrates around ||X||_F^2 (relative std sqrt(2/p)
    # per column); a dropped 1/sqrt(p) or a wrong variance fails at once
    d, n, p = 4096, 6, 256
    X = np.random.default_rng(5).standard_normal((d, n))
    ratios = [np.linalg.norm(orc.gaussian_sketch(X, p, sd)) ** 2 / np.linalg.norm(X) ** 2
              for sd in range(4)]
    assert abs(np.mean(ratios) - 1.0) < 0.06
