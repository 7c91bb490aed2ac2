"""Pins of the oracle's dense steps: Gaussian-stage GEMM (integer-exact
products, low-precision rounding by definition), Householder QR and the
triangular solves of Algorithm 1, Cholesky of the normal equations."""
import os

import numpy as np
import pytest
import torch

import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gemm_integer_exact(orc):
    rng = np.random.default_rng(3)
    G = rng.integers(-50, 51, (37, 300)).astype(np.float64)
    Y = rng.integers(-50, 51, (300, 9)).astype(np.float64)
    Z = orc.gemm(G, Y)
    assert np.array_equal(Z, (G.astype(np.int64) @ Y.astype(np.int64)).astype(np.float64))


def test_gemm_random_within_bound(orc):
    rng = np.random.default_rng(4)
    G = rng.standard_normal((20, 5000))
    Y = rng.standard_normal((5000, 7))
    Z = orc.gemm(G, Y)
    bound = 5000 * np.finfo(float).eps * (np.abs(G) @ np.abs(Y))
    assert np.all(np.abs(Z - G @ Y) <= bound)


def test_round_bf16_golden(orc):
    rows = []
    with open(os.path.join(GOLDEN, "bf16_rounding.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                a, b = (int(t, 16) for t in line.split())
                rows.append((a, b))
    x = np.array([a for a, _ in rows], dtype=np.uint32).view(np.float32)
    got = orc.round_bf16(x).view(np.uint32) >> 16
    assert list(got) == [b for _, b in rows]


def test_round_bf16_and_fp16_match_torch(orc):
    x = np.random.default_rng(5).standard_normal(100000).astype(np.float32) * 3.0
    tb = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    th = torch.from_numpy(x).to(torch.float16).to(torch.float32).numpy()
    assert np.array_equal(orc.round_bf16(x), tb)
    assert np.array_equal(orc.round_fp16(x), th)


@pytest.mark.parametrize("m,c", [(40, 7), (128, 33), (9, 9), (5, 1)])
def test_householder_r(orc, m, c):
    Z = np.random.default_rng(m * 1000 + c).standard_normal((m, c))
    R = orc.householder_r(Z)
    assert np.allclose(np.tril(R, -1), 0)
    # R^T R = Z^T Z
    assert np.allclose(R.T @ R, Z.T @ Z, rtol=0, atol=50 * c * np.finfo(float).eps * np.linalg.norm(Z) ** 2)
    # |R| agrees with LAPACK's QR up to row signs
    Rl = np.linalg.qr(Z, mode="r")
    assert np.allclose(np.abs(R), np.abs(Rl), atol=1e-12 * np.linalg.norm(Z))
    # sign convention: R[j, j] = -sign(x_0) ||x||
    assert R[0, 0] == pytest.approx(-np.sign(Z[0, 0]) * np.linalg.norm(Z[:, 0]))


def test_triangular_solves(orc):
    rng = np.random.default_rng(6)
    R = np.triu(rng.standard_normal((30, 30))) + 10 * np.eye(30)
    c = rng.standard_normal(30)
    assert np.allclose(R @ orc.back_substitution(R, c), c, atol=1e-12)
    assert np.allclose(R.T @ orc.forward_substitution_transposed(R, c), c, atol=1e-12)


def test_lstsq_from_sketch_is_textbook_lstsq(orc):
    # with S = identity the sketched problem is the problem itself: Algorithm 1
    # steps 2-3 on [A b] must give numpy's least-squares solution
    rng = np.random.default_rng(7)
    A = rng.standard_normal((200, 12))
    b = rng.standard_normal(200)
    x, _ = orc.lstsq_from_sketch(np.hstack([A, b[:, None]]))
    xn = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.allclose(x, xn, rtol=1e-12, atol=1e-12)


def test_cholesky(orc):
    rng = np.random.default_rng(8)
    M = rng.standard_normal((50, 10))
    Gm = M.T @ M
    R, info = orc.cholesky_upper(Gm)
    assert info == 0 and np.allclose(R.T @ R, Gm, atol=1e-12 * np.abs(Gm).max())
    assert np.allclose(R, np.linalg.cholesky(Gm).T, atol=1e-12)
    _, info = orc.cholesky_upper(np.diag([1.0, -1.0, 2.0]))
    assert info == 2


def test_split_bf16x3(orc):
    y = (np.random.default_rng(9).standard_normal(20000) * 10.0 ** np.random.default_rng(10).integers(-8, 8, 20000)).astype(np.float32)
    s = orc.split_bf16x3(y)
    # three bfloat16 parts carry 24 significant bits: y is recovered to 2^-24 |y|
    assert np.all(np.abs(s - y.astype(np.float64)) <= 2.0 ** -24 * np.abs(y))
    # values already in bfloat16 are their own first part
    yb = orc.round_bf16(y)
    assert np.array_equal(orc.split_bf16x3(yb), yb.astype(np.float64))
