"""GPU parity of the refinement's operator pass, v = A^T (A p) for FP32 A in
double-single arithmetic (the conjugate-gradient operator of the
preconditioned normal equations, Section 6.3), against the oracle's correctly
rounded sums.  Bound, per element: |v - v*|_j <= 2^-36 (|A|^T |A| |p|)_j
(each product sum carried to about 2^-44 of its terms; the margin covers the
extraction grid, which sits up to 2^4 above a row's largest term).  Shapes
cover every width class (16 .. 256, and the generic body above 256), ragged
row tails, the three copy widths (lda a multiple of 4, even, odd), and
inputs with heavy cancellation: an ill-conditioned A with p in its small
singular directions, column scales over 8 decades, row scales over 10."""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
BOUND = 2.0 ** -36


@pytest.fixture(scope="module")
def msk():
    import paper_2508_14209_gb300 as m
    from paper_2508_14209_gb300 import build

    assert torch.cuda.is_available()
    build.build()
    m.load()
    return m


def _dev(A32, lda=None):
    d, n = A32.shape
    A = inputs.colmajor_empty(d, n, torch.float32, "cuda", lda)
    A.copy_(torch.from_numpy(np.ascontiguousarray(A32)))
    return A


def _check(msk, orc, A32, p, lda=None):
    A = _dev(A32, lda)
    v = msk.msk_normal_apply(A, torch.from_numpy(p).cuda()).cpu().numpy()
    want = orc.normal_apply(A32, p)
    Aa = np.abs(A32.astype(np.float64))
    scale = Aa.T @ (Aa @ np.abs(p))
    err = np.abs(v - want)
    ok = err <= BOUND * scale
    assert ok.all(), (float((err / np.where(scale > 0, scale, 1)).max()), np.flatnonzero(~ok)[:8])
    return float((err / np.where(scale > 0, scale, 1)).max())


@pytest.mark.parametrize("d,n,lda_pad", [(1, 1, 0), (37, 5, 0), (1000, 16, 3), (4099, 17, 1),
                                         (2053, 32, 0), (5000, 64, 4), (1027, 100, 2),
                                         (3001, 128, 0), (1500, 200, 1), (777, 256, 0),
                                         (900, 300, 0), (20000, 64, 0)])
def test_normal_apply_random(msk, orc, d, n, lda_pad):
    rng = np.random.default_rng(d * 31 + n)
    A32 = rng.standard_normal((d, n)).astype(np.float32)
    p = rng.standard_normal(n)
    _check(msk, orc, A32, p, d + lda_pad)


@pytest.mark.parametrize("n", [16, 64, 128, 256])
def test_normal_apply_ill_conditioned(msk, orc, n):
    # A = G diag(sigma) V^T with sigma down to 1e-8 and p = V diag(1/sigma) z:
    # A p is about G z while |A| |p| is about 1e8 larger
    d = 6000
    A, _, _ = inputs.ls_problem(d, n, -8.0, seed=n, dtype=torch.float32)
    A32 = A.numpy()
    V = inputs.haar_orthogonal(n, n).numpy()
    sig = inputs.log_spaced_sigma(n, -8.0).numpy()
    z = np.random.default_rng(n).standard_normal(n)
    p = V @ (z / sig)
    _check(msk, orc, A32, p)


def test_normal_apply_column_and_row_scales(msk, orc):
    rng = np.random.default_rng(5)
    d, n = 3000, 48
    s = np.power(10.0, -8.0 * np.arange(n) / (n - 1))
    rs = np.power(10.0, -10.0 * rng.random(d))
    A32 = (rng.standard_normal((d, n)) * s[None, :] * rs[:, None]).astype(np.float32)
    p = rng.standard_normal(n) / s
    _check(msk, orc, A32, p)


def test_normal_apply_zero_and_bad_arguments(msk):
    A = inputs.colmajor_empty(100, 8, torch.float32, "cuda")
    A.zero_()
    v = msk.msk_normal_apply(A, torch.ones(8, dtype=torch.float64, device="cuda"))
    assert torch.count_nonzero(v).item() == 0
    L = msk.load()
    assert L.msk_normal_apply_workspace(0, 8) == 0
    assert L.msk_normal_apply_workspace(100, 513) == 0
    assert L.msk_normal_apply(None, 100, 8, 100, None, None, None, 0, None) == -1
