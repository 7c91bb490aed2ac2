"""GPU parity of randomized Cholesky QR (Section 6.3, Algorithms 4 and 5)
against the oracle, through the C ABI, with the same sketch S = G C as the
oracle: the least-squares solution is the minimiser (relative residual within
1e-8 of the oracle's QR solver, no sketching distortion, at kappa up to 1e10
where the normal equations fail); the factorisation is A's own QR (Q and R
equal to the oracle's to ~kappa u, Q^T Q = I, Q R = A), also in place."""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu
EPS64 = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def msk():
    import paper_2508_14209_gb300 as m
    from paper_2508_14209_gb300 import build

    assert torch.cuda.is_available()
    build.build()
    m.load()
    return m


def _dev(A, msk, lda=None):
    d, n = A.shape
    out = msk.colmajor(d, n, A.dtype, "cuda", lda=lda)
    out.copy_(A)
    return out


# Sketch sizes: the paper's k = 2 n^2, p = 4 n where the oracle's plain
# (compensated) G Y product stays within a few seconds; smaller k and p
# (p >= n + 1) for the widest cases.
CASES = [  # d, n, k, p, log10 sigma_min, dtype, gemm precision, lda padding
    (20000 + 3, 128, 4096, 512, -6, "f64", "f64", 0), (5003, 37, 2738, 148, -10, "f64", "f64", 2),
    (3001, 1, 4, 4, -2, "f64", "f64", 0), (9000, 256, 4096, 512, -4, "f64", "f64", 0),
    (40000, 64, 8192, 256, -8, "f32", "bf16x3", 0), (30001, 48, 4608, 192, -6, "f32", "f32", 1),
    (7001, 400, 2048, 416, -3, "f64", "f64", 0),
]


@pytest.mark.parametrize("d,n,k,p,lsig,dt,prec,pad", CASES)
def test_rcq_lstsq_is_the_minimiser(msk, orc, d, n, k, p, lsig, dt, prec, pad):
    dtype = torch.float64 if dt == "f64" else torch.float32
    A, b, _ = inputs.ls_problem(d, n, lsig, seed=500 + n, dtype=dtype)
    seed = 0x5EED0003 + n
    x, info, rc = msk.rcq_lstsq(_dev(A, msk, d + pad), b.cuda(), k, p, seed,
                                msk.GEMM_PRECS[prec])
    assert rc == 0
    An, bn = A.numpy(), b.numpy()
    xg = x.cpu().numpy()
    rg = orc.relres(An, bn, xg)
    # the library's residual is a plain FP64 pass, the oracle's compensated:
    # at kappa 1e10 the cancellation in b - A x leaves ~1e-10 between them
    assert abs(info["relres"] - rg) <= 1e-8 * rg
    xo, io = orc.rand_cholqr_lstsq(An, bn, k, p, seed, prec)
    assert io == 0
    ro = orc.relres(An, bn, xo)
    re = orc.relres(An, bn, orc.lstsq_exact(An, bn))
    assert abs(rg - re) <= 1e-8 * re
    assert abs(rg - ro) <= 1e-8 * ro
    _, rs, _ = orc.sns_lstsq(An, bn, k, p, seed, prec)
    assert rg <= (1 + 1e-8) * rs


@pytest.mark.parametrize("d,n,k,p,lsig,dt,prec,inplace", [
    (20000 + 3, 128, 4096, 512, -6, "f64", "f64", False), (4099, 33, 2178, 132, -2, "f64", "f64", True),
    (3001, 1, 4, 4, -2, "f64", "f64", False), (50000, 64, 8192, 256, -4, "f32", "bf16x3", False),
    (9000, 300, 2048, 320, -5, "f64", "f64", True)])
def test_rcq_qr_is_the_qr_of_A(msk, orc, d, n, k, p, lsig, dt, prec, inplace):
    dtype = torch.float64 if dt == "f64" else torch.float32
    A, _, _ = inputs.ls_problem(d, n, lsig, seed=600 + n, dtype=dtype)
    seed = 0x5EED0007 + n
    Ad = _dev(A, msk)
    Q, R, rc = msk.rcq_qr(Ad, k, p, seed, msk.GEMM_PRECS[prec], Q=Ad if inplace else None)
    assert rc == 0
    if inplace:
        assert Q.data_ptr() == Ad.data_ptr()
    An = A.numpy().astype(np.float64)
    Qg, Rg = Q.cpu().numpy(), R.cpu().numpy()
    assert np.all(np.tril(Rg, -1) == 0.0)
    nA = np.linalg.norm(An, 2)
    kappa = 10.0 ** (-lsig)
    assert np.abs(Qg.T @ Qg - np.eye(n)).max() < 100 * n * EPS64
    assert np.abs(Qg @ Rg - An).max() < 100 * n * EPS64 * nA
    Qo, Ro, io = orc.rand_cholqr(A.numpy(), k, p, seed, prec)
    assert io == 0
    assert np.allclose(Rg, Ro, rtol=0, atol=100 * n * kappa * EPS64 * nA)
    assert np.allclose(Qg, Qo, rtol=0, atol=100 * n * kappa * EPS64)


def test_rcq_zero_column_reports_the_pivot(msk):
    d, n = 4096, 12
    A, b, _ = inputs.ls_problem(d, n, -2, seed=700)
    A[:, 5] = 0.0
    x, _, rc = msk.rcq_lstsq(_dev(A, msk), b.cuda(), 2 * n * n, 4 * n, 9)
    assert rc == 6 and torch.isnan(x).all()
    _, _, rc = msk.rcq_qr(_dev(A, msk), 2 * n * n, 4 * n, 9)
    assert rc == 6
