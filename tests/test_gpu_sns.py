"""GPU parity of FP64 sketch-and-solve with each of the three sketches the
paper compares (Section 6.3): the multisketch S = G C, the CountSketch C alone
(QR of the k x (n+1) sketch) and the Gaussian G alone (p x d, generated inside
the product), each against the oracle with the same S: relative residual
within 1e-8 relative, and at least the exact minimiser's."""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("d,n,k,lsig,dt,pad", [
    (20000 + 3, 16, 512, -4, "f64", 0), (65536, 32, 2048, -8, "f64", 1), (30001, 24, 1152, -6, "f32", 0),
    (5000, 8, 128, -2, "f64", 3), (100000, 64, 8192, -6, "f64", 0)])
def test_countsketch_only_sns(msk, orc, d, n, k, lsig, dt, pad):
    dtype = torch.float64 if dt == "f64" else torch.float32
    A, b, _ = inputs.ls_problem(d, n, lsig, seed=800 + n, dtype=dtype)
    seed = 0x5EED0003 + n
    x, info, rc = msk.sns_lstsq(_dev(A, msk, d + pad), b.cuda(), msk.SKETCH_COUNT, k, 0, seed)
    assert rc == 0
    An, bn = A.numpy(), b.numpy()
    rg = orc.relres(An, bn, x.cpu().numpy())
    assert abs(info["relres"] - rg) <= 1e-10 * rg
    _, ro, _ = orc.sns_lstsq_count(An, bn, k, seed)
    assert abs(rg - ro) <= 1e-8 * ro
    re = orc.relres(An, bn, orc.lstsq_exact(An, bn))
    assert rg >= (1 - 1e-8) * re


@pytest.mark.parametrize("d,n,p,lsig,dt,pad", [
    (20000 + 3, 16, 64, -4, "f64", 0), (40000, 32, 128, -6, "f32", 2), (3001, 1, 4, -2, "f64", 0),
    (12345, 20, 21, -3, "f64", 1)])
def test_gaussian_only_sns(msk, orc, d, n, p, lsig, dt, pad):
    dtype = torch.float64 if dt == "f64" else torch.float32
    A, b, _ = inputs.ls_problem(d, n, lsig, seed=900 + n, dtype=dtype)
    seed = 0x5EED0005 + n
    x, info, rc = msk.sns_lstsq(_dev(A, msk, d + pad), b.cuda(), msk.SKETCH_GAUSS, 0, p, seed)
    assert rc == 0
    An, bn = A.numpy(), b.numpy()
    rg = orc.relres(An, bn, x.cpu().numpy())
    assert abs(info["relres"] - rg) <= 1e-10 * rg
    _, ro, _ = orc.sns_lstsq_gauss(An, bn, p, seed)
    assert abs(rg - ro) <= 1e-8 * ro
    re = orc.relres(An, bn, orc.lstsq_exact(An, bn))
    assert rg >= (1 - 1e-8) * re


def test_multisketch_kind_is_ms_lstsq(msk):
    d, n = 30000, 24
    A, b, _ = inputs.ls_problem(d, n, -5, seed=990)
    Ad, bd = _dev(A, msk), b.cuda()
    k, p, seed = 2 * n * n, 4 * n, 17
    x1, i1, rc1 = msk.sns_lstsq(Ad, bd, msk.SKETCH_MULTI, k, p, seed)
    x2, i2, rc2 = msk.ms_lstsq(Ad, bd, k, p, seed, msk.GEMM_F64)
    # the same computation; the atomic CountSketch adds in no fixed order, so
    # the two runs agree to rounding, not bit for bit
    assert rc1 == rc2 == 0
    assert torch.allclose(x1, x2, rtol=1e-9, atol=0)
    assert abs(i1["relres"] - i2["relres"]) <= 1e-9 * i2["relres"]
