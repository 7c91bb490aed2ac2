"""GPU parity of the SRHT (Section 5) against the oracle, through the C ABI:
bit-exact on integer-valued inputs (every butterfly sum is exact, so only the
final division by sqrt(k) rounds, once on each side), within the FP64
transform's error bound on Gaussian inputs, for one-pass (d <= 2^13) and
two-pass columns up to 2^23 rows; and sketch-and-solve with it within 1e-8
of the oracle's with the same S."""
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


@pytest.mark.parametrize("d,n,k,with_b,pad,dt", [
    (2, 1, 3, False, 0, "f64"), (16, 3, 7, True, 1, "f64"), (8192, 5, 100, True, 0, "f64"),
    (16384, 4, 1000, False, 0, "f64"), (1 << 17, 7, 4096, True, 4, "f64"),
    (1 << 20, 2, 5000, True, 0, "f32"), (1 << 23, 1, 2000, True, 0, "f64")])
def test_srht_integer_inputs_bit_exact(msk, orc, d, n, k, with_b, pad, dt):
    dtype = torch.float64 if dt == "f64" else torch.float32
    A = inputs.integer_matrix(d, n, 70 + n, lo=-5, hi=5, dtype=dtype)
    b = inputs.integer_matrix(d, 1, 71 + n, lo=-5, hi=5)[:, 0].contiguous() if with_b else None
    seed = 0x5EED0009 + d
    Y = msk.srht_sketch(_dev(A, msk, d + pad), k, seed, b=None if b is None else b.cuda())
    Yo = orc.srht(A.numpy(), k, seed, b=None if b is None else b.numpy())
    assert np.array_equal(Y.cpu().numpy(), Yo)


@pytest.mark.parametrize("d,n,k,with_b", [(4096, 9, 333, True), (1 << 15, 33, 2048, False),
                                          (1 << 19, 16, 8192, True)])
def test_srht_gaussian_inputs_within_bound(msk, orc, d, n, k, with_b):
    A = inputs.normal_matrix(d, n, 80 + n)
    b = inputs.normal_matrix(d, 1, 81 + n)[:, 0].contiguous() if with_b else None
    seed = 0x5EED000A + d
    Y = msk.srht_sketch(_dev(A, msk), k, seed, b=None if b is None else b.cuda()).cpu().numpy()
    An = A.numpy()
    X = An if b is None else np.hstack([An, b.numpy()[:, None]])
    Yo = orc.srht(An, k, seed, b=None if b is None else b.numpy())
    # each output is a +-1 sum of the column's d entries through m = log2(d)
    # levels of additions (error <= m u sum|x| on each side), then one division
    m = int(np.log2(d))
    bound = (2 * m + 2) * EPS64 * np.abs(X).sum(axis=0) / np.sqrt(k)
    assert np.all(np.abs(Y - Yo) <= bound[None, :])


@pytest.mark.parametrize("d,n,k,lsig,dt", [(1 << 14, 16, 512, -4, "f64"), (1 << 17, 32, 2048, -8, "f64"),
                                           (1 << 16, 24, 1152, -6, "f32")])
def test_srht_sns(msk, orc, d, n, k, lsig, dt):
    dtype = torch.float64 if dt == "f64" else torch.float32
    A, b, _ = inputs.ls_problem(d, n, lsig, seed=1000 + n, dtype=dtype)
    seed = 0x5EED000B + n
    x, info, rc = msk.sns_lstsq(_dev(A, msk), b.cuda(), msk.SKETCH_SRHT, k, 0, seed)
    assert rc == 0
    An, bn = A.numpy(), b.numpy()
    rg = orc.relres(An, bn, x.cpu().numpy())
    assert abs(info["relres"] - rg) <= 1e-9 * rg
    _, ro, _ = orc.sns_lstsq_srht(An, bn, k, seed)
    assert abs(rg - ro) <= 1e-8 * ro
    re = orc.relres(An, bn, orc.lstsq_exact(An, bn))
    assert rg >= (1 - 1e-8) * re
