"""GPU parity of the tcgen05 tensor-core Gaussian stage (BF16, FP16 and the
split-BF16x3 products) against the oracle on the same FP32 Y: the oracle
rounds / splits the same binary32 values (same decisions), then contracts in
FP64; the GPU's FP32 accumulation stays within (parts*k + 2) * 2^-24 sum|G||Y|."""
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


SHAPES = [(128, 64, 16), (64, 1000, 1), (256, 8192, 64), (256, 8192, 65), (200, 777, 33),
          (512, 4096, 129), (1024, 2048, 257), (384, 640, 300)]


@pytest.mark.parametrize("prec", ["bf16", "f16", "bf16x3"])
@pytest.mark.parametrize("p,k,ncol", SHAPES)
def test_tensor_gemm_matches_oracle(msk, orc, prec, p, k, ncol):
    seed = 0x5EED0006 + p + ncol
    Y = torch.randn(k, ncol, generator=torch.Generator().manual_seed(k + ncol), dtype=torch.float32)
    Z = msk.msk_gemm(seed, p, Y.cuda(), gemm_prec=msk.GEMM_PRECS[prec])
    torch.cuda.synchronize()
    Zg = Z.cpu().numpy()
    G = orc.gaussian(seed, p, k)
    if prec == "bf16":
        Gu, Yu = orc.round_bf16(G), orc.round_bf16(Y.numpy())
    elif prec == "f16":
        Gu, Yu = orc.round_fp16(G), orc.round_fp16(Y.numpy())
    else:
        Gu, Yu = orc.round_bf16(G), orc.split_bf16x3(Y.numpy())
    Gu, Yu = Gu.astype(np.float64), Yu.astype(np.float64)
    Zo = orc.gemm(Gu, Yu)
    assert msk.msk_take_timeout() == msk.MSK_OK  # no bounded wait gave up
    parts = 3 if prec == "bf16x3" else 1
    bound = (parts * k + 2) * 2.0 ** -24 * (np.abs(Gu) @ np.abs(Yu))
    assert np.all(np.abs(Zg - Zo) <= bound)


def test_tensor_gemm_is_deterministic(msk):
    Y = torch.randn(8192, 65, dtype=torch.float32, device="cuda")
    Z1 = msk.msk_gemm(3, 256, Y, gemm_prec=msk.GEMM_BF16X3).clone()
    Z2 = msk.msk_gemm(3, 256, Y, gemm_prec=msk.GEMM_BF16X3)
    assert torch.equal(Z1, Z2)


@pytest.mark.parametrize("d,n", [(40000, 64), (5001, 8)])
def test_multisketch_bf16x3_end_to_end(msk, orc, d, n):
    k, p, seed = 2 * n * n, 4 * n, 0x5EED0007
    A = inputs.normal_matrix(d, n, seed, torch.float32)
    b = inputs.normal_matrix(d, 1, seed + 1)[:, 0].contiguous()
    Ad = msk.colmajor(d, n, torch.float32, "cuda")
    Ad.copy_(A)
    Z = msk.ms_sketch(Ad, k, p, seed, b=b.cuda(), gemm_prec=msk.GEMM_BF16X3).cpu().numpy()
    bn = b.numpy().astype(np.float32).astype(np.float64)
    Zo, Gu, Yu = orc.multisketch(A.numpy(), k, p, seed, b=bn, gemm_prec="bf16x3")
    absY = orc.bucket_abs_sums(A.numpy(), k, seed, b=bn)
    bound = (3 * k + 2) * 2.0 ** -24 * (np.abs(Gu) @ np.abs(Yu)) + np.abs(Gu) @ (2e-5 * absY)
    assert np.all(np.abs(Z - Zo) <= bound)


@pytest.mark.parametrize("d,n,lsig", [(1 << 15, 32, -8), (60000, 64, -6)])
def test_refined_bf16x3_reaches_minimiser(msk, orc, d, n, lsig):
    A, b, _ = inputs.ls_problem(d, n, lsig, seed=500 + n, dtype=torch.float32)
    k, p, seed = 2 * n * n, 4 * n, 0x5EED0008
    Ad = msk.colmajor(d, n, torch.float32, "cuda")
    Ad.copy_(A)
    x, info, rc = msk.ms_lstsq(Ad, b.cuda(), k, p, seed, msk.GEMM_BF16X3, refine=True, tol=1e-12,
                               max_iter=20)
    assert rc == 0, info
    An, bn = A.numpy(), b.numpy()
    ro = orc.relres(An, bn, orc.lstsq_exact(An, bn))
    rg = orc.relres(An, bn, x.cpu().numpy())
    assert abs(rg - ro) <= 1e-8 * ro
    _, r_sns64, _ = orc.sns_lstsq(An.astype(np.float64), bn, k, p, seed, "f64")
    assert rg <= (1 + 1e-8) * r_sns64


def test_bounded_wait_expires_and_is_reported(msk):
    """An mbarrier wait that nothing completes gives up after its limit (1 s),
    records a timeout that msk_take_timeout reports once, and leaves the
    context usable."""
    assert msk.msk_take_timeout() == msk.MSK_OK
    msk.msk_selftest_wait()
    assert msk.msk_take_timeout() == msk.MSK_ETIMEOUT
    assert msk.msk_take_timeout() == msk.MSK_OK  # the record was cleared
    Y = torch.randn(1024, 9, dtype=torch.float32, device="cuda")
    Z = msk.msk_gemm(5, 32, Y, gemm_prec=msk.GEMM_BF16)
    assert torch.isfinite(Z).all() and msk.msk_take_timeout() == msk.MSK_OK


def _f64_stage_inputs(k, ncol, seed):
    """FP64 Y with N(0,1) columns and, where there is room, the awkward ones:
    a zero column, a column of subnormal-scale entries (1e-310), one spanning
    six decades, one of huge entries (1e300) and one with a single nonzero."""
    g = torch.Generator().manual_seed(seed)
    Y = torch.randn(k, ncol, generator=g, dtype=torch.float64)
    if ncol >= 6:
        Y[:, 1] = 0.0
        Y[:, 2] *= 1e-310
        Y[:, 3] = torch.sign(Y[:, 3]) * 10.0 ** (-6.0 * torch.rand(k, generator=g, dtype=torch.float64))
        Y[:, 4] *= 1e300
        Y[:, 5] = 0.0
        Y[k // 3, 5] = -3.25
    return Y


# The FP64 Gaussian stage from k = 1024 up runs on the tensor cores by exact
# 8-bit slicing of G and Y; below, and with the knob off, on the FP64 SIMT
# kernel.  Both must stay within the FP64 dot-product bound of the oracle's
# compensated product on the same binary32 G, and give the same Z to that
# bound as each other; repeated calls are bitwise equal.
@pytest.mark.parametrize("p,k,ncol", [(256, 8192, 64), (512, 32768, 129), (200, 1024, 1), (130, 5000, 65),
                                      (1024, 2048, 257), (128, 1024, 16), (300, 3001, 7), (64, 1500, 33)])
def test_f64_stage_sliced_matches_oracle(msk, orc, p, k, ncol):
    seed = 0x5EED0007 + p + ncol
    Y = _f64_stage_inputs(k, ncol, k + ncol)
    Yd = Y.cuda()
    Z = msk.msk_gemm(seed, p, Yd, gemm_prec=msk.GEMM_F64).cpu().numpy()
    Z2 = msk.msk_gemm(seed, p, Yd, gemm_prec=msk.GEMM_F64).cpu().numpy()
    assert msk.msk_take_timeout() == msk.MSK_OK
    assert np.array_equal(Z, Z2)
    G = orc.gaussian(seed, p, k).astype(np.float64)
    Yh = Y.numpy()
    Zo = orc.gemm(G, Yh)
    bound = (k + 2) * np.finfo(np.float64).eps * (np.abs(G) @ np.abs(Yh))
    assert np.all(np.abs(Z - Zo) <= bound)
    msk.tune_set("gemm.f64_ozaki", 0)
    try:
        Zs = msk.msk_gemm(seed, p, Yd, gemm_prec=msk.GEMM_F64).cpu().numpy()
    finally:
        msk.tune_clear("gemm.f64_ozaki")
    assert np.all(np.abs(Zs - Zo) <= bound)
