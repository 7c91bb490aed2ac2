"""GPU parity of the sketching steps against the CPU oracle, through the
C ABI: hash/sign bit-exact, Gaussian bit-exact, CountSketch within
64 eps64 (FP64) / 1e-5 (FP32) of each bucket's absolute sum, multisketch within
the GEMM rounding bound."""
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


def to_dev(A, lda=None):
    """Host column-major tensor -> device column-major (optionally lda > d)."""
    import paper_2508_14209_gb300 as m

    d, n = A.shape
    Ad = m.colmajor(d, n, A.dtype, "cuda", lda=lda)
    Ad.copy_(A)
    return Ad


@pytest.mark.parametrize("i0,count,k", [(0, 1 << 20, 2048), (12345, 100000, 1000),
                                        (0, 1 << 24, 131072), (5, 7, 1), (0, 0, 3)])
def test_hash_bit_exact(msk, orc, i0, count, k):
    seed = 0x5EED0001
    h, s = msk.cs_hash(seed, i0, count, k)
    ho, so = orc.hash_rows(seed, i0, count, k)
    assert np.array_equal(h.cpu().numpy().astype(np.uint32), ho)
    assert np.array_equal(s.cpu().numpy(), so)


@pytest.mark.parametrize("p,k", [(256, 8192), (7, 333), (1, 1)])
def test_gaussian_bit_exact(msk, orc, p, k):
    seed = 0x5EED0002
    Go = orc.gaussian(seed, p, k)
    G32 = msk.ms_gaussian(seed, p, k, msk.GEMM_F32).cpu().numpy()
    assert np.array_equal(G32.view(np.uint32), Go.view(np.uint32))
    G64 = msk.ms_gaussian(seed, p, k, msk.GEMM_F64).cpu().numpy()
    assert np.array_equal(G64, Go.astype(np.float64))
    Gb = msk.ms_gaussian(seed, p, k, msk.GEMM_BF16).float().cpu().numpy()
    assert np.array_equal(Gb, orc.round_bf16(Go))
    Gh = msk.ms_gaussian(seed, p, k, msk.GEMM_F16).float().cpu().numpy()
    assert np.array_equal(Gh, orc.round_fp16(Go))


CASES = [  # d, n, k, with_b, lda_pad
    (0, 3, 5, False, 0), (1, 1, 1, False, 0), (31, 2, 7, True, 3), (33, 5, 11, False, 1),
    (1000, 1, 37, True, 0), (1000, 32, 64, False, 0), (4097, 33, 2048, True, 5),
    (65536 + 17, 64, 2048, True, 0), (20000, 129, 512, False, 2), (3000, 257, 300, True, 0),
    (700, 600, 40, True, 0),
]


def _inputs(d, n, with_b, dtype, seed, lda_pad):
    A = inputs.normal_matrix(d, n, seed, dtype)
    b = inputs.normal_matrix(d, 1, seed + 1)[:, 0].contiguous() if with_b else None
    return A, b, to_dev(A, lda=d + lda_pad if d else None), (None if b is None else b.cuda())


@pytest.mark.parametrize("strategy", [0, 1])
@pytest.mark.parametrize("d,n,k,with_b,lda_pad", CASES)
def test_countsketch_f64(msk, orc, strategy, d, n, k, with_b, lda_pad):
    seed = 0x5EED0001 + d
    A, b, Ad, bd = _inputs(d, n, with_b, torch.float64, seed, lda_pad)
    Y = msk.cs_sketch(Ad, k, seed, b=bd, strategy=strategy).cpu().numpy()
    An, bn = A.numpy(), (None if b is None else b.numpy())
    Yo = orc.countsketch(An, k, seed, b=bn)
    tol = 64 * EPS64 * orc.bucket_abs_sums(An, k, seed, b=bn)
    assert np.all(np.abs(Y - Yo) <= tol)


@pytest.mark.parametrize("strategy", [0, 1])
@pytest.mark.parametrize("d,n,k,with_b,lda_pad", CASES)
def test_countsketch_f32(msk, orc, strategy, d, n, k, with_b, lda_pad):
    seed = 0x5EED0002 + d
    A, b, Ad, bd = _inputs(d, n, with_b, torch.float32, seed, lda_pad)
    Y = msk.cs_sketch(Ad, k, seed, b=bd, strategy=strategy).cpu().numpy().astype(np.float64)
    An = A.numpy()
    bn = None if b is None else b.numpy().astype(np.float32).astype(np.float64)  # GPU rounds b
    Yo = orc.countsketch(An, k, seed, b=bn)
    tol = 1e-5 * orc.bucket_abs_sums(An, k, seed, b=bn)
    assert np.all(np.abs(Y - Yo) <= tol)


# FP32 sketches with few buckets run the shared-memory-privatised kernel
# (k <= 256 by default, any k that fits with cs.f32.priv = 2; rows >= 16 k;
# k x cs floats per CTA, cs >= 4 columns per slice): one slice (k = 512),
# four slices (k = 2048, 33 columns), a ragged last chunk, lda padding; the
# knob cs.f32.priv = 0 gives the tile kernels on the same input.
@pytest.mark.parametrize("d,n,k,with_b,lda_pad", [(40000, 16, 512, True, 0), (150001, 32, 2048, True, 3),
                                                 (70001, 9, 300, False, 1), (200000, 33, 2048, False, 0),
                                                 (16384, 1, 512, True, 0), (50000, 8, 128, True, 2)])
@pytest.mark.parametrize("priv", [2, 1, 0])
def test_countsketch_f32_private(msk, orc, d, n, k, with_b, lda_pad, priv):
    seed = 0x5EED0006 + d
    A, b, Ad, bd = _inputs(d, n, with_b, torch.float32, seed, lda_pad)
    msk.tune_set("cs.f32.priv", priv)
    try:
        Y = msk.cs_sketch(Ad, k, seed, b=bd).cpu().numpy().astype(np.float64)
    finally:
        msk.tune_clear("cs.f32.priv")
    An = A.numpy()
    bn = None if b is None else b.numpy().astype(np.float32).astype(np.float64)
    Yo = orc.countsketch(An, k, seed, b=bn)
    tol = 1e-5 * orc.bucket_abs_sums(An, k, seed, b=bn)
    assert np.all(np.abs(Y - Yo) <= tol)


def test_countsketch_row_pitch(msk, orc):
    # Y with a leading dimension larger than ncol: the padding is left alone
    d, n, k, seed = 5000, 9, 100, 17
    A = inputs.normal_matrix(d, n, seed)
    Ybig = torch.full((k, 16), 7.0, dtype=torch.float64, device="cuda")
    msk.cs_sketch(to_dev(A), k, seed, Y=Ybig[:, :n])
    Yc = Ybig.cpu().numpy()
    assert np.all(Yc[:, n:] == 7.0)
    Yo = orc.countsketch(A.numpy(), k, seed)
    assert np.all(np.abs(Yc[:, :n] - Yo) <= 64 * EPS64 * orc.bucket_abs_sums(A.numpy(), k, seed))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_integer_inputs_exact_any_order(msk, orc, dtype):
    d, n, k, seed = 200000, 7, 1024, 23
    A = inputs.integer_matrix(d, n, 3, dtype=dtype)
    Yo = orc.countsketch(A.numpy(), k, seed)
    for strategy in (0, 1):
        Y = msk.cs_sketch(to_dev(A), k, seed, strategy=strategy).cpu().numpy().astype(np.float64)
        assert np.array_equal(Y, Yo)


def test_sorted_is_bitwise_reproducible(msk):
    d, n, k, seed = 300001, 17, 4096, 99
    Ad = to_dev(inputs.normal_matrix(d, n, seed))
    Y1 = msk.cs_sketch(Ad, k, seed, strategy=1)
    Y2 = msk.cs_sketch(Ad, k, seed, strategy=1)
    assert torch.equal(Y1, Y2)


def test_sorted_long_bucket_lists(msk, orc):
    # k = 1: one bucket holding every row (exercises the long-list sort path)
    d, n, seed = 5000, 3, 5
    A = inputs.normal_matrix(d, n, seed)
    Y = msk.cs_sketch(to_dev(A), 1, seed, strategy=1).cpu().numpy()
    Yo = orc.countsketch(A.numpy(), 1, seed)
    assert np.all(np.abs(Y - Yo) <= 64 * EPS64 * orc.bucket_abs_sums(A.numpy(), 1, seed))


def test_full_size_sampled_buckets_f64(msk, orc):
    # configs: 65536 x 32 (k = 2048) whole, 2^22 x 64 (k = 8192) on sampled buckets
    for d, n, k, seed in ((65536, 32, 2048, 0x5EED0001), (1 << 22, 64, 8192, 0x5EED0002)):
        A = inputs.normal_matrix(d, n, seed, device="cuda")
        Y = msk.cs_sketch(A, k, seed).cpu().numpy()
        Ah = A.cpu().numpy()
        lst = np.unique(np.r_[np.random.default_rng(1).integers(0, k, 48), 0, k - 1])
        Yb, ab, _ = orc.countsketch_buckets(Ah, k, seed, lst)
        assert np.all(np.abs(Y[lst] - Yb) <= 64 * EPS64 * ab)
        # column sums of SA equal s^T A: a property of every entry at once
        _, s = orc.hash_rows(seed, 0, d, k)
        cs = s.astype(np.float64) @ Ah
        assert np.allclose(Y.sum(axis=0), cs, rtol=0, atol=1e-9 * np.abs(Ah).sum(axis=0).max())


@pytest.mark.parametrize("prec", ["f64", "f32"])
# column counts 7, 32, 4, 64, 129, 65, 33: tiles of 32, 48 and 64 columns
@pytest.mark.parametrize("d,n,k,p,with_b,dtype", [
    (5000, 6, 72, 24, True, torch.float64), (20000, 32, 2048, 128, False, torch.float64),
    (3001, 3, 18, 12, True, torch.float32), (40000, 64, 8192, 256, False, torch.float32),
    (30000, 128, 4096, 200, True, torch.float64), (12000, 64, 2048, 130, True, torch.float64),
    (9000, 32, 1024, 97, True, torch.float32)])
def test_multisketch_simt(msk, orc, prec, d, n, k, p, with_b, dtype):
    seed = 0x5EED0003 + n
    A, b, Ad, bd = _inputs(d, n, with_b, dtype, seed, 0)
    gp = msk.GEMM_PRECS[prec]
    Z = msk.ms_sketch(Ad, k, p, seed, b=bd, gemm_prec=gp).cpu().numpy()
    An = A.numpy()
    bn = None if b is None else (b.numpy() if dtype == torch.float64 else
                                 b.numpy().astype(np.float32).astype(np.float64))
    Zo, Gu, Yu = orc.multisketch(An, k, p, seed, b=bn, gemm_prec=prec)
    u_cs = 64 * EPS64 if dtype == torch.float64 else 1e-5
    u_mm = EPS64 if prec == "f64" else 2.0 ** -24
    absY = orc.bucket_abs_sums(An, k, seed, b=bn)
    bound = (k + 2) * u_mm * (np.abs(Gu) @ np.abs(Yu)) + np.abs(Gu) @ (u_cs * absY)
    assert np.all(np.abs(Z - Zo) <= bound)


def test_multisketch_stage_events_and_side_stream(msk, orc):
    """With "ms.overlap_gauss" the FP64 multisketch samples G's slices on a
    side stream beside its CountSketch; the result is the oracle's within the
    FP64 bound with and without it, and the stage-event hook's events bracket
    the CountSketch inside the call's span."""
    d, n, k, p, seed = 70001, 64, 8192, 256, 0x5EED0009
    A = inputs.normal_matrix(d, n, seed, dtype=torch.float64)
    Ad = msk.colmajor(d, n, torch.float64, "cuda")
    Ad.copy_(A)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    msk.tune_set("ms.overlap_gauss", 1)
    try:
        ev[0].record()
        Z = msk.ms_sketch(Ad, k, p, seed, gemm_prec=msk.GEMM_F64, cs_events=(ev[1], ev[2]))
        ev[3].record()
        torch.cuda.synchronize()
    finally:
        msk.tune_clear("ms.overlap_gauss")
    Z2 = msk.ms_sketch(Ad, k, p, seed, gemm_prec=msk.GEMM_F64).cpu().numpy()
    cs_ms, all_ms = ev[1].elapsed_time(ev[2]), ev[0].elapsed_time(ev[3])
    assert 0.0 < cs_ms <= all_ms
    Zo, Gu, Yu = orc.multisketch(A.numpy(), k, p, seed, gemm_prec="f64")
    absY = orc.bucket_abs_sums(A.numpy(), k, seed)
    bound = (k + 2) * EPS64 * (np.abs(Gu) @ np.abs(Yu)) + np.abs(Gu) @ (64 * EPS64 * absY)
    for Zg in (Z.cpu().numpy(), Z2):
        assert np.all(np.abs(Zg - Zo) <= bound)
