"""ms_sketch_host (the multisketch of a HOST matrix, streamed in row blocks
that are copied while the previous block is sketched) against the oracle and
against ms_sketch on the device copy: same Z within the multisketch bound, for
ragged blocks, padded leading dimensions, pinned and pageable host memory,
FP64 and FP32 A, the narrow kernels with replicas of Y, the FP64 sketch of
FP32 A and the split-BF16 tensor-core stage.  And ms_sketch_rows: the blocks
of a row partition (global row indices) add up to the whole matrix's Z."""
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


def _host(A, lda, pinned):
    d, n = A.shape
    buf = torch.empty((max(n, 1), lda), dtype=A.dtype, pin_memory=pinned)
    H = buf[:n, :d].t()
    H.copy_(A)
    return H


@pytest.mark.parametrize("d,n,k,p,with_b,dt,prec,chunk,pad,pinned", [
    (50000, 7, 98, 28, True, "f64", "f64", 4096, 0, True),
    (50001, 64, 8192, 256, False, "f64", "f64", 0, 0, False),
    (40000, 16, 512, 64, True, "f32", "bf16x3", 1000, 0, True),
    (30000, 16, 512, 64, True, "f64", "f64", 3000, 5, True),
    (20000, 33, 2178, 132, True, "f32", "f64", 777, 2, True),
    (3000, 5, 50, 20, False, "f64", "f64", 4096, 0, True)])
def test_ms_sketch_host_matches(msk, orc, d, n, k, p, with_b, dt, prec, chunk, pad, pinned):
    dtype = torch.float64 if dt == "f64" else torch.float32
    seed = 0x5EED000C + n
    A = inputs.normal_matrix(d, n, seed, dtype)
    b = inputs.normal_matrix(d, 1, seed + 1)[:, 0].contiguous() if with_b else None
    Ah = _host(A, d + pad, pinned)
    bh = None if b is None else (b.pin_memory() if pinned else b)
    gp = msk.GEMM_PRECS[prec]
    Z = msk.ms_sketch_host(Ah, k, p, seed, b=bh, gemm_prec=gp, chunk_rows=chunk).numpy()
    Ad = msk.colmajor(d, n, dtype, "cuda")
    Ad.copy_(A)
    Zd = msk.ms_sketch(Ad, k, p, seed, b=None if b is None else b.cuda(), gemm_prec=gp).cpu().numpy()
    An = A.numpy()
    ydt64 = dtype == torch.float64 or prec == "f64"
    bn = None if b is None else (b.numpy() if ydt64 else b.numpy().astype(np.float32).astype(np.float64))
    Zo, Gu, Yu = orc.multisketch(An, k, p, seed, b=bn, gemm_prec=prec)
    u_cs = 64 * EPS64 if dtype == torch.float64 else 1e-5
    u_mm = EPS64 if prec == "f64" else 2.0 ** -24
    parts = 3 if prec == "bf16x3" else 1
    absY = orc.bucket_abs_sums(An, k, seed, b=bn)
    bound = (parts * k + 2) * u_mm * (np.abs(Gu) @ np.abs(Yu)) + np.abs(Gu) @ (u_cs * absY)
    assert np.all(np.abs(Z - Zo) <= bound)
    assert np.all(np.abs(Z - Zd) <= 2 * bound)


def test_ms_sketch_host_empty_rows(msk):
    A = torch.empty((0, 3), dtype=torch.float64)
    Z = msk.ms_sketch_host(A.t().contiguous().t(), 10, 4, 1, gemm_prec=msk.GEMM_F64)
    assert Z.shape == (4, 3) and torch.count_nonzero(Z) == 0


@pytest.mark.parametrize("dt,prec,nblk", [("f64", "f64", 3), ("f32", "bf16x3", 4), ("f32", "f64", 2)])
def test_ms_sketch_rows_blocks_add_up(msk, orc, dt, prec, nblk):
    """Section 7's row distribution on one GPU: the multisketches of the
    blocks of a row partition (global row indices) add up to the whole
    matrix's, as the all-reduce of ms_sketch_distributed assumes."""
    from paper_2508_14209_gb300.distributed import ms_sketch_distributed, row_partition

    dtype = torch.float64 if dt == "f64" else torch.float32
    d, n, k, p, seed = 30011, 12, 288, 48, 0x5EED000D
    A = inputs.normal_matrix(d, n, seed, dtype)
    b = inputs.normal_matrix(d, 1, seed + 1)[:, 0].contiguous()
    gp = msk.GEMM_PRECS[prec]
    Ad = msk.colmajor(d, n, dtype, "cuda")
    Ad.copy_(A)
    bd = b.cuda()
    Zs = 0
    for r in range(nblk):
        r0, m = row_partition(d, nblk, r)
        Ab = msk.colmajor(m, n, dtype, "cuda")
        Ab.copy_(A[r0:r0 + m])
        Zr = ms_sketch_distributed(Ab, r0, k, p, seed, b_local=bd[r0:r0 + m].contiguous(), gemm_prec=gp)
        Zs = Zs + Zr.cpu().numpy()
    An = A.numpy()
    ydt64 = dtype == torch.float64 or prec == "f64"
    bn = b.numpy() if ydt64 else b.numpy().astype(np.float32).astype(np.float64)
    Zo, Gu, Yu = orc.multisketch(An, k, p, seed, b=bn, gemm_prec=prec)
    u_cs = 64 * EPS64 if dtype == torch.float64 else 1e-5
    u_mm = EPS64 if prec == "f64" else 2.0 ** -24
    parts = 3 if prec == "bf16x3" else 1
    absY = orc.bucket_abs_sums(An, k, seed, b=bn)
    bound = nblk * ((parts * k + 2) * u_mm * (np.abs(Gu) @ np.abs(Yu)) + np.abs(Gu) @ (u_cs * absY))
    assert np.all(np.abs(Zs - Zo) <= bound)
    Zw = msk.ms_sketch(Ad, k, p, seed, b=bd, gemm_prec=gp).cpu().numpy()
    assert np.all(np.abs(Zs - Zw) <= 2 * bound)
