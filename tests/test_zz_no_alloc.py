"""msk_gemm_noalloc — the Gaussian-stage GEMM for callers that may not allocate
device memory (its scratch is a fixed array inside the library) — must give
what msk_gemm gives with a caller workspace.  Collected last on purpose; it
passes on its own in a fresh process and after the other tests."""
import numpy as np
import pytest
import torch

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


def _oracle_bound(orc, seed, p, Y, prec):
    """The oracle's Z = G Y on the inputs rounded to the stage's precision
    (Gaussian and Y as the multisketch rounds them) and the rounding bound of
    that stage's accumulation, the bound every Gaussian-stage parity test of
    this suite uses."""
    Yh = Y.double().cpu().numpy()
    G = orc.gaussian(seed, p, Y.shape[0])
    k = Y.shape[0]
    if prec in ("f64", "f32"):
        Gu, Yu = G.astype(np.float64), Yh
    elif prec == "bf16":
        Gu, Yu = orc.round_bf16(G).astype(np.float64), orc.round_bf16(Yh.astype(np.float32)).astype(np.float64)
    elif prec == "f16":
        Gu, Yu = orc.round_fp16(G).astype(np.float64), orc.round_fp16(Yh.astype(np.float32)).astype(np.float64)
    else:
        Gu, Yu = orc.round_bf16(G).astype(np.float64), orc.split_bf16x3(Yh.astype(np.float32))
    u = EPS64 if prec == "f64" else 2.0 ** -24
    terms = 3 * k + 2 if prec == "bf16x3" else k + 2
    return orc.gemm(Gu, Yu), terms * u * (np.abs(Gu) @ np.abs(Yu))


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16", "f16", "bf16x3"])
def test_noalloc_matches_workspace_entry_point(msk, orc, prec):
    """Two calls in a row, each bit for bit what msk_gemm gives with a caller
    workspace (the same kernels and the same fixed reduction order), and
    within the stage's rounding bound of the oracle."""
    gp = msk.GEMM_PRECS[prec]
    dt = torch.float64 if prec == "f64" else torch.float32
    p, k, ncol = 256, 8192, 65
    gen = torch.Generator().manual_seed(7)
    for call, seed in enumerate((0x5EED0004, 0x5EED0005)):
        Y = torch.randn(k, ncol, generator=gen, dtype=torch.float64).to(dt).cuda()
        Zref = msk.msk_gemm(seed, p, Y, gemm_prec=gp).cpu().numpy()
        Z = msk.msk_gemm_noalloc(seed, p, Y, gemm_prec=gp).cpu().numpy()
        assert np.array_equal(Z, Zref), f"call {call}"
        Zo, bound = _oracle_bound(orc, seed, p, Y, prec)
        assert np.all(np.abs(Z - Zo) <= bound), f"call {call}"


def test_noalloc_does_not_grow_device_memory(msk):
    Y = torch.randn(4096, 33, dtype=torch.float64, device="cuda")
    msk.msk_gemm_noalloc(3, 128, Y)  # first call on the device: address set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for s in range(3):
        msk.msk_gemm_noalloc(4 + s, 128, Y)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_oversized_problem(msk):
    # 512 x 32768 binary32 G alone is 64 MiB, beyond the fixed array
    Y = torch.zeros(32768, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(msk.MskError) as ei:
        msk.msk_gemm_noalloc(1, 512, Y)
    assert ei.value.code == msk.MSK_ENOMEM
    assert "scratch" in str(ei.value)
