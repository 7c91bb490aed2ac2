"""The C-ABI library loads and exports every symbol include/msketch.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_14209_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "msketch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:[a-z_0-9]+\s+)*[a-z_0-9]+[\s*]+([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_parses():
    names = declared_functions()
    assert "cs_sketch" in names and "ms_lstsq" in names and "ne_lstsq" in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    import paper_2508_14209_gb300 as msk

    assert sorted(msk.EXPORTS) == declared_functions()


def test_version_and_workspace_queries(lib):
    import paper_2508_14209_gb300 as msk

    assert "sm_103a" in msk.version()
    # pure host-side size queries
    # FP64 atomic: replicas of Y while the sketch has few 128-byte lines
    # (16 x 64 rows x 5 columns at k = 64), none at k = 8192, n = 64
    assert msk.msk_cs_workspace(1000, 4, 64, msk.MSK_F64, msk.CS_ATOMIC) == 16 * 64 * 5 * 8
    assert msk.msk_cs_workspace(1000, 64, 8192, msk.MSK_F64, msk.CS_ATOMIC) == 0
    assert msk.msk_cs_workspace(1000, 4, 64, msk.MSK_F32, msk.CS_ATOMIC) == 0
    assert msk.msk_cs_workspace(1000, 4, 64, msk.MSK_F64, msk.CS_SORTED) >= 1000 * 4


def test_argument_checks_return_before_any_device_work(lib):
    """Invalid arguments are refused with the documented negative codes
    before any pointer is touched (the pointers below are never
    dereferenced)."""
    import paper_2508_14209_gb300 as msk

    L = msk.load()
    fake = ctypes.c_void_p(16)
    # srht_sketch: d must be a power of two (-3); k >= 1 (-7)
    assert L.srht_sketch(fake, msk.MSK_F64, 1000, 4, 1000, None, 10, 1, fake, 4, None, 0, None) == -3
    assert L.srht_sketch(fake, msk.MSK_F64, 1024, 4, 1024, None, 0, 1, fake, 4, None, 0, None) == -7
    # sns_lstsq: unknown sketch kind (-7); GAUSS needs n+1 <= p (-9)
    assert L.sns_lstsq(fake, msk.MSK_F64, 100, 4, 100, fake, 9, 50, 8, 1, fake, None, None, 0, None) == -7
    assert L.sns_lstsq(fake, msk.MSK_F64, 100, 4, 100, fake, msk.SKETCH_GAUSS, 0, 4, 1, fake, None, None,
                       0, None) == -9
    # rcq_lstsq / rcq_qr: n <= 400 (-4), p >= n + 1 (-8)
    assert L.rcq_lstsq(fake, msk.MSK_F64, 10000, 401, 10000, fake, 400000, 1604, 1, msk.GEMM_F64, fake,
                       None, None, 0, None) == -4
    assert L.rcq_qr(fake, msk.MSK_F64, 10000, 20, 10000, 800, 20, 1, msk.GEMM_F64, fake, 10000, fake, 20,
                    None, 0, None) == -8
    # msk_householder_qr: c <= 512 (-3)
    assert L.msk_householder_qr(fake, 1000, 513, 1000, None) == -3
    # workspace queries are pure host arithmetic
    assert msk.msk_srht_workspace(1 << 20, 7, True, 4096) >= (1 << 20) * 8 * 8
    assert msk.msk_srht_workspace(1000, 7, True, 4096) == 0  # not a power of two


def test_gemm_wrappers_refuse_operands_the_c_side_cannot_check():
    """msk_gemm and msk_gemm_noalloc take Y and Z through void pointers whose
    element type follows gemm_prec: the binding refuses a Y of the wrong
    dtype (a float32 Y read as float64 would overrun it), a column-strided Y,
    a Z of the wrong dtype, shape or layout, and host tensors — all before
    any call into the library."""
    import torch

    import paper_2508_14209_gb300 as msk

    k, ncol, p = 64, 5, 8
    y64 = torch.zeros((k, ncol), dtype=torch.float64)
    y32 = torch.zeros((k, ncol), dtype=torch.float32)
    for fn in (msk.msk_gemm, msk.msk_gemm_noalloc):
        with pytest.raises(ValueError, match="float64"):
            fn(1, p, y32, gemm_prec=msk.GEMM_F64)
        for prec in (msk.GEMM_F32, msk.GEMM_BF16, msk.GEMM_F16, msk.GEMM_BF16X3):
            with pytest.raises(ValueError, match="float32"):
                fn(1, p, y64, gemm_prec=prec)
        with pytest.raises(ValueError, match="row-major"):
            fn(1, p, torch.zeros((k, 2 * ncol), dtype=torch.float64)[:, ::2], gemm_prec=msk.GEMM_F64)
        with pytest.raises(ValueError, match="2-D"):
            fn(1, p, torch.zeros(k, dtype=torch.float64), gemm_prec=msk.GEMM_F64)
        with pytest.raises(ValueError, match="Z must be float64"):
            fn(1, p, y64, gemm_prec=msk.GEMM_F64, Z=torch.zeros((p, ncol), dtype=torch.float32))
        with pytest.raises(ValueError, match="Z must be float64"):
            fn(1, p, y64, gemm_prec=msk.GEMM_F64, Z=torch.zeros((p + 1, ncol), dtype=torch.float64))
        with pytest.raises(ValueError, match="column-major"):
            fn(1, p, y64, gemm_prec=msk.GEMM_F64, Z=torch.zeros((p, ncol), dtype=torch.float64))
        with pytest.raises(ValueError, match="CUDA"):
            fn(1, p, y64, gemm_prec=msk.GEMM_F64, Z=msk.colmajor(p, ncol, torch.float64, "cpu"))
        with pytest.raises(ValueError, match="unknown gemm_prec"):
            fn(1, p, y64, gemm_prec=9)
