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
    assert msk.msk_cs_workspace(1000, 4, 64, msk.MSK_F64, msk.CS_ATOMIC) == 0
    assert msk.msk_cs_workspace(1000, 4, 64, msk.MSK_F64, msk.CS_SORTED) >= 1000 * 4
