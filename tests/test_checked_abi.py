"""The checked build (MSK_CHECKED, relocatable device code) compiles, loads
without a GPU, exports every symbol the header declares and says it is
checked; the regular build says it is not."""
import ctypes

import pytest

from test_abi import declared_functions


@pytest.mark.parametrize("checked", [False, True])
def test_build_flavour_exports_and_identifies_itself(checked):
    from paper_2508_14209_gb300 import build

    L = ctypes.CDLL(build.build(checked=checked))
    for name in declared_functions():
        assert hasattr(L, name), name
    assert L.msk_checked_build() == (1 if checked else 0)
