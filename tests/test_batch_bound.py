"""The server admits requests by msk_batch_item_bound, an additive upper
bound of each item's part of msk_batch_workspace: over any batch the bounds
must add up to at least the batch's workspace, so that an admitted batch
always fits.  Host arithmetic only (no GPU)."""
import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def msk():
    import paper_2508_14209_gb300 as m
    from paper_2508_14209_gb300 import build

    build.build()
    m.load()
    return m


def _problem(d, n, pad):
    # untouched host buffers: only shapes, strides and addresses are read
    A = torch.empty((n, d + pad), dtype=torch.float32)[:, :d].t()
    b = torch.empty(d, dtype=torch.float64)
    return A, b, 1


@pytest.mark.parametrize("refine", [True, False])
def test_item_bounds_add_up_to_batch_workspace(msk, refine):
    rng = np.random.default_rng(5)
    for trial in range(40):
        m = int(rng.integers(1, 33))
        probs = [_problem(int(2 ** rng.uniform(14, 21)), int(rng.choice([16, 32, 64, 128, 256])),
                          int(rng.integers(0, 3))) for _ in range(m)]
        need = msk.msk_batch_workspace(probs, refine=refine)
        bound = sum(msk.msk_batch_item_bound(p, refine=refine) for p in probs)
        assert need > 0 and bound >= need, (trial, m, need, bound)
        # and not wildly above it (admission stays close to the real need)
        assert bound <= 1.25 * need + 8192 * m


def test_item_bound_rejects_unsupported_width(msk):
    A, b, s = _problem(4096, 20, 0)
    assert msk.msk_batch_item_bound((A, b, s)) == 0
