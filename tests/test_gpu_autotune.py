"""The autotuner (msk_autotune) on the GPU: it times every candidate of every
knob, leaves the fastest values set, the cache records them, and the batch
solved with the tuned schedule still reaches the oracle's least-squares
minimiser (knobs change speed, not results)."""
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu

SPECS = [(6000, 16, -3), (30011, 32, -6), (50000, 64, -8), (20000, 128, -4)]


@pytest.fixture(scope="module")
def msk():
    import paper_2508_14209_gb300 as m
    from paper_2508_14209_gb300 import build

    assert torch.cuda.is_available()
    build.build()
    m.load()
    m.tune_clear()
    yield m
    m.tune_clear()


def test_autotune_sets_fastest_and_keeps_results(msk, orc, tmp_path):
    from paper_2508_14209_gb300 import autotune

    probs, host = [], []
    for j, (d, n, ls) in enumerate(SPECS):
        A, b, _ = inputs.ls_problem(d, n, ls, seed=900 + j, dtype=torch.float32)
        Ad = msk.colmajor(d, n, torch.float32, "cuda")
        Ad.copy_(A)
        probs.append((Ad, b.cuda(), 0x5EED0005 + j))
        host.append((A.numpy(), b.numpy()))
    cache = str(tmp_path / "tune.json")
    rep = autotune.tune(probs, cache=cache, tol=1e-10, max_iter=6, reps=2)
    assert set(rep["knobs"]) == set(autotune.KNOBS)
    for name, e in rep["knobs"].items():
        ms = {int(k): v for k, v in e["ms"].items()}
        assert len(ms) >= 2 and all(v > 0 for v in ms.values())
        assert e["chosen"] == min(ms, key=ms.get)
        assert msk.tune_get(name, -1) == e["chosen"]
    sig = autotune.signature([tuple(A.shape) for A, _, _ in probs])
    assert autotune.lookup(cache, autotune.device_key(0), sig) == autotune.chosen(rep)
    xs, infos, rc = msk.msk_batch_lstsq(probs, refine=True, tol=1e-12, max_iter=10)
    assert rc == 0, infos
    for (An, bn), x in zip(host, xs):
        ro = orc.relres(An, bn, orc.lstsq_exact(An, bn))
        rb = orc.relres(An, bn, x.cpu().numpy())
        assert abs(rb - ro) <= 1e-8 * ro
