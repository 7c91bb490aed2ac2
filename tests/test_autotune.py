"""Host logic of the autotuning cache (no GPU): batch signatures, the JSON
cache round trip, and applying a stored choice to the library's registry."""
import json

import pytest

KN = {"cs.fixed": 1, "cs.l2_budget_bytes": 33554432, "batch.kt_per": 8, "batch.round": 2,
      "pass.ctas_per_sm": 3}


def fake_report(values):
    return {"knobs": {k: {"chosen": v, "timed_on": "batch", "ms": {str(v): 1.0, "0": 2.0}}
                      for k, v in values.items()}, "reps": 3, "requests": 4}


@pytest.fixture
def reg():
    import paper_2508_14209_gb300 as msk
    from paper_2508_14209_gb300 import build

    build.build()
    msk.load()
    msk.tune_clear()
    yield msk
    msk.tune_clear()


def test_signature_is_order_free_and_separates_classes():
    from paper_2508_14209_gb300.autotune import signature

    a = signature([(20000, 16), (1 << 20, 128), (70000, 64)])
    b = signature([(70000, 64), (20000, 16), (1 << 20, 128)])
    assert a == b == "n16,64,128;d2^14-2^20;m3"
    assert signature([(20000, 16)]) != signature([(20000, 32)])
    with pytest.raises(ValueError):
        signature([])


def test_cache_round_trip_and_apply(reg, tmp_path):
    from paper_2508_14209_gb300 import autotune

    path = str(tmp_path / "tune.json")
    assert autotune.lookup(path, "dev", "sig") is None
    assert autotune.apply_cached(path, "dev", "sig") is False
    autotune.record(path, "dev", "sig", fake_report(KN))
    autotune.record(path, "dev", "other", fake_report(dict(KN, **{"batch.round": 8})))
    assert autotune.lookup(path, "dev", "sig") == KN
    assert json.load(open(path))["dev"]["other"]["chosen"]["batch.round"] == 8
    assert autotune.apply_cached(path, "dev", "sig") is True
    for name, v in KN.items():
        assert reg.tune_get(name, -1) == v


def test_apply_refuses_unknown_knobs(reg):
    from paper_2508_14209_gb300 import autotune

    with pytest.raises(KeyError):
        autotune.apply({"no.such.knob": 1})
    assert reg.tune_get("no.such.knob", -7) == -7
