"""Autotuning cache around the library's tuner (msk_autotune).

`tune(problems, cache)` times the registry knobs on a representative batch
(the C tuner does the timing and leaves the fastest values set), and records
the chosen values in a JSON cache keyed by the device and a signature of the
batch (the width classes present and the span of row counts).  `apply_cached`
sets a stored choice in the registry before serving, so that a process does
not re-tune what it has measured before.  Knobs change speed only, never
results beyond rounding order.
"""
from __future__ import annotations

import json
import math
import os

from . import load, msk_autotune, tune_set

KNOBS = ("cs.fixed", "cs.l2_budget_bytes", "batch.kt_per", "batch.round", "pass.ctas_per_sm")


def signature(shapes) -> str:
    """Key of a batch from its (d, n) shapes: the sorted width classes present,
    the floor/ceil of log2 of the row counts, and the batch size."""
    shapes = [(int(d), int(n)) for d, n in shapes]
    if not shapes:
        raise ValueError("empty batch")
    ns = sorted({n for _, n in shapes})
    lo = min(math.floor(math.log2(max(d, 1))) for d, _ in shapes)
    hi = max(math.ceil(math.log2(max(d, 1))) for d, _ in shapes)
    return f"n{','.join(map(str, ns))};d2^{lo}-2^{hi};m{len(shapes)}"


def device_key(device=0) -> str:
    import torch

    p = torch.cuda.get_device_properties(device)
    return f"{p.name};sm{p.major}{p.minor};{p.multi_processor_count}sm"


def chosen(report: dict) -> dict:
    """{knob: value} from a tuner report."""
    return {name: int(entry["chosen"]) for name, entry in report["knobs"].items()}


def apply(values: dict) -> None:
    """Set knob values in the registry (unknown names are refused)."""
    for name, value in values.items():
        if name not in KNOBS:
            raise KeyError(f"unknown knob {name!r}")
        tune_set(name, int(value))


def _read(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def record(path: str, device: str, sig: str, report: dict) -> None:
    """Store a tuner report's choice under (device, signature)."""
    table = _read(path)
    table.setdefault(device, {})[sig] = {"chosen": chosen(report), "report": report}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(path: str, device: str, sig: str):
    """Stored {knob: value} for (device, signature), or None."""
    entry = _read(path).get(device, {}).get(sig)
    return None if entry is None else dict(entry["chosen"])


def apply_cached(path: str, device: str, sig: str) -> bool:
    """Apply a stored choice; False when the cache has none for this key."""
    values = lookup(path, device, sig)
    if values is None:
        return False
    apply(values)
    return True


def tune(problems, cache: str | None = None, refine=True, tol=1e-6, max_iter=4, reps=3):
    """Run the tuner on [(A, b, seed), ...], leave its choice set, and record
    it in `cache` (if given).  Returns the tuner report."""
    load()
    report = msk_autotune(problems, refine=refine, tol=tol, max_iter=max_iter, reps=reps)
    if cache:
        dev = problems[0][0].device
        record(cache, device_key(dev), signature([tuple(A.shape) for A, _, _ in problems]), report)
    return report
