"""Autotuner of the size-bin launch shapes (rsai_set_tuning).

For a built handle it times graph-replayed rebuilds under each candidate
shape (warps per CTA of the warp bins, the largest |J| given to the
register-resident QR, and whether columns start in the half-warp bin), keeps
the fastest and caches it in a
JSON file keyed by GPU name, precision and a coarse signature of the problem
(n and nnz/n rounded to powers of two), so later builds of similar problems
start from the cached shape.  The CTA shapes leave results bit-identical;
the register-QR threshold changes only the rounding of the LS solutions.
"""
from __future__ import annotations

import json
import math
import os

from . import rsai

DEFAULT_CANDIDATES = [
    dict(warp_bin_warps=w, warp_bin_ctas_per_sm=0, small_qr_max_p=sp, global_bin_ctas=0, half_bin=hb)
    for hb in (0, 1) for w in (2, 4, 8) for sp in (0, 8, 16)
]


def cache_path() -> str:
    return os.environ.get("RSAI_TUNING_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "rsai_gb300",
                                                            "tuning.json"))


def signature(n: int, nnz: int, precision: str) -> str:
    import torch

    gpu = torch.cuda.get_device_name(torch.cuda.current_device()).replace(" ", "_")
    return f"{gpu}|{precision}|n2^{round(math.log2(max(n, 1)))}|d2^{round(math.log2(max(nnz / max(n, 1), 1)))}"


def _time_rebuild(handle, steps: int) -> float:
    import torch

    handle.rebuild()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        handle.rebuild()
        e1.record(st)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return sorted(ms)[len(ms) // 2]


def tune(handle: "rsai.Handle", nnz: int, precision: str, candidates=None, steps: int = 3, path: str | None = None,
         use_cache: bool = True) -> dict:
    """Pick the fastest launch shape for ``handle``; returns {"tuning", "ms", "trials", "cached"}."""
    path = path or cache_path()
    key = signature(handle.n, nnz, precision)
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        handle.set_tuning(**cache[key]["tuning"])
        return {**cache[key], "cached": True}
    trials = []
    for cand in candidates or DEFAULT_CANDIDATES:
        try:
            handle.set_tuning(**cand)
        except rsai.RSAIError:
            continue  # not resident on this GPU
        trials.append({"tuning": cand, "ms": _time_rebuild(handle, steps)})
    best = min(trials, key=lambda t: t["ms"])
    handle.set_tuning(**best["tuning"])
    entry = {"tuning": best["tuning"], "ms": best["ms"], "trials": trials}
    cache[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    return {**entry, "cached": False}
