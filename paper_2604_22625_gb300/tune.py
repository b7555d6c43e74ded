"""Autotuner of the batched solve's schedule (host side).

Two knobs decide how a batch runs: ``cta_work`` (asset-periods per CTA, which
sets every instance's cluster size and therefore the launch groups and their
tile widths) and ``check_every`` (iterations between the FP64 KKT / restart
checks).  ``tune()`` times each candidate on a stratified sample of the batch
(every k-th instance in work order, solved to the requested tolerance by the
GPU), keeps the fastest whose solves all converge, and caches the choice in a
JSON file keyed by a signature of the batch (instance-size histogram,
precision, tolerance, device name), so a later batch of the same shape reuses
it without timing.

The timing function is injectable, which lets the search and the cache be
tested without a GPU.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass
from typing import Callable, Dict, Iterable, List, Optional, Sequence

CTA_WORK = (4096.0, 8192.0, 16384.0)
CHECK_EVERY = (32, 64, 128)


@dataclass
class Choice:
    cta_work: float
    check_every: int
    seconds: float

    def options(self) -> dict:
        return {"cta_work": self.cta_work, "check_every": self.check_every}


def _bucket(x: float) -> int:
    """Power-of-two bucket of a size (for the signature)."""
    b = 0
    x = max(1.0, float(x))
    while x >= 2.0:
        x /= 2.0
        b += 1
    return b


def signature(problems: Sequence, precision: str, tol: float, device: str = "") -> str:
    """Key of a batch shape: histogram of (kind, log2 asset-periods, k + m)
    buckets, precision, tolerance and device name."""
    hist: Dict[str, int] = {}
    for p in problems:
        T = int(getattr(p, "T", 0))
        P = T - 1 if T >= 2 else 1
        key = f"{'m' if T >= 2 else 's'}{_bucket(p.F.shape[0] * P)}:{_bucket(p.F.shape[1] + p.A.shape[0])}"
        hist[key] = hist.get(key, 0) + 1
    blob = json.dumps({"h": sorted(hist.items()), "prec": precision, "tol": tol, "dev": device}, sort_keys=True)
    return hashlib.sha1(blob.encode()).hexdigest()[:16]


def sample(problems: Sequence, fraction: float = 0.125, min_count: int = 8) -> List:
    """Every k-th instance in decreasing work order (stratified over sizes)."""
    order = sorted(range(len(problems)),
                   key=lambda i: -problems[i].F.shape[0] * max(1, int(getattr(problems[i], "T", 0)) - 1))
    count = max(min(min_count, len(order)), int(round(fraction * len(order))))
    step = max(1, len(order) // count)
    return [problems[i] for i in order[::step][:count]]


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, data: dict) -> None:
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def default_cache_path() -> str:
    return os.path.join(os.path.expanduser("~"), ".cache", "flashfolio_gb300", "tune.json")


def tune(problems: Sequence, precision: str = "bf16", tol: float = 1e-6,
         timer: Optional[Callable[[Sequence, dict], Optional[float]]] = None,
         cache_path: Optional[str] = None, device: str = "",
         cta_work: Iterable[float] = CTA_WORK, check_every: Iterable[int] = CHECK_EVERY,
         fraction: float = 0.125) -> Choice:
    """Best (cta_work, check_every) for this batch shape, from the cache or by
    timing every candidate on a sample.  ``timer(sample, options)`` returns
    the seconds of one solve of the sample with those options, or None if an
    instance failed to converge (the candidate is then dropped)."""
    cache_path = cache_path or default_cache_path()
    sig = signature(problems, precision, tol, device)
    cache = _load(cache_path)
    if sig in cache:
        c = cache[sig]
        return Choice(float(c["cta_work"]), int(c["check_every"]), float(c["seconds"]))
    if timer is None:
        timer = gpu_timer(precision, tol)
    smp = sample(problems, fraction)
    best: Optional[Choice] = None
    for cw in cta_work:
        for ce in check_every:
            t = timer(smp, {"cta_work": float(cw), "check_every": int(ce)})
            if t is None:
                continue
            if best is None or t < best.seconds:
                best = Choice(float(cw), int(ce), float(t))
    if best is None:
        raise RuntimeError("no candidate schedule solved the sample")
    cache[sig] = {"cta_work": best.cta_work, "check_every": best.check_every, "seconds": best.seconds}
    _store(cache_path, cache)
    return best


def gpu_timer(precision: str, tol: float):
    """Timer that solves the sample on the current CUDA device (device time)."""
    import torch

    from . import api

    def run(smp: Sequence, opts: dict) -> Optional[float]:
        br = api.BatchRunner(smp, precision=precision, tol=tol, **opts)
        br.run()
        br.finish()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        br.run()
        br.finish()       # instances at the FP32 rounding floor are solved again in FP64, inside the time
        e1.record()
        torch.cuda.synchronize()
        if any(i["status"] != 0 for i in br.results()):
            return None
        return e0.elapsed_time(e1) / 1e3

    return run
