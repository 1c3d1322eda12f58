"""Autotuner for the batched qdot's one persistent launch.

The streaming kernel's launch shape (threads per CTA, CTAs per SM -- which
sets how many warps split the concatenated items of all pairs -- and
shared-memory staging on or off) is picked by timing every candidate on the
caller's own batch with CUDA events and keeping the fastest.  Results are
cached in a JSON file keyed by device, block size and the batch's shape, so a
batch of the same shape is tuned once.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import statistics

from . import _abi

# (threads per CTA, CTAs per SM, staged)
CANDIDATES = [(256, c, s) for c in (2, 3, 4) for s in (1, 0)] + [(128, c, s) for c in (4, 6, 8) for s in (1, 0)]


def cache_path() -> str:
    return os.environ.get("QDOT_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "qdot_gb300", "batched_tuning.json"))


def shape_key(device_name: str, block: int, ns) -> str:
    total = max(1, int(sum(ns)))
    longest = max([1] + [int(v) for v in ns])
    return f"{device_name}|B={block}|count={len(ns)}|total=2^{round(math.log2(total))}|max=2^{round(math.log2(longest))}"


def _load_cache(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, key, entry):
    data = _load_cache(path)
    data[key] = entry
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_batched(batch, reps: int = 5, use_cache: bool = True, path: str | None = None):
    """Pick the fastest launch shape for `batch` (a paper_2105_00115_gb300.Batch);
    sets batch.tuning and returns (tuning, {candidate: median ms})."""
    import torch
    path = path or cache_path()
    key = shape_key(torch.cuda.get_device_name(), batch.p.block, batch.ns_host)
    if use_cache:
        hit = _load_cache(path).get(key)
        if hit:
            batch.tuning = _abi.BatchedTuning(hit["threads_per_cta"], hit["ctas_per_sm"], 0, hit["staged"])
            return batch.tuning, hit.get("times_ms", {})
    stream = torch.cuda.current_stream()
    times = {}
    for threads, ctas, staged in CANDIDATES:
        batch.tuning = _abi.BatchedTuning(threads, ctas, 0, staged)
        batch.launch(stream=stream)  # warm-up (also sets the kernel attributes)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.launch(stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        times[f"{threads}x{ctas}{'s' if staged else 'r'}"] = statistics.median(ms)
    best = min(times, key=times.get)
    threads, rest = best.split("x")
    staged = 1 if rest.endswith("s") else 0
    ctas = int(rest[:-1])
    batch.tuning = _abi.BatchedTuning(int(threads), ctas, 0, staged)
    if use_cache:
        _store(path, key, {"threads_per_cta": int(threads), "ctas_per_sm": ctas, "staged": staged,
                           "times_ms": times})
    return batch.tuning, times
