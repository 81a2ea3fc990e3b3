"""Autotuner for the batched GMM kernels.

The tunable shape is the backward work item: how many points one
(instance, component group) item covers (`chunk_points`, which also fixes how
many partial sums the finalize combines), and how many persistent CTAs share
an SM (`ctas_per_sm`, 0 = as many as fit). For a given set of instances the
tuner times every candidate pair with CUDA events (best of `reps` runs after a
warm-up) and keeps the fastest. Results are cached in a JSON file keyed by the
device name and a digest of the instance shapes, so the search runs once per
workload and device. Default cache: $GPA_TUNE_CACHE, else
~/.cache/gpa_autotune.json.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import _lib

CHUNKS = (1024, 2048, 4096, 8192, 16384)
CTAS = (0, 1)


def _cache_path(path=None):
    return path or os.environ.get("GPA_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                                      "gpa_autotune.json")


def signature(instances) -> str:
    shapes = [(int(i["x"].shape[0]), int(i["x"].shape[1]), int(i["alpha"].shape[0]), int(i.get("prec", 0)))
              for i in instances]
    h = hashlib.sha256(json.dumps(shapes).encode()).hexdigest()[:16]
    return f"{torch.cuda.get_device_name(instances[0]['x'].device)}|{len(shapes)}|{h}"


def _time(batch, ctas, reps):
    stream = torch.cuda.current_stream()
    batch.zero_grads()
    batch.run(ctas)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        batch.zero_grads()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run(ctas)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_batched(instances, chunks=CHUNKS, ctas=CTAS, reps=3, cache_path=None, refresh=False):
    """Return {"chunk_points", "ctas_per_sm", "ms", "table"} for these instances."""
    path = _cache_path(cache_path)
    key = signature(instances)
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache and not refresh:
        return cache[key]
    table = []
    for cp in chunks:
        batch = _lib.GmmBatch(instances, chunk_points=cp)
        batch.prepare()
        for c in ctas:
            table.append({"chunk_points": cp, "ctas_per_sm": c, "ms": _time(batch, c, reps)})
        del batch
        torch.cuda.empty_cache()
    best = min(table, key=lambda r: r["ms"])
    result = {"chunk_points": best["chunk_points"], "ctas_per_sm": best["ctas_per_sm"], "ms": best["ms"],
              "table": table}
    cache[key] = result
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    return result
