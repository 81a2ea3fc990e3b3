"""Autotuner for the batched GMM kernels, per padded-dimension class.

The batched form runs each class (padded dimension 8, 16, 32, 64, 128) in
kernels of its own, one class after another, so each class is tuned on its
own instances alone. Its settings (gpa_batched_opts in include/gpa.h):

* chunk_points: how many points one backward work item covers (which also
  fixes how many partial sums the finalize combines);
* ctas_per_sm: persistent CTAs per SM of the class's forward and backward
  kernels (0 = as many as fit);
* small_groups (D <= 16 and D <= 32 only): whether instances with few
  components take their backward items in the small component group (10 and 6
  components per CTA instead of 42 and 25), where that leaves fewer threads
  idle.

For each class the tuner times every candidate with CUDA events (best of
`reps` runs after a warm-up) and keeps the fastest; a class of tensor-core
instances only (its stages one launch each over all its instances) has only
its backward chunk size to tune. Results are cached in a JSON file keyed by the device name and a
digest of the instance shapes, so the search runs once per workload and
device. Default cache: $GPA_TUNE_CACHE, else ~/.cache/gpa_autotune.json.
"""
from __future__ import annotations

import hashlib
import json
import os

import torch

from . import _lib

CHUNKS = (1024, 2048, 4096, 8192, 16384, 65536)
CTAS = (0, 1)
SMALL_CLASSES = (1, 2)  # D <= 16, D <= 32


def _cache_path(path=None):
    return path or os.environ.get("GPA_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                                      "gpa_autotune.json")


def signature(instances) -> str:
    shapes = [(int(i["x"].shape[0]), int(i["x"].shape[1]), int(i["alpha"].shape[0]), int(i.get("prec", 0)))
              for i in instances]
    h = hashlib.sha256(json.dumps(shapes).encode()).hexdigest()[:16]
    return f"per-class|{torch.cuda.get_device_name(instances[0]['x'].device)}|{len(shapes)}|{h}"


def class_of(inst) -> int:
    return _lib.batch_class(int(inst["x"].shape[1]), int(inst.get("prec", 0)))


def _time(batch, reps):
    stream = torch.cuda.current_stream()
    batch.zero_grads()
    batch.run()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        batch.zero_grads()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run()
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def _tune_class(c, sub, chunks, ctas, reps, small=True):
    table = []
    smalls = (0, 1) if small and c in SMALL_CLASSES else (0,)
    for cp in chunks:
        for sg in smalls:
            for ct in ctas:
                setting = {"chunk_points": cp, "ctas_per_sm": ct, "small_groups": sg}
                batch = _lib.GmmBatch(sub, opts={c: setting})
                batch.prepare()
                table.append(dict(setting, ms=_time(batch, reps)))
                del batch
        torch.cuda.empty_cache()
    best = min(table, key=lambda r: r["ms"])
    return {k: best[k] for k in ("chunk_points", "ctas_per_sm", "small_groups")}, best["ms"], table


def tune_batched(instances, chunks=CHUNKS, ctas=CTAS, reps=3, cache_path=None, refresh=False):
    """Return {"opts": {class: settings}, "classes": {class: {"n", "ms", "table"}}}
    for these instances; "opts" goes to GmmBatch(..., opts=...)."""
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
        return _normalize(cache[key])
    opts, classes = {}, {}
    for c in range(_lib.BATCH_CLASSES):
        sub = [i for i in instances if class_of(i) == c]
        if not sub:
            continue
        fp32 = any(int(i.get("prec", 0)) == _lib.PREC_FP32 for i in sub)
        # a class of tensor-core instances only has its backward chunk size to tune
        opts[c], ms, table = _tune_class(c, sub, chunks, ctas if fp32 else (0,), reps, small=fp32)
        classes[c] = {"n": len(sub), "ms": ms, "table": table}
    result = {"opts": opts, "classes": classes}
    cache[key] = result
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    return _normalize(json.loads(json.dumps(result)))


def _normalize(r):
    """Class keys back to int after a JSON round trip."""
    return {"opts": {int(c): v for c, v in r["opts"].items()},
            "classes": {int(c): v for c, v in r["classes"].items()}}
