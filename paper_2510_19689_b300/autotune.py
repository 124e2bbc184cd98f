"""Autotuner for the tensor-core kernels' launch shape.

The search space is the one tabnet_set_tile_config exposes: epilogue
warpgroups per 128-row tile, depth of the weight-staging ring, and tiles
resident per SM.  Every candidate the library accepts is timed with CUDA
events on the caller's stream (median of a few launches after warm-up) and
the fastest one is applied and cached as JSON keyed by GPU name, model
content hash, precision and a power-of-two bucket of the row count.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional

import torch

from . import tabnet

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "tabnet_b300", "autotune.json")


def _bucket(rows: int) -> int:
    b = 1
    while b < rows:
        b *= 2
    return b


def cache_key(model: "tabnet.Model", rows: int) -> str:
    name = torch.cuda.get_device_name(model.device)
    return f"{name}|{model.dims.content_hash:016x}|p{model.precision}|r{_bucket(rows)}"


def candidates(model: "tabnet.Model"):
    n = model.dims.n_d + model.dims.n_a
    nwgs = [2] if n == 128 else ([1] if n == 16 else [1, 2])
    for nwg in nwgs:
        for cps in (1, 2, 3, 4):
            for slots in (1, 2, 3, 4, 6, 8):
                yield dict(nwg=nwg, n_slots=slots, ctas_per_sm=cps)


def _time(model, args, stream, reps: int, warmup: int) -> float:
    for _ in range(warmup):
        model.forward(*args, stream=stream)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        model.forward(*args, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


def tune(model: "tabnet.Model", x_num, x_cat, rows: int, logits, masks=None, agg=None,
         stream: Optional[torch.cuda.Stream] = None, reps: int = 5, warmup: int = 2,
         cache_path: Optional[str] = DEFAULT_CACHE, use_cache: bool = True) -> Dict:
    """Pick and apply the fastest launch shape for this model and batch size.

    Returns {"config": {...}, "ms": best, "tried": [(config, ms), ...]}."""
    stream = stream or torch.cuda.current_stream(model.device)
    key = cache_key(model, rows)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        cfg = cache[key]["config"]
        try:
            model.set_tile_config(**cfg)
            return dict(cache[key], cached=True)
        except tabnet.TabnetError:
            pass
    args = (x_num, x_cat, rows, logits, masks, agg)
    tried = []
    seen = set()
    for cand in candidates(model):
        try:
            model.set_tile_config(**cand)
        except tabnet.TabnetError:
            continue
        actual = model.tile_config()
        sig = tuple(sorted(actual.items()))
        if sig in seen:
            continue
        seen.add(sig)
        tried.append((actual, _time(model, args, stream, reps, warmup)))
    if not tried:
        raise RuntimeError("no launch shape accepted")
    best_cfg, best_ms = min(tried, key=lambda t: t[1])
    model.set_tile_config(**best_cfg)
    entry = {"config": best_cfg, "ms": best_ms, "tried": tried}
    if cache_path:
        cache[key] = {"config": best_cfg, "ms": best_ms}
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return entry
