"""Autotuner of the tensor-core GEMM configuration.

Times every configuration of the mixed-precision batched complex GEMM (pipeline depth and K-part
policy) on the block size and batch the sweeps use, picks the fastest, and caches the choice in
``_tune/tc_<gpu>_b<b>_n<batch>.json`` beside the package so later runs reuse it.
"""
from __future__ import annotations

import json
import os

import torch

from . import negf as _n

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune")


def _key(b, batch):
    name = torch.cuda.get_device_name().replace(" ", "_")
    return os.path.join(CACHE, f"tc_{name}_b{b}_n{batch}.json")


def load_cached(path: str):
    """The cached record at `path`, or None when there is none or it was written for another set
    of configurations (a library with a different configuration count)."""
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if not isinstance(rec, dict):
        return None
    n = _n.tc_config_count()
    c = rec.get("config")
    if rec.get("n_configs") != n or not isinstance(c, int) or not 0 <= c < n:
        return None
    return rec


def tune_tc(b: int, batch: int, reps: int = 3, use_cache: bool = True) -> dict:
    """Select and return the best configuration for b x b x b products in batches of `batch`."""
    path = _key(b, batch)
    rec = load_cached(path) if use_cache else None
    if rec is not None:
        _n.tc_config(rec["config"])
        return rec
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn((batch, b, b), dtype=torch.complex128, device="cuda", generator=g)
    B = torch.randn((batch, b, b), dtype=torch.complex128, device="cuda", generator=g)
    C = torch.empty_like(A)
    times = {}
    for c in range(_n.tc_config_count()):
        _n.tc_config(c)
        _n.zgemm(A, B, C, precision=_n.PREC_MIXED)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            _n.zgemm(A, B, C, precision=_n.PREC_MIXED)
        e1.record()
        torch.cuda.synchronize()
        times[c] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    _n.tc_config(best)
    rec = {"b": b, "batch": batch, "config": best, "n_configs": _n.tc_config_count(), "ms": times}
    os.makedirs(CACHE, exist_ok=True)
    with open(path, "w") as fh:
        json.dump(rec, fh)
    return rec
