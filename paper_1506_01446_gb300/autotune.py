"""Autotuner: per size class, measure candidate tile configurations and keep
the fastest.

A candidate is a tile size (tile_log2), keys held per thread in registers
(keys_per_thread_log2), the fused-stride cutoff (global_bits: the most
strides at or above the tile size one pass may take; 0 = automatic, 8), the
L2 prefetch distance (l2_prefetch, in resident waves) and the register cap
(ctas_per_sm: 3 = kernels capped for three resident CTAs per SM, 2 = kernels
bounded for two, the default).
For every size class 2^k the tuner times each candidate with CUDA events on
data already in device memory, picks the fastest, installs it with
bitonic_set_class_options and caches the choices as JSON per GPU name (path:
$BITONIC_TUNE_CACHE, else ~/.cache/bitonic_gb300/tune.json).  load() installs
a cached set without measuring.
"""
from __future__ import annotations

import json
import os
import statistics

from . import set_class_options, sort_, sort_pairs_

CANDIDATES_U32 = (
    dict(tile_log2=14, keys_per_thread_log2=6, global_bits=8, l2_prefetch=1, ctas_per_sm=3),
    dict(tile_log2=14, keys_per_thread_log2=6, global_bits=0, l2_prefetch=1, ctas_per_sm=3),
    dict(tile_log2=14, keys_per_thread_log2=6, global_bits=8, l2_prefetch=1, ctas_per_sm=2),
    dict(tile_log2=14, keys_per_thread_log2=6, global_bits=0, l2_prefetch=1, ctas_per_sm=2),
    dict(tile_log2=14, keys_per_thread_log2=6, global_bits=8, l2_prefetch=0, ctas_per_sm=3),
    dict(tile_log2=13, keys_per_thread_log2=5, global_bits=0, l2_prefetch=1, ctas_per_sm=2),
)
CANDIDATES_PAIRS = (
    dict(tile_log2=13, keys_per_thread_log2=5, global_bits=0, l2_prefetch=1, ctas_per_sm=3),
    dict(tile_log2=13, keys_per_thread_log2=5, global_bits=0, l2_prefetch=1, ctas_per_sm=2),
    dict(tile_log2=13, keys_per_thread_log2=5, global_bits=7, l2_prefetch=1, ctas_per_sm=3),
    dict(tile_log2=12, keys_per_thread_log2=4, global_bits=0, l2_prefetch=1, ctas_per_sm=2),
)


def default_cache_path() -> str:
    return os.environ.get("BITONIC_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "bitonic_gb300", "tune.json")


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _time_candidate(kind, k, cand, reps):
    import torch
    n = 1 << k
    gen = torch.Generator(device="cuda").manual_seed(k)
    src = torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, device="cuda", generator=gen)
    buf = src.clone()
    vals = torch.arange(n, dtype=torch.int32, device="cuda") if kind == "pairs" else None
    set_class_options(8 if kind == "pairs" else 4, k, cand)

    def run():
        if kind == "pairs":
            sort_pairs_(buf, vals)
        else:
            sort_(buf)

    for _ in range(2):
        buf.copy_(src)
        run()
    times = []
    for _ in range(reps):
        buf.copy_(src)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def tune(classes=tuple(range(16, 29, 2)), pair_classes=tuple(range(16, 27, 2)), reps: int = 5,
         cache_path: str | None = None, apply: bool = True) -> dict:
    """Measures every candidate for each size class; returns and caches the choices."""
    result = {"gpu": _gpu_name(), "uint32": {}, "pairs": {}}
    for kind, ks, cands in (("uint32", classes, CANDIDATES_U32), ("pairs", pair_classes, CANDIDATES_PAIRS)):
        kb = 8 if kind == "pairs" else 4
        for k in ks:
            timed = []
            for cand in cands:
                try:
                    ms = _time_candidate(kind, k, cand, reps)
                except RuntimeError:
                    continue  # the planner rejects this choice for the class
                timed.append((ms, cand))
            set_class_options(kb, k, None)
            if not timed:
                continue
            best_ms, best = min(timed, key=lambda t: t[0])
            result[kind][str(k)] = dict(best, ms=best_ms,
                                        tried={json.dumps(c, sort_keys=True): m for m, c in timed})
    path = cache_path or default_cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(result, f, indent=1)
    if apply:
        install(result)
    return result


def install(choices: dict) -> int:
    """Installs a tuning result's choices; returns how many classes were set."""
    count = 0
    for kind, kb in (("uint32", 4), ("pairs", 8)):
        for k, c in choices.get(kind, {}).items():
            opts = {f: c[f] for f in ("tile_log2", "keys_per_thread_log2", "global_bits", "l2_prefetch",
                                      "min_row_log2", "ctas_per_sm") if f in c}
            set_class_options(kb, int(k), opts)
            count += 1
    return count


def load(cache_path: str | None = None, gpu_name: str | None = None) -> dict | None:
    """Installs the cached choices for this GPU, if any; returns them."""
    path = cache_path or default_cache_path()
    if not os.path.exists(path):
        return None
    with open(path) as f:
        choices = json.load(f)
    name = gpu_name if gpu_name is not None else _gpu_name()
    if choices.get("gpu") != name:
        return None
    install(choices)
    return choices
