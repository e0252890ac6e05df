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

Segmented batches (tune_segmented) are tuned per class of segment count,
ceil(log2 nseg), on a batch the caller supplies: the packed-tile size
(tile_log2: 16K keys as 256 threads x 64, or 8K keys as 256 x 32), the
smallest size class a segment is padded to (tile_log2 - class_floor_gap, so
a tile holds at most 2^gap segments) and the persistent CTAs per SM; the
choice goes in with bitonic_set_segmented_options and into the same cache.
"""
from __future__ import annotations

import json
import os
import statistics

from . import (set_class_options, set_segmented_options, sort_, sort_pairs_, sort_segmented_,
               sort_segmented_pairs_)

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


SEG_CANDIDATES_KEYS = tuple(dict(tile_log2=t, class_floor_gap=g, ctas_per_sm=c)
                            for t in (14, 13) for g in (10, 8) for c in (2, 1))
SEG_CANDIDATES_PAIRS = tuple(dict(tile_log2=13, class_floor_gap=g, ctas_per_sm=c)
                             for g in (10, 8, 6) for c in (2, 1))


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


def _seg_class(nseg: int) -> int:
    c = 0
    while (1 << c) < nseg:
        c += 1
    return c


def tune_segmented(keys, offsets, pairs: bool = False, reps: int = 5, cache_path: str | None = None,
                   apply: bool = True) -> dict:
    """Times every packed-tile candidate on the batch (numpy uint32 keys and
    int32 offsets, nseg = offsets.size - 1), installs the fastest for the
    batch's class of segment count and merges it into the cache."""
    import numpy as np
    import torch
    nseg = int(offsets.size) - 1
    cls = _seg_class(nseg)
    src = torch.from_numpy(np.ascontiguousarray(keys).view(np.int32)).cuda()
    buf = src.clone()
    offs = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int32)).cuda()
    vals = torch.arange(src.numel(), dtype=torch.int32, device="cuda") if pairs else None
    vbuf = vals.clone() if pairs else None
    timed = []
    for cand in (SEG_CANDIDATES_PAIRS if pairs else SEG_CANDIDATES_KEYS):
        set_segmented_options(pairs, cls, cand)

        def run():
            buf.copy_(src)
            if pairs:
                vbuf.copy_(vals)
                sort_segmented_pairs_(buf, vbuf, offs)
            else:
                sort_segmented_(buf, offs)

        for _ in range(2):
            run()
        times = []
        for _ in range(reps):
            buf.copy_(src)
            if pairs:
                vbuf.copy_(vals)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            if pairs:
                sort_segmented_pairs_(buf, vbuf, offs)
            else:
                sort_segmented_(buf, offs)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        timed.append((statistics.median(times), cand))
    set_segmented_options(pairs, cls, None)
    best_ms, best = min(timed, key=lambda t: t[0])
    entry = dict(best, ms=best_ms, tried={json.dumps(c, sort_keys=True): m for m, c in timed})
    path = cache_path or default_cache_path()
    choices = {"gpu": _gpu_name(), "uint32": {}, "pairs": {}}
    if os.path.exists(path):
        with open(path) as f:
            old = json.load(f)
        if old.get("gpu") == choices["gpu"]:
            choices = old
    choices.setdefault("segmented_pairs" if pairs else "segmented_keys", {})[str(cls)] = entry
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(choices, f, indent=1)
    if apply:
        set_segmented_options(pairs, cls, best)
    return {"class_log2_nseg": cls, **entry}


def install(choices: dict) -> int:
    """Installs a tuning result's choices; returns how many classes were set."""
    count = 0
    for kind, pairs in (("segmented_keys", False), ("segmented_pairs", True)):
        for c, opt in choices.get(kind, {}).items():
            set_segmented_options(pairs, int(c), {f: opt[f] for f in ("tile_log2", "class_floor_gap",
                                                                      "ctas_per_sm") if f in opt})
            count += 1
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
