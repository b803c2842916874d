"""Autotuner of the batched fragment kernel (ms_batch_run).

The knobs are the kernel's launch shape and pipeline: warps per CTA (block size),
chunks in flight per warp (the software-pipeline unroll), chunks per tile (the
unit of work a warp or CTA packs into one scheduling step), CTAs per SM, the
decoder variant (width-specialised code, or one compact loop with a smaller
instruction footprint) and the schedule (tiles to warps from a work counter, or
round-robin to CTAs so that the warps of one SM decode few distinct widths).

``tune`` times every candidate on the caller's batch with CUDA events and
returns the fastest.  Results are cached per device and batch signature in a
JSON file (``MS_AUTOTUNE_CACHE``, default ``~/.cache/morphstore_gb300/autotune.json``).
All candidates give the same bits: the choice changes time only.
"""
from __future__ import annotations

import itertools
import json
import math
import os

import torch

from . import morphstore as ms

TILES = (16, 64, 256)
CTAS_PER_SM = (0,)


def candidates(variants=None, tiles=TILES, ctas=CTAS_PER_SM):
    """Every built (warps, depth, compact, schedule) variant with every tile size and
    CTA cap that the variant accepts, as ms_batch_config tuples: the work-counter
    schedule (0) needs tiles of at least two pipeline depths, the per-CTA schedule (1)
    at least one chunk per warp, the CTA-streamed schedule (2) takes any tile."""
    out = []
    for (w, d, c, s), t, k in itertools.product(variants or ms.BATCH_VARIANTS, tiles, ctas):
        if (s == 0 and t >= 2 * d) or (s == 1 and t >= w) or s == 2:
            out.append((w, d, t, k, c, s))
    return out


def cache_path() -> str:
    return os.environ.get("MS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "morphstore_gb300", "autotune.json"))


def signature(batch: "ms.Batch", device) -> str:
    """Device name and SM count, fragment count, and the batch's size on a log2 grid."""
    p = torch.cuda.get_device_properties(device)
    info = batch.info()
    rows = max(info["rows"], 1)
    return "%s/%dsm/f%d/r2^%d/b%.1f" % (p.name, p.multi_processor_count, batch.n, round(math.log2(rows)),
                                          8.0 * info["bytes"] / rows)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def time_config(batch, sums, cfg, reps=3, stream=None) -> float:
    """Median milliseconds of one run of `cfg` (after one untimed run)."""
    stream = stream or torch.cuda.current_stream()
    batch.run(sums, cfg=cfg, stream=stream)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run(sums, cfg=cfg, stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return sorted(times)[len(times) // 2]


def tune(batch, sums, cands=None, reps=3, use_cache=True, stream=None):
    """Fastest configuration for `batch`: (config tuple, {config: ms}).  A cached
    entry for the same signature is returned without timing when use_cache."""
    path = cache_path()
    key = signature(batch, sums.device)
    if use_cache:
        hit = _load(path).get(key)
        if hit:
            return tuple(hit["cfg"]), {tuple(hit["cfg"]): hit["ms"]}
    table = {}
    for cfg in cands or candidates():
        try:
            table[tuple(cfg)] = time_config(batch, sums, cfg, reps=reps, stream=stream)
        except ms.MSError as e:
            if e.code != ms.MS_ERR_INVALID_ARG:  # a variant whose shared memory does not fit is skipped
                raise
    best = min(table, key=table.get)
    if use_cache:
        data = _load(path)
        data[key] = {"cfg": list(best), "ms": table[best]}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
        except OSError:
            pass
    return best, table
