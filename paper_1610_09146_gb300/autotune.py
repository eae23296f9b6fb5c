"""Autotuner for the batched path: per grid size and dtype, the algorithm family
(store-some or recompute-all) and the tile size (points per work item) that give
the shortest RK3 step on this GPU.

Each candidate is timed on a batch of identical instances of that grid (enough
copies to fill the GPU, at least ~8 M points or 4 instances), with CUDA events
around a few graph-replayed steps after a warm-up.  Results are cached as JSON
keyed by GPU name, dtype and grid, in $FDGB300_AUTOTUNE_CACHE or
~/.cache/fdgb300/autotune.json.
"""
from __future__ import annotations

import json
import os

FAMILIES = ("recompute_all", "store_some")
TILES = (256, 1024, 4096)


def cache_path() -> str:
    return os.environ.get("FDGB300_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fdgb300", "autotune.json"))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def key(gpu: str, dtype: str, n: int) -> str:
    return f"{gpu}|{dtype}|{n}"


def copies_for(n: int) -> int:
    """Identical instances used to time a grid: about 8 M points, at least 4."""
    return max(4, (8 << 20) // (n ** 3))


def time_candidate(n, dtype, family, tile, steps=4, warmup=2):
    import torch

    from . import Batch, dt_for_grid
    spec = dict(n=n, dt=dt_for_grid(n), algorithm=family, tile_points=tile)
    with Batch([spec] * copies_for(n), dtype=dtype) as b:
        b.step(warmup)
        st = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        b.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps


def tune(n: int, dtype: str, families=FAMILIES, tiles=TILES, refresh=False, path=None):
    """Best (family, tile_points, ms_per_step_per_copy) for an n^3 grid, from the cache
    unless refresh; otherwise timed now and stored."""
    import torch
    path = path or cache_path()
    gpu = torch.cuda.get_device_name()
    data = _load(path)
    k = key(gpu, dtype, n)
    if not refresh and k in data:
        e = data[k]
        return e["family"], e["tile_points"], e["ms_per_instance_step"]
    results = []
    for fam in families:
        for tile in tiles:
            ms = time_candidate(n, dtype, fam, tile)
            results.append((ms / copies_for(n), fam, tile))
    results.sort()
    best = results[0]
    data = _load(path)
    data[k] = {"family": best[1], "tile_points": best[2], "ms_per_instance_step": best[0],
               "candidates": [{"family": f, "tile_points": t, "ms_per_instance_step": m} for m, f, t in results]}
    _save(path, data)
    return best[1], best[2], best[0]


def choose(specs, dtype: str, refresh=False, path=None):
    """Copies of `specs` (dicts with at least n) with algorithm and tile_points set to the
    tuned choice for each distinct grid size."""
    sizes = sorted({s["n"] if isinstance(s["n"], int) else max(s["n"]) for s in specs})
    best = {n: tune(n, dtype, refresh=refresh, path=path) for n in sizes}
    out = []
    for s in specs:
        n = s["n"] if isinstance(s["n"], int) else max(s["n"])
        fam, tile, _ = best[n]
        out.append(dict(s, algorithm=fam, tile_points=tile))
    return out, best
