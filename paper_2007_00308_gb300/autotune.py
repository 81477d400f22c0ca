"""Autotuner for the launch parameters of a stroking step.

The tunables are the context's launch parameters (``ps_set_tuning``): ribs per
warp task in the rib kernel, links per thread in the link-setup kernel, and
CTAs per SM of the binning passes.  They change how the work is split over
threads, never what is computed, so any choice gives identical outputs.

``tune`` runs coordinate descent: for each tunable in turn it times every
candidate on the caller's own step (median of ``reps`` runs after a warm-up)
and keeps the fastest, and it repeats the sweep until nothing changes.  A
candidate is judged by the kernels its tunable changes (the context's
per-kernel CUDA events): a whole step is dominated by the coverage kernel,
whose run-to-run spread is larger than the differences being chosen between.
``tuned`` caches the choice in a JSON file keyed by device and workload
signature.  ``reserve_bins`` sizes the (quad, tile) bin reservation from the
entries a step actually produced.

The 16x16-pixel tile of the rasterizer is fixed: its per-path sample masks
(512 B each) are what fits 96 paths of a tile into each of the two coverage
CTAs an SM holds; a 32x32 tile would fit 24.
"""
from __future__ import annotations

import json
import math
import os
import statistics

from . import (PS_TUNE_BIN_BLOCKS, PS_TUNE_EMIT_SLABS, PS_TUNE_SETUP_LINKS, TUNE_CANDIDATES,
               TUNE_NAMES)

_KEY_OF = {v: k for k, v in TUNE_NAMES.items()}


def default_cache_path() -> str:
    return os.environ.get("PS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "polarstroke",
                                       "autotune.json"))


def signature(device: str, n_seg: int, n_path: int, n_rib: int, canvas=(0, 0)) -> str:
    """Workload key: sizes bucketed to powers of two, so nearby workloads share a choice."""
    def b(x):
        return 0 if x <= 0 else int(math.log2(x))
    return f"{device}|seg2^{b(n_seg)}|path2^{b(n_path)}|rib2^{b(n_rib)}|{canvas[0]}x{canvas[1]}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: dict) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(ctx, params: dict) -> None:
    for name, v in params.items():
        ctx.set_tuning(_KEY_OF[name], int(v))


def current(ctx) -> dict:
    return {TUNE_NAMES[k]: ctx.get_tuning(k) for k in TUNE_CANDIDATES}


# the kernels whose launch each tunable shapes (profiling slot names)
KERNELS_OF = {PS_TUNE_EMIT_SLABS: ("k_emit",), PS_TUNE_SETUP_LINKS: ("k_link_setup",),
              PS_TUNE_BIN_BLOCKS: ("k_bin_count", "k_bin_scatter")}


def _cuda_timer(ctx, step, flush):
    import torch

    def run():
        if flush is not None:
            flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        out = dict(ctx.profile_read())
        out["step"] = e0.elapsed_time(e1)
        return out
    return run


def _cost(sample, key=None) -> float:
    """Milliseconds that decide ``key``: its kernels' time when the sample has
    them, else the whole step."""
    if not isinstance(sample, dict):
        return float(sample)
    names = KERNELS_OF.get(key, ())
    if names and all(n in sample for n in names):
        return float(sum(sample[n] for n in names))
    return float(sample["step"])


def tune(ctx, step, *, reps: int = 5, rounds: int = 3, flush=None, timer=None) -> dict:
    """Coordinate descent over the tunables.  ``step()`` runs one step on the
    current stream; ``timer()`` returns one run's milliseconds, either a number
    or a dict of per-kernel times plus "step" (the default: CUDA events around
    ``step`` and the context's kernel events, with profiling switched on for
    the search and off after it).  Returns {"params", "ms", "default_ms",
    "trials"}, "ms" and "default_ms" being whole-step times."""
    own = timer is None
    if own:
        ctx.profile(True)
    run = timer if timer is not None else _cuda_timer(ctx, step, flush)

    def measure(key=None):
        run()  # warm-up with the new setting
        return statistics.median(_cost(run(), key) for _ in range(reps))

    try:
        start = current(ctx)
        default_ms = measure()
        trials = []
        for _ in range(rounds):
            changed = False
            for key, cands in TUNE_CANDIDATES.items():
                was = ctx.get_tuning(key)
                res = {}
                for v in cands:
                    ctx.set_tuning(key, v)
                    res[v] = measure(key)
                    trials.append({TUNE_NAMES[key]: v, "ms": res[v]})
                v_best = min(res, key=res.get)
                ctx.set_tuning(key, v_best)
                if v_best != was:
                    changed = True
            if not changed:
                break
        best_ms = measure()
    finally:
        if own:
            ctx.profile(False)
    return {"params": current(ctx), "ms": best_ms, "default_ms": default_ms, "start": start,
            "trials": trials}


def tuned(ctx, step, key: str, cache_path: str | None = None, **kw) -> dict:
    """The cached choice for ``key`` if there is one (applied to ``ctx``), else a
    fresh ``tune`` whose result is cached."""
    path = cache_path or default_cache_path()
    cache = load_cache(path)
    hit = cache.get(key)
    if isinstance(hit, dict) and isinstance(hit.get("params"), dict) and \
            set(hit["params"]) == set(_KEY_OF):
        apply(ctx, hit["params"])
        return dict(hit, cached=True)
    res = tune(ctx, step, **kw)
    entry = {"params": res["params"], "ms": res["ms"], "default_ms": res["default_ms"]}
    cache[key] = entry
    save_cache(path, cache)
    return dict(entry, cached=False)


def reserve_bins(ctx, n_tile: int, pairs: int, headroom: float = 1.05) -> int:
    """Reserve bin entries for a workload whose step produced ``pairs`` (quad,
    tile) entries (``ps_raster_stats``), with a little headroom."""
    n = int(math.ceil(pairs * headroom)) + 1024
    ctx.reserve(n_tile=n_tile, n_pair=n)
    return n
