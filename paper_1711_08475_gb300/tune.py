"""Cached tile shapes from the autotuner.

The cache is a JSON file (default: ~/.cache/fpmatch/autotune.json, or
$FPMATCH_TUNE_CACHE) keyed by GPU model and SM count, library version,
fingerprint type, width, q-gram length and combined types, k, metric, form, the
dictionary size rounded to a power of two and the length mix of the pattern sample (its shares of seven
length classes, in tenths).  A miss runs fp_autotune on the given pattern
sample.  tuned_plan_opts does the same for batched plans whose batches mix
several (k, metric) pairs: it times every tile on a plan over the sample.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import Plan, _strings, fp_autotune, fp_version

LENGTH_CLASSES = (0, 4, 8, 16, 32, 64, 128, 256)


def length_mix(offsets) -> str:
    """Shares of the patterns in the length classes 0-3, 4-7, ..., 128-255 (tenths)."""
    lens = np.diff(np.asarray(offsets, dtype=np.int64))
    if lens.size == 0:
        return "empty"
    h, _ = np.histogram(lens, bins=LENGTH_CLASSES)
    return "".join(str(int(round(10 * c / lens.size))) for c in h)


def cache_path() -> str:
    return os.environ.get("FPMATCH_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fpmatch", "autotune.json"))


def _key(index, k, metric, mode, offsets) -> str:
    import torch
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    info = index.info()
    words = max(1, int(info["n_words"]))
    size = 1 << (words - 1).bit_length()
    return "|".join(str(x) for x in (props.name, props.multi_processor_count, fp_version(), info["type"],
                                     info["width_bits"], info.get("qgram", 1), info.get("combined", 0), k, metric,
                                     mode, size,
                                     length_mix(offsets)))


def _load():
    path = cache_path()
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            pass
    return {}


def _store(cache):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _host_offsets(offsets):
    try:
        import torch
        if isinstance(offsets, torch.Tensor):
            return offsets.cpu().numpy()
    except ImportError:
        pass
    return np.asarray(offsets)


def tuned_opts(index, sample_chars, sample_offsets=None, k: int = 1, metric: str = "ham", mode: str = "tiled",
               reps: int = 2, refresh: bool = False) -> dict:
    """{"tile_queries", "words_per_thread", "variant"} for this GPU and workload."""
    chars, offsets, _ = _strings(sample_chars, sample_offsets)
    key = _key(index, k, metric, mode, _host_offsets(offsets))
    cache = _load()
    if not refresh and key in cache:
        return cache[key]
    best, _ = fp_autotune(index, chars, offsets, k, metric, mode, reps)
    opts = {"tile_queries": best["tile_queries"], "words_per_thread": best["words_per_thread"],
            "variant": best["variant"], "ms": best["ms"]}
    cache[key] = opts
    _store(cache)
    return opts


PLAN_TILES = (32, 64, 128, 256)


def tuned_plan_opts(index, sample_chars, sample_offsets=None, batches=(), reps: int = 2,
                    refresh: bool = False) -> dict:
    """{"tile_queries", "variant", "ms", "candidates"} for batched plans.

    The sample holds patterns of every (k, metric) batch of the workload, a
    uniform share of each, so its pairs are spread over the groups as the
    workload's are.  Every tile (patterns per tile x population-count-only or
    mixed k = 1 test) runs the sample through a plan without a graph, `reps`
    times after one warm-up, timed by the library's stage events; every
    candidate must return the match lists of the first, and the fastest wins."""
    chars, offsets, n = _strings(sample_chars, sample_offsets)
    groups = sorted({(int(k), str(m)) for _, k, m in batches})
    key = "plan|" + _key(index, groups, "mixed", "fused", _host_offsets(offsets))
    cache = _load()
    if not refresh and key in cache:
        return cache[key]
    total_chars = int(_host_offsets(offsets)[-1]) if n else 0
    ref = None
    cands = []
    for tq in PLAN_TILES:
        for variant in (0, 1):
            plan = Plan(index, max(n, 1), max(total_chars, 1), max(len(batches), 1), tile_queries=tq,
                        variant=variant, graph=False)
            try:
                r = plan.run(chars, offsets, batches=batches)
                got = r.csr()
                r.free()
                ms = []
                for _ in range(reps):
                    r = plan.run(chars, offsets, batches=batches)
                    ms.append(r.stats()["ms_total"])
                    r.free()
            finally:
                plan.free()
            if ref is None:
                ref = got
            elif not (np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])):
                raise RuntimeError(f"autotune: tile {tq} / variant {variant} changed the match lists")
            cands.append({"tile_queries": tq, "variant": variant, "ms": float(min(ms))})
    best = min(cands, key=lambda c: c["ms"])
    opts = {"tile_queries": best["tile_queries"], "variant": best["variant"], "ms": best["ms"], "candidates": cands}
    cache[key] = opts
    _store(cache)
    return opts
