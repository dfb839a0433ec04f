"""Cached tile shapes from the autotuner.

The cache is a JSON file (default: ~/.cache/fpmatch/autotune.json, or
$FPMATCH_TUNE_CACHE) keyed by GPU model and SM count, library version,
fingerprint type and width, k, metric, form and the dictionary size rounded
to a power of two.  A miss runs fp_autotune on the given pattern sample.
"""
from __future__ import annotations

import json
import os

from . import fp_autotune, fp_version


def cache_path() -> str:
    return os.environ.get("FPMATCH_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fpmatch", "autotune.json"))


def _key(index, k, metric, mode) -> str:
    import torch
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    info = index.info()
    words = max(1, int(info["n_words"]))
    size = 1 << (words - 1).bit_length()
    return "|".join(str(x) for x in (props.name, props.multi_processor_count, fp_version(), info["type"],
                                     info["width_bits"], k, metric, mode, size))


def tuned_opts(index, sample_chars, sample_offsets=None, k: int = 1, metric: str = "ham", mode: str = "tiled",
               reps: int = 2, refresh: bool = False) -> dict:
    """{"tile_queries", "words_per_thread", "variant"} for this GPU and workload."""
    path = cache_path()
    key = _key(index, k, metric, mode)
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if not refresh and key in cache:
        return cache[key]
    best, _ = fp_autotune(index, sample_chars, sample_offsets, k, metric, mode, reps)
    opts = {"tile_queries": best["tile_queries"], "words_per_thread": best["words_per_thread"],
            "variant": best["variant"], "ms": best["ms"]}
    cache[key] = opts
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return opts
