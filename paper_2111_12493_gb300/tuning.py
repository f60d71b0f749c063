"""Autotuned options kept between runs, keyed by the shape of the graph.

bisim_autotune times candidate degree-class thresholds, hub chunk sizes and,
on a batched context, the batch split, on the context's own graph. That costs
a few dozen refinement runs; `autotune_cached` looks the context's shape up in
a JSON file first. On a hit the stored settings go to the context through
bisim_retune (nothing is timed); on a miss the tuner runs and its choice is
stored under the shape's key. Results never depend on these settings, only the
time does, so a graph of the same shape can share them.

The key holds what the tuned settings depend on: batched or not, the counts
of vertices, edges and graphs, the vertices in each degree bucket (all rounded
to two significant digits), the direction, the label filter's size, the hash
width and the device's name.
"""

from __future__ import annotations

import json
import os
import tempfile

from . import bisim

_VERSION = 1


def _round2(x: int) -> int:
    """A count x >= 0 rounded half up to two significant digits."""
    x = int(x)
    if x <= 0:
        return 0
    step = 10 ** max(0, len(str(x)) - 2)
    return (x + step // 2) // step * step


def shape_key(stats: dict, options: dict, device: str) -> str:
    parts = [
        "batched" if stats["n_graphs"] > 1 else "single",
        f"n{_round2(stats['n_vertices'])}",
        f"m{_round2(stats['n_edges'])}",
        f"g{_round2(stats['n_graphs'])}",
        f"s{_round2(stats['n_small'])}",
        f"w{_round2(stats['n_mid'])}",
        f"h{_round2(stats['n_hub'])}",
        f"dir{options.get('direction', 0)}",
        f"lf{options.get('n_label_filter', 0)}",
        f"hb{options.get('hash_bits', 64)}",
        device.replace("|", "/"),
    ]
    return "|".join(parts)


class TuneCache:
    """A JSON file of {shape key: tuned settings}; written whole on every store,
    through a temporary file renamed over it."""

    def __init__(self, path: str):
        self.path = path
        self.entries: dict = {}
        if os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
            if data.get("version") == _VERSION:
                self.entries = dict(data.get("entries", {}))

    def lookup(self, key: str):
        hit = self.entries.get(key)
        return None if hit is None else {k: int(hit[k]) for k in bisim.TUNING_FIELDS if k in hit}

    def store(self, key: str, settings: dict) -> None:
        self.entries[key] = {k: int(settings[k]) for k in bisim.TUNING_FIELDS}
        folder = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(folder, exist_ok=True)
        fd, tmp = tempfile.mkstemp(prefix=".tune", dir=folder)
        with os.fdopen(fd, "w") as f:
            json.dump({"version": _VERSION, "entries": self.entries}, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "no-device"


def autotune_cached(ctx, cache: TuneCache, options=None, rounds: int = 2, stream=None) -> tuple:
    """Tuned settings for `ctx`, from the cache when its shape is known.

    `options` are the bisim_options the context was created with (None: the
    defaults). Returns (settings dict, True when they came from the cache).
    """
    opts = options if options is not None else bisim.default_options()
    key = shape_key(bisim.bisim_get_stats(ctx), {f: getattr(opts, f) for f, _ in opts._fields_}, _device_name())
    hit = cache.lookup(key)
    if hit is not None:
        bisim.bisim_retune(ctx, stream=stream, **hit)
        return hit, True
    tuned = bisim.bisim_autotune(ctx, rounds=rounds, stream=stream)
    settings = {k: int(tuned[k]) for k in bisim.TUNING_FIELDS}
    cache.store(key, settings)
    return settings, False
