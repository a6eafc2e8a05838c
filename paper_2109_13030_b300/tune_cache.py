"""Persistent cache of the grouped launch's autotuned settings.

The autotuner (am_group_autotune) times the block sizes that fit every
problem of a group, and the caps on the warp-pair group kernels' trajectory
slots per CTA, and keeps the fastest.  The choice depends on the shapes in
the group, not on the data, so it is stored in a JSON file keyed by the
sorted problem shapes (q, m, n, batch rounded to a power of two), the
problems' kernel choices, the precision form, the SM count and the
iteration count; a later group of the same key reuses it without timing.
"""
from __future__ import annotations

import json
import os


def batch_bucket(B: int) -> int:
    """Smallest power of two >= B (tile counts, hence timings, change slowly in B)."""
    b = 1
    while b < B:
        b <<= 1
    return b


def key(shapes, precision: int, sms: int, iters: int, kernels=None) -> str:
    """shapes: iterable of (q, m, n, B) per problem; kernels: the problems'
    kernel options in the same order (None: the small-tile default for all)."""
    shapes = list(shapes)
    ks = [0] * len(shapes) if kernels is None else [int(k) for k in kernels]
    norm = sorted((int(q), int(m), int(n), batch_bucket(int(B)), k) for (q, m, n, B), k in zip(shapes, ks))
    return json.dumps({"shapes": norm, "precision": int(precision), "sms": int(sms), "iters": int(iters)},
                      sort_keys=True)


def load(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def lookup(path: str, k: str):
    """(threads, ms, warp_slots) stored for key k, or None (an entry without
    warp_slots reads 0: as many as fit)."""
    v = load(path).get(k)
    if isinstance(v, dict) and "threads" in v:
        return int(v["threads"]), float(v.get("ms", 0.0)), int(v.get("warp_slots", 0))
    return None


def store(path: str, k: str, threads: int, ms: float, warp_slots: int = 0) -> None:
    data = load(path)
    data[k] = {"threads": int(threads), "ms": float(ms), "warp_slots": int(warp_slots)}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
