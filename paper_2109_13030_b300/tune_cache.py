"""Persistent cache of the grouped launch's autotuned block size.

The autotuner (am_group_autotune) times the block sizes that fit every
problem of a group and keeps the fastest.  The choice depends on the shapes
in the group, not on the data, so it is stored in a JSON file keyed by the
sorted problem shapes (q, m, n, batch rounded to a power of two), the
precision form, the SM count and the iteration count; a later group of the
same key reuses it without timing.
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


def key(shapes, precision: int, sms: int, iters: int) -> str:
    """shapes: iterable of (q, m, n, B) per problem."""
    norm = sorted((int(q), int(m), int(n), batch_bucket(int(B))) for q, m, n, B in shapes)
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
    """(threads, ms) stored for key k, or None."""
    v = load(path).get(k)
    if isinstance(v, dict) and "threads" in v:
        return int(v["threads"]), float(v.get("ms", 0.0))
    return None


def store(path: str, k: str, threads: int, ms: float) -> None:
    data = load(path)
    data[k] = {"threads": int(threads), "ms": float(ms)}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
