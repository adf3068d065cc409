"""Persistent tuning cache for libdot's per-context shape table.

Entries are keyed by (GPU name, SM count, op, size bucket), where the size
bucket is the bit length of the limb count m (the granularity of the
library's table).  The cache is a small JSON file at $DOT_TUNE_CACHE, or
~/.cache/dot_gb300/tuning.json.  Values are the knobs of dot_tune_set: the
multiply's columns per thread block R, or the segments per thread of the
tiled add/sub.
"""
from __future__ import annotations

import json
import os

OPS = {0: "add", 1: "sub", 2: "mul"}


def cache_path() -> str:
    p = os.environ.get("DOT_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "dot_gb300", "tuning.json")


def bucket(m: int) -> int:
    return int(m).bit_length()


def key(gpu: str, sms: int, op: int, m: int) -> str:
    return f"{gpu}|{sms}|{OPS[op]}|{bucket(m)}"


def load(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save(entries: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(ctx, gpu: str, sms: int, entries: dict | None = None) -> int:
    """Load every cached knob for this GPU into the context; returns how many."""
    entries = load() if entries is None else entries
    n = 0
    for k, v in entries.items():
        g, s, op, b = k.split("|")
        if g != gpu or int(s) != sms:
            continue
        opc = {name: code for code, name in OPS.items()}[op]
        ctx.tune_set(opc, 1 << (int(b) - 1), int(v["knob"]))
        n += 1
    return n


def tune(ctx, gpu: str, sms: int, op: int, m: int, batch: int, path: str | None = None):
    """Autotune (op, m) on the context, store the result in the cache file and
    return (knob, ms per call)."""
    knob, ms = ctx.autotune(op, m, batch)
    entries = load(path)
    entries[key(gpu, sms, op, m)] = {"knob": knob, "ms": ms, "m": m, "batch": batch}
    save(entries, path)
    return knob, ms


def device_identity(device: int = 0):
    import torch
    p = torch.cuda.get_device_properties(device)
    return p.name, p.multi_processor_count
