"""Autotuning of the batched pair kernel with an on-disk cache.

nbody_autotune (C ABI) times the NBODY_NTUNE launch shapes on the batch
itself and keeps the fastest.  Results are cached in a JSON file keyed by the
GPU name and a signature of the batch (the sorted sizes rounded to the
padding granularity), so a later run on the same GPU and batch shape selects
the cached candidate with nbody_set_tuning instead of timing again.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import nbody as nb

CACHE = os.environ.get("NBODY_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache",
                                    "paper_2511_22468_gb300", "autotune.json"))


def _key(gpu_name, sizes):
    padded = sorted(((int(n) + 1023) // 1024) * 1024 for n in sizes)
    sig = hashlib.sha256(json.dumps(padded).encode()).hexdigest()[:16]
    return "%s|%d|%s" % (gpu_name, len(padded), sig)


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(h, sizes, gpu_name, probe_steps=3, use_cache=True):
    """Select the launch shape of batch context h; returns (choice, source,
    timings or None)."""
    key = _key(gpu_name, sizes)
    db = _load() if use_cache else {}
    if key in db:
        nb.nbody_set_tuning(h, db[key]["choice"])
        return db[key]["choice"], "cache", None
    best, ms = nb.nbody_autotune(h, probe_steps)
    db = _load()
    db[key] = {"choice": best, "ms": ms}
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + ".%d.tmp" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, CACHE)
    except OSError:
        pass
    return best, "measured", ms
