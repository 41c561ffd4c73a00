"""Persistent autotuning results.

rk4_chain_autotune times every candidate tiling (and, for batches, the persistent against the
blocked scheme), which takes seconds at large N.  The cache keeps its choice in a JSON file so
that a later run on the same kind of GPU and workload applies it directly: the environment
variable RK4CHAIN_TUNE_CACHE (or an explicit ``path``) names the file.  Entries are keyed by
the GPU name, model, precision, number of chains, total sites rounded to a power of two, and a
caller-supplied scheme tag (for example the tableau and coupling range); the value is the
kernel and the (block, v, k) tiling.  Writes replace the file atomically; two processes
writing at once can lose one entry, never corrupt the file.  A cached choice is a tiling the
autotuner once measured fastest: results are bit-identical whichever tiling runs.  An entry
the library rejects when it is applied (written by a build with other kernel limits) is tuned
again and replaced.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

ENV = "RK4CHAIN_TUNE_CACHE"


def make_key(device: str, model: int, precision: int, nchains: int, total_sites: int, scheme: str = "rk4") -> str:
    """Cache key of a workload; sites are bucketed to the nearest power of two."""
    bucket = int(round(math.log2(max(int(total_sites), 1))))
    return f"{device}|m{int(model)}|p{int(precision)}|c{int(nchains)}|n2^{bucket}|{scheme}"


def load(path: str) -> dict:
    """The cache's entries ({} when the file is missing or unreadable)."""
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(path: str, key: str, entry: dict) -> None:
    """Add or replace one entry (atomic replace of the whole file)."""
    data = load(path)
    data[key] = entry
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".rk4tune", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def autotune(h, state, comp, ws, key: str, *, probe_steps: int = 16, path: str | None = None, tuner=None,
             apply=None, get_kernel=None) -> dict:
    """Apply the cached choice for `key` to handle h, or run the autotuner and cache its choice.

    Returns the tiling dict with "kernel" and "cached" added.  tuner / apply / get_kernel
    default to rk4_chain_autotune, rk4_chain_set_kernel + rk4_chain_set_tiling and
    rk4_chain_get_kernel (they can be replaced, e.g. to test the cache without a GPU).
    Without a path (argument or RK4CHAIN_TUNE_CACHE) this is plain rk4_chain_autotune."""
    from . import (RK4Error, rk4_chain_autotune, rk4_chain_get_kernel, rk4_chain_set_kernel,
                   rk4_chain_set_tiling)
    tuner = tuner or (lambda: rk4_chain_autotune(h, state, comp, ws, probe_steps))
    get_kernel = get_kernel or (lambda: rk4_chain_get_kernel(h))

    def _apply(entry):
        rk4_chain_set_kernel(h, entry["kernel"])
        rk4_chain_set_tiling(h, entry["block"], entry["v"], entry["k"])

    apply = apply or _apply
    path = path or os.environ.get(ENV)
    if path:
        entry = load(path).get(key)
        if entry and all(f in entry for f in ("kernel", "block", "v", "k")):
            try:
                apply(entry)
                return dict(entry, cached=True)
            except RK4Error:
                pass  # a stale entry (a tiling the library no longer accepts): tune again
    best = dict(tuner())
    best["kernel"] = int(get_kernel())
    if path:
        store(path, key, {f: best[f] for f in ("kernel", "block", "v", "k", "G") if f in best})
    return dict(best, cached=False)
