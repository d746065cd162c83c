"""Autotuner front end: tpc_autotune (native, in libtpcca.so) picks the
execution fields -- schedule, grid bin size, tracklets per warp, threads per
row, lanes per hit of the neighbour finder -- for a workload by timing it on the device; this module keeps the
winners in a JSON cache keyed by GPU and workload shape, so a serving
process tunes once per workload class.

The fields change speed only: every value gives bit-identical results.
"""
from __future__ import annotations

import ctypes as C
import json
import math
import os

import numpy as np

from . import capi
from .capi import lib

FIELDS = ("schedule", "bin_target", "tracklets_per_warp", "threads_per_row", "lanes_per_hit")
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "tpc_gb300_autotune.json")


def workload_key(row_counts, n_events, device_name=""):
    """GPU name, events per call (power-of-two bucket) and mean clusters per
    event (power-of-two bucket)."""
    n = int(np.asarray(row_counts, dtype=np.int64).sum())
    per_ev = n / max(1, n_events)
    return f"{device_name}|ev{1 << max(0, int(math.log2(max(1, n_events))))}|" \
           f"cl{1 << max(0, int(math.log2(max(1.0, per_ev))))}"


def load_cache(path=DEFAULT_CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=DEFAULT_CACHE):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(tracker, clusters, row_counts, n_events, reps=3, cache_path=None, device_name=""):
    """Tune `tracker` for this batch (host numpy or device torch clusters).
    With cache_path, a cached choice for the same workload key is applied
    without timing, and new choices are stored.  Returns (fields, ms)."""
    key = workload_key(row_counts, n_events, device_name)
    cache = load_cache(cache_path) if cache_path else {}
    if key in cache and all(f in cache[key] for f in FIELDS):
        tracker.set_params(**{f: cache[key][f] for f in FIELDS})
        return {f: cache[key][f] for f in FIELDS}, cache[key].get("ms")
    rc_arr = np.ascontiguousarray(row_counts, dtype=np.int32)
    is_dev = hasattr(clusters, "is_cuda") and clusters.is_cuda
    if not is_dev:
        clusters = np.ascontiguousarray(clusters, dtype=np.float32)
    ptr = C.c_void_p(clusters.data_ptr()) if is_dev else clusters.ctypes.data_as(C.c_void_p)
    best = capi.tpc_params()
    ms = C.c_float()
    rc = lib().tpc_autotune(tracker.h, ptr, rc_arr.ctypes.data_as(C.c_void_p), int(n_events),
                            capi.TPC_MEM_DEVICE if is_dev else capi.TPC_MEM_HOST, int(reps),
                            C.byref(best), C.byref(ms))
    tracker.check(rc)
    C.memmove(C.byref(tracker.params), C.byref(best), C.sizeof(best))
    fields = {f: getattr(best, f) for f in FIELDS}
    if cache_path:
        cache[key] = dict(fields, ms=float(ms.value))
        save_cache(cache, cache_path)
    return fields, float(ms.value)
