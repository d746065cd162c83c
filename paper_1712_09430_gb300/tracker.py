"""Python convenience layer over the C ABI: numpy/torch in, numpy out.

All work happens in libtpcca.so.  torch is used only for device memory and
streams (device-resident inputs, pinned host buffers, the current stream).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi
from .capi import lib

TRACK_DTYPE = np.dtype([("event", np.int32), ("sector", np.int32), ("tracklet", np.int32),
                        ("x", np.float32), ("p", np.float32, 5), ("cov_y", np.float32, 6),
                        ("cov_z", np.float32, 3), ("chi2", np.float32), ("ndf", np.int32),
                        ("nhits", np.int32), ("hit_off", np.int32)])
assert TRACK_DTYPE.itemsize == C.sizeof(capi.tpc_track)
FIT_DTYPE = np.dtype([("x", np.float32), ("p", np.float32, 5), ("cov", np.float32, 15),
                      ("chi2", np.float32), ("ndf", np.int32), ("status", np.int32)])
assert FIT_DTYPE.itemsize == C.sizeof(capi.tpc_fit)
MERGE_DTYPE = np.dtype([("next", np.int32), ("chi2", np.float32)])
assert MERGE_DTYPE.itemsize == C.sizeof(capi.tpc_merge)
T0_DTYPE = np.dtype([("collision", np.int32), ("u", np.float32), ("dz", np.float32)])
assert T0_DTYPE.itemsize == C.sizeof(capi.tpc_t0)


class TrackerError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{capi.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _set(p, k, v):
    """Set field k of a tpc_params; a name that is not a field is an error
    (a ctypes structure would otherwise keep it as a plain attribute)."""
    if k not in {f for f, _ in type(p)._fields_}:
        raise TypeError(f"unknown tracker parameter {k!r}")
    if k == "field":
        v = (C.c_float * 5)(*[float(x) for x in v])
    setattr(p, k, v)


def default_params(**over) -> capi.tpc_params:
    """tpc_params_default() with the named fields replaced."""
    p = capi.tpc_params()
    lib().tpc_params_default(C.byref(p))
    for k, v in over.items():
        _set(p, k, v)
    return p


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class Result:
    """Tracks (structured numpy array, TRACK_DTYPE), their hit ids, with
    params.refit the full Kalman filter refit of each track (FIT_DTYPE), and
    with params.merge each track's merge link (MERGE_DTYPE)."""

    def __init__(self, tracks, hit_ids, fits=None, merges=None, t0s=None):
        self.tracks = tracks
        self.hit_ids = hit_ids
        self.fits = fits
        self.merges = merges
        self.t0s = t0s

    def hits_of(self, m):
        t = self.tracks[m]
        return self.hit_ids[t["hit_off"]:t["hit_off"] + t["nhits"]]

    @property
    def hit_off(self):
        off = np.zeros(len(self.tracks) + 1, np.int64)
        off[1:] = np.cumsum(self.tracks["nhits"])
        return off


class Tracker:
    """One tpc_tracker on the current CUDA device."""

    def __init__(self, row_x, bz=0.5, params=None, n_sectors=36, tan_half_open=None, z_max=250.0,
                 **param_over):
        import math
        self._xr = np.ascontiguousarray(row_x, dtype=np.float32)
        g = capi.tpc_geometry()
        g.n_rows = len(self._xr)
        g.n_sectors = n_sectors
        g.row_x = self._xr.ctypes.data_as(C.POINTER(C.c_float))
        g.tan_half_open = math.tan(math.radians(10.0)) if tan_half_open is None else tan_half_open
        g.z_max = z_max
        self.n_rows, self.n_sectors = g.n_rows, n_sectors
        p = params if params is not None else default_params(**param_over)
        h = C.c_void_p()
        rc = lib().tpc_tracker_create(C.byref(g), float(bz), C.byref(p), C.byref(h))
        if rc != capi.TPC_OK:
            raise TrackerError(rc, lib().tpc_last_error(None).decode())
        self.h = h
        self.params = p
        self._est_tracks = 1024
        self._est_hits = 65536

    def close(self):
        """Destroy the tracker (device memory, streams, graphs); idempotent."""
        if getattr(self, "h", None):
            lib().tpc_tracker_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def error(self):
        """Message of the last failed call (tpc_last_error)."""
        return lib().tpc_last_error(self.h).decode()

    def check(self, rc, ok=(capi.TPC_OK,)):
        """Raise TrackerError(rc, message) unless rc is one of `ok`."""
        if rc not in ok:
            raise TrackerError(rc, self.error())
        return rc

    def set_params(self, **over):
        """Change parameters by name (tpc_tracker_set_params); the others keep
        their current values.  Invalid values raise and change nothing."""
        p = capi.tpc_params()
        C.memmove(C.byref(p), C.byref(self.params), C.sizeof(p))
        for k, v in over.items():
            _set(p, k, v)
        self.check(lib().tpc_tracker_set_params(self.h, C.byref(p)))
        self.params = p

    def track(self, clusters, row_counts, n_events, stream=None, cap_tracks=None, cap_hits=None):
        """Track a batch.  clusters: numpy float32 [N, 4] (host) or a torch
        CUDA tensor (device).  row_counts: numpy int32, host."""
        rc_arr = np.ascontiguousarray(row_counts, dtype=np.int32)
        is_dev = hasattr(clusters, "is_cuda") and clusters.is_cuda
        if not is_dev:
            clusters = np.ascontiguousarray(clusters, dtype=np.float32)
        kind = capi.TPC_MEM_DEVICE if is_dev else capi.TPC_MEM_HOST
        fixed = cap_tracks is not None or cap_hits is not None
        ct = cap_tracks if cap_tracks is not None else self._est_tracks
        ch = cap_hits if cap_hits is not None else self._est_hits
        tracks = np.zeros(max(ct, 1), TRACK_DTYPE)
        hits = np.zeros(max(ch, 1), np.int32)
        opt = self._optional(max(ct, 1))
        out = capi.tpc_output(tracks.ctypes.data, hits.ctypes.data, ct, ch, capi.TPC_MEM_HOST, 0, 0,
                              *self._ptrs(opt))
        rc = lib().tpc_track_sectors(self.h, _ptr(clusters), _ptr(rc_arr), int(n_events), kind,
                                     C.byref(out), stream)
        if rc == capi.TPC_ERR_OUTPUT_TRUNCATED and not fixed:
            # the estimate was short: fetch the rest (no recompute)
            ct, ch = max(out.n_tracks, 1), max(out.n_hits, 1)
            self._est_tracks, self._est_hits = int(ct * 1.25) + 16, int(ch * 1.25) + 256
            tracks = np.zeros(ct, TRACK_DTYPE)
            hits = np.zeros(ch, np.int32)
            opt = self._optional(ct)
            out = capi.tpc_output(tracks.ctypes.data, hits.ctypes.data, ct, ch, capi.TPC_MEM_HOST,
                                  0, 0, *self._ptrs(opt))
            rc = lib().tpc_fetch_output(self.h, C.byref(out))
        self.check(rc)
        return Result(tracks[:out.n_tracks], hits[:out.n_hits],
                      *[a[:out.n_tracks] if a is not None else None for a in opt])

    def _optional(self, n):
        """Buffers of the optional per-track outputs the params switch on:
        fits (refit), merges (merge), t0s (t0)."""
        p = self.params
        return (np.zeros(n, FIT_DTYPE) if p.refit else None,
                np.zeros(n, MERGE_DTYPE) if p.merge else None,
                np.zeros(n, T0_DTYPE) if p.t0 else None)

    @staticmethod
    def _ptrs(opt):
        return [a.ctypes.data if a is not None else None for a in opt]

    # ---- serving (continuous batching) -----------------------------------
    def stream_configure(self, arena_bytes=0, max_batch_events=64, max_inflight=2, no_copy=False,
                         max_batch_clusters=capi.TPC_STREAM_BATCH_CLUSTERS):
        """Set up the request loop (tpc_stream_configure): device arena bytes
        (0: half of the free device memory, at most 24 GiB), events and
        clusters per batch (max_batch_clusters 0: no limit), batches in
        flight (1..8); no_copy: submitted host buffers are read in place
        (pinned memory the caller keeps alive until the result is polled)."""
        self.check(lib().tpc_stream_configure(self.h, int(arena_bytes), int(max_batch_events),
                                              int(max_inflight),
                                              capi.TPC_STREAM_NO_COPY if no_copy else 0,
                                              int(max_batch_clusters)))

    def stream_set_batching(self, min_batch_clusters=0, max_wait_us=0):
        """Batching policy (tpc_stream_set_batching): while a batch runs, form
        the next one only once min_batch_clusters clusters are pending, a
        batch is full, or the oldest request has waited max_wait_us."""
        self.check(lib().tpc_stream_set_batching(self.h, int(min_batch_clusters), int(max_wait_us)))

    def stream_stats(self):
        """Counters of the request loop (batches, events, device and host ms)."""
        st = capi.tpc_stream_stats()
        self.check(lib().tpc_stream_get_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def submit(self, clusters, row_counts, n_events=1, tag=0):
        """Returns a ticket, or None when the request is not admitted now.
        clusters: numpy float32 [N, 4] or a (pinned) torch CPU tensor; with
        no_copy the caller keeps it alive until the result is polled."""
        cl = clusters if hasattr(clusters, "data_ptr") else np.ascontiguousarray(clusters,
                                                                                 dtype=np.float32)
        rc_arr = np.ascontiguousarray(row_counts, dtype=np.int32)
        t = C.c_uint64()
        rc = lib().tpc_stream_submit(self.h, _ptr(cl), _ptr(rc_arr), int(n_events), int(tag),
                                     C.byref(t))
        if rc == capi.TPC_BUSY:
            return None
        self.check(rc)
        return int(t.value)

    def poll(self, ticket, timeout_us=0):
        """Result of a ticket, or None while it is pending.  A first call
        with no capacity learns the sizes; the second fills exact arrays."""
        out = capi.tpc_output(None, None, 0, 0, capi.TPC_MEM_HOST, 0, 0)
        rc = lib().tpc_stream_poll(self.h, int(ticket), C.byref(out), int(timeout_us))
        if rc == capi.TPC_PENDING:
            return None
        if rc == capi.TPC_OK:       # an empty result
            return Result(np.zeros(0, TRACK_DTYPE), np.zeros(0, np.int32), *self._optional(0))
        if rc != capi.TPC_ERR_OUTPUT_TRUNCATED:
            self.check(rc)
        tracks = np.empty(max(out.n_tracks, 1), TRACK_DTYPE)
        hits = np.empty(max(out.n_hits, 1), np.int32)
        opt = self._optional(max(out.n_tracks, 1))
        out = capi.tpc_output(tracks.ctypes.data, hits.ctypes.data, len(tracks), len(hits),
                              capi.TPC_MEM_HOST, 0, 0, *self._ptrs(opt))
        self.check(lib().tpc_stream_poll(self.h, int(ticket), C.byref(out), 0))
        return Result(tracks[:out.n_tracks], hits[:out.n_hits],
                      *[a[:out.n_tracks] if a is not None else None for a in opt])

    def poll_view(self, ticket, timeout_us=0):
        """Result of a ticket without a copy (numpy views of the library's
        pinned buffers), or None while pending.  The views stay valid until
        release(ticket)."""
        v = capi.tpc_stream_view()
        rc = lib().tpc_stream_poll_view(self.h, int(ticket), C.byref(v), int(timeout_us))
        if rc == capi.TPC_PENDING:
            return None
        self.check(rc)
        return self._view_result(v)

    def _view_result(self, v):
        """Numpy views of a tpc_stream_view."""
        def arr(ptr, n, dt):
            if n == 0 or not ptr:
                return np.zeros(0, dt)
            return np.frombuffer((C.c_char * (n * dt.itemsize)).from_address(ptr), dtype=dt)
        fits = arr(v.fits, v.n_tracks, FIT_DTYPE) if self.params.refit else None
        merges = arr(v.merges, v.n_tracks, MERGE_DTYPE) if self.params.merge else None
        t0s = arr(v.t0s, v.n_tracks, T0_DTYPE) if self.params.t0 else None
        return Result(arr(v.tracks, v.n_tracks, TRACK_DTYPE), arr(v.hit_ids, v.n_hits, np.dtype(np.int32)),
                      fits, merges, t0s)

    def poll_any(self, timeout_us=0):
        """(ticket, Result as numpy views) of whichever ticket finished first
        and has not been taken yet, or None; the views stay valid until
        release(ticket).  A failed request raises TrackerError (its ticket
        is released)."""
        v = capi.tpc_stream_view()
        t = C.c_uint64()
        rc = lib().tpc_stream_poll_any(self.h, C.byref(t), C.byref(v), int(timeout_us))
        if rc == capi.TPC_PENDING:
            return None
        self.check(rc)
        return int(t.value), self._view_result(v)

    def release(self, ticket):
        """Return a ticket's result buffers (after poll_view) to the library."""
        self.check(lib().tpc_stream_release(self.h, int(ticket)))

    def dump(self, what):
        """Per-stage results of the last call (tpc_debug_dump, capi.TPC_DUMP_*)
        as numpy arrays: links [2, N], start hits [T], tracklet states [T, 16],
        tracklet counts and survival [2, T], work counts [4, T], tracklet
        clusters [T, n_rows]."""
        n = C.c_int64()
        # probe the size
        rc = lib().tpc_debug_dump(self.h, what, _ptr(np.zeros(1, np.int32)), 0, C.byref(n))
        if rc not in (capi.TPC_OK, capi.TPC_ERR_OUTPUT_TRUNCATED):
            self.check(rc)
        k = int(n.value)
        if what in (capi.TPC_DUMP_LINKS_RAW, capi.TPC_DUMP_LINKS, capi.TPC_DUMP_TRACKLET_N):
            a = np.zeros((2, k), np.int32)
        elif what == capi.TPC_DUMP_STARTS:
            a = np.zeros(k, np.int32)
        elif what == capi.TPC_DUMP_TRACKLETS:
            a = np.zeros((k, 16), np.float32)
        elif what == capi.TPC_DUMP_TRACKLET_WORK:
            a = np.zeros((4, k), np.int32)
        else:
            a = np.zeros((k, self.n_rows), np.int32)
        self.check(lib().tpc_debug_dump(self.h, what, _ptr(a), a.nbytes, C.byref(n)))
        return a

    def stage_times(self):
        """ms of: grid, neighbours, clean + start hits, tracklets, selection +
        output, whole call, final refit."""
        ms = (C.c_float * 7)()
        self.check(lib().tpc_stage_times(self.h, ms, 7))
        return list(ms)
