"""Thin ctypes binding of include/tpc_tracker.h (argument marshalling only).

The functions keep the C names.  Every stage of the tracker runs in the CUDA
kernels of libtpcca.so; this module only moves pointers and sizes.  There is
no CPU fallback: if the library cannot be loaded, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build_ext

TPC_OK = 0
TPC_PENDING = 1
TPC_BUSY = 2
TPC_ERR_INVALID = -1
TPC_ERR_NOMEM = -2
TPC_ERR_OUTPUT_TRUNCATED = -3
TPC_ERR_TIMEOUT = -4
TPC_ERR_DEVICE = -5
TPC_ERR_CANCELLED = -6
TPC_ERR_UNKNOWN_TICKET = -7
TPC_MEM_HOST = 0
TPC_MEM_DEVICE = 1
TPC_MAX_ROWS = 256
TPC_MAX_ROW_CLUSTERS = 4096
TPC_DUMP_LINKS_RAW = 0
TPC_DUMP_LINKS = 1
TPC_DUMP_STARTS = 2
TPC_DUMP_TRACKLETS = 3
TPC_DUMP_TRACKLET_N = 4
TPC_DUMP_TRACKLET_HITS = 5
TPC_DUMP_TRACKLET_WORK = 6
TPC_NOALLOC_MAX_CLUSTERS = 65536
TPC_NOALLOC_SCRATCH_BYTES = 8 << 20
TPC_STREAM_NO_COPY = 1
TPC_STREAM_BATCH_CLUSTERS = 1 << 22  # default cluster limit of one serving batch

STATUS_NAMES = {0: "TPC_OK", 1: "TPC_PENDING", 2: "TPC_BUSY", -1: "TPC_ERR_INVALID",
                -2: "TPC_ERR_NOMEM", -3: "TPC_ERR_OUTPUT_TRUNCATED", -4: "TPC_ERR_TIMEOUT",
                -5: "TPC_ERR_DEVICE", -6: "TPC_ERR_CANCELLED", -7: "TPC_ERR_UNKNOWN_TICKET"}


class tpc_geometry(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("n_sectors", C.c_int), ("row_x", C.POINTER(C.c_float)),
                ("tan_half_open", C.c_float), ("z_max", C.c_float)]


class tpc_params(C.Structure):
    _fields_ = [("k_win", C.c_float), ("d_max2", C.c_float), ("l_seed", C.c_int),
                ("sigma_y", C.c_float), ("sigma_z", C.c_float),
                ("var_s", C.c_float), ("var_q", C.c_float), ("var_t", C.c_float),
                ("n_sigma", C.c_float), ("w_min", C.c_float), ("w_max", C.c_float),
                ("s_max", C.c_float), ("y_margin", C.c_float), ("g_max", C.c_int),
                ("n_min_tracklet", C.c_int), ("n_min_track", C.c_int),
                ("own_num", C.c_int), ("own_den", C.c_int),
                ("exact_fp32", C.c_int), ("bin_target", C.c_float),
                ("threads_per_row", C.c_int), ("tracklets_per_warp", C.c_int),
                ("plain_per_sector", C.c_int), ("use_graph", C.c_int), ("n_queues", C.c_int),
                ("schedule", C.c_int), ("refit", C.c_int), ("field", C.c_float * 5),
                ("merge", C.c_int), ("merge_chi2", C.c_float), ("merge_gap", C.c_float),
                ("merge_overlap", C.c_float), ("merge_window", C.c_float),
                ("t0", C.c_int), ("t0_y_cut", C.c_float), ("t0_bin", C.c_float),
                ("t0_radius", C.c_float), ("t0_window", C.c_int), ("t0_n_min", C.c_int),
                ("count_work", C.c_int), ("debug_wait_polls", C.c_int),
                ("lanes_per_hit", C.c_int)]


class tpc_track(C.Structure):
    _fields_ = [("event", C.c_int32), ("sector", C.c_int32), ("tracklet", C.c_int32),
                ("x", C.c_float), ("p", C.c_float * 5), ("cov_y", C.c_float * 6),
                ("cov_z", C.c_float * 3), ("chi2", C.c_float), ("ndf", C.c_int32),
                ("nhits", C.c_int32), ("hit_off", C.c_int32)]


class tpc_fit(C.Structure):
    _fields_ = [("x", C.c_float), ("p", C.c_float * 5), ("cov", C.c_float * 15),
                ("chi2", C.c_float), ("ndf", C.c_int32), ("status", C.c_int32)]


class tpc_merge(C.Structure):
    _fields_ = [("next", C.c_int32), ("chi2", C.c_float)]


class tpc_t0(C.Structure):
    _fields_ = [("collision", C.c_int32), ("u", C.c_float), ("dz", C.c_float)]


class tpc_output(C.Structure):
    _fields_ = [("tracks", C.c_void_p), ("hit_ids", C.c_void_p), ("cap_tracks", C.c_int32),
                ("cap_hits", C.c_int32), ("mem_kind", C.c_int32), ("n_tracks", C.c_int32),
                ("n_hits", C.c_int32), ("fits", C.c_void_p), ("merges", C.c_void_p),
                ("t0s", C.c_void_p)]


class tpc_stream_stats(C.Structure):
    _fields_ = [("batches", C.c_int64), ("events", C.c_int64), ("clusters", C.c_int64),
                ("refetches", C.c_int64), ("max_batch_events", C.c_int64), ("gpu_ms", C.c_double),
                ("host_launch_ms", C.c_double), ("host_finish_ms", C.c_double),
                ("host_copy_ms", C.c_double), ("max_launch_ms", C.c_double),
                ("max_submit_ms", C.c_double)]


class tpc_stream_view(C.Structure):
    _fields_ = [("tracks", C.c_void_p), ("hit_ids", C.c_void_p), ("fits", C.c_void_p),
                ("merges", C.c_void_p), ("t0s", C.c_void_p), ("n_tracks", C.c_int32),
                ("n_hits", C.c_int32)]


_LIB = None


def lib() -> C.CDLL:
    """Load libtpcca.so (building it in-tree first if it is missing)."""
    global _LIB
    if _LIB is None:
        path = build_ext.LIB
        if not build_ext.up_to_date():
            path = build_ext.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA tracker library missing: {path}")
        L = C.CDLL(path)
        P, V = C.POINTER, C.c_void_p
        L.tpc_params_default.argtypes = [P(tpc_params)]
        L.tpc_params_default.restype = None
        L.tpc_tracker_create.argtypes = [P(tpc_geometry), C.c_double, P(tpc_params), P(V)]
        L.tpc_tracker_destroy.argtypes = [V]
        L.tpc_tracker_destroy.restype = None
        L.tpc_tracker_set_params.argtypes = [V, P(tpc_params)]
        L.tpc_track_sectors.argtypes = [V, V, V, C.c_int, C.c_int, P(tpc_output), V]
        L.tpc_fetch_output.argtypes = [V, P(tpc_output)]
        L.tpc_autotune.argtypes = [V, V, V, C.c_int, C.c_int, C.c_int, P(tpc_params), P(C.c_float)]
        L.tpc_stream_submit.argtypes = [V, V, V, C.c_int, C.c_uint64, P(C.c_uint64)]
        L.tpc_stream_poll.argtypes = [V, C.c_uint64, P(tpc_output), C.c_int]
        L.tpc_stream_configure.argtypes = [V, C.c_size_t, C.c_int, C.c_int, C.c_int, C.c_int64]
        L.tpc_stream_set_batching.argtypes = [V, C.c_int64, C.c_int]
        L.tpc_stream_get_stats.argtypes = [V, P(tpc_stream_stats)]
        L.tpc_stream_poll_view.argtypes = [V, C.c_uint64, P(tpc_stream_view), C.c_int]
        L.tpc_stream_release.argtypes = [V, C.c_uint64]
        L.tpc_stream_poll_any.argtypes = [V, P(C.c_uint64), P(tpc_stream_view), C.c_int]
        L.tpc_debug_dump.argtypes = [V, C.c_int, V, C.c_int64, P(C.c_int64)]
        L.tpc_stage_times.argtypes = [V, P(C.c_float), C.c_int]
        L.tpc_last_error.argtypes = [V]
        L.tpc_last_error.restype = C.c_char_p
        L.tpc_links_noalloc.argtypes = [P(tpc_geometry), P(tpc_params), V, V, V, V]
        _LIB = L
    return _LIB


def exported_symbols():
    """Names the header declares (for the load/export test)."""
    import re
    hdr = os.path.join(build_ext.INCLUDE, "tpc_tracker.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(tpc_\w+)\s*\(", text, re.M)))
