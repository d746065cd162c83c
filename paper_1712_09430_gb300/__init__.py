"""GB300-native TPC sector tracker: CA seeding + simplified Kalman-filter track
following (ALICE HLT Phase I), hand-written CUDA for sm_103a behind a C ABI.

    from paper_1712_09430_gb300 import Tracker, synth
    ev = synth.central_event()
    with Tracker(synth.row_x(), bz=ev.bz) as tr:
        res = tr.track(ev.clusters, ev.row_counts, 1)
"""
from .tracker import TRACK_DTYPE, Result, Tracker, TrackerError, default_params  # noqa: F401
