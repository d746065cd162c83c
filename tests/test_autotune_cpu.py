"""Host side of the autotuner (no GPU): workload keys, the JSON cache, and a
cached choice applied without timing."""
import json

import numpy as np

from paper_1712_09430_gb300 import autotune


def test_workload_key_buckets():
    rc = np.zeros(36 * 159, np.int32)
    rc[:10] = 100                      # 1000 clusters in one event
    assert autotune.workload_key(rc, 1, "GB300") == "GB300|ev1|cl512"
    rc8 = np.tile(rc, 8)
    assert autotune.workload_key(rc8, 8, "GB300") == "GB300|ev8|cl512"
    # events per call and clusters per event fall into power-of-two buckets
    assert autotune.workload_key(np.tile(rc, 5), 5) == autotune.workload_key(np.tile(rc, 7), 7)
    assert autotune.workload_key(rc, 1) != autotune.workload_key(np.tile(rc, 2), 2)
    assert autotune.workload_key(np.zeros(0, np.int32), 0) == "|ev1|cl1"


def test_cache_round_trip_and_bad_files(tmp_path):
    p = tmp_path / "sub" / "cache.json"
    assert autotune.load_cache(str(p)) == {}
    c = {"k": {"schedule": 2, "bin_target": 0.25, "tracklets_per_warp": 32, "threads_per_row": 128,
               "ms": 5.8}}
    autotune.save_cache(c, str(p))
    assert autotune.load_cache(str(p)) == c
    p.write_text("{not json")
    assert autotune.load_cache(str(p)) == {}


def test_cached_choice_is_applied_without_timing(tmp_path):
    class FakeTracker:
        def __init__(self):
            self.applied = None

        def set_params(self, **kw):
            self.applied = kw

    rc = np.zeros(36 * 159, np.int32)
    rc[:4] = 50
    key = autotune.workload_key(rc, 1, "dev")
    choice = {"schedule": 1, "bin_target": 2.0, "tracklets_per_warp": 4, "threads_per_row": 64,
              "lanes_per_hit": 4}
    path = tmp_path / "c.json"
    path.write_text(json.dumps({key: dict(choice, ms=1.5)}))
    tr = FakeTracker()
    fields, ms = autotune.tune(tr, np.zeros((200, 4), np.float32), rc, 1, cache_path=str(path),
                               device_name="dev")
    assert fields == choice and ms == 1.5 and tr.applied == choice
