"""Pin of event independence in the oracle.

The sectors of an event, and the events of a batch, are tracked
independently (Sec. 3.1: one sector per GPU work item; Sec. 3.2: several
events share the GPU), which is what lets the batched GPU form run many
events in one launch.  The oracle tracking three events in one call must
give, event by event, what it gives for each event alone: links, start hits,
tracklet states and clusters, and tracks, with cluster positions, tracklet
numbers and unit numbers offset by the events before, bit for bit in both
modes."""
import numpy as np
import pytest

import oracle
from paper_1712_09430_gb300 import synth as S

XR = S.row_x()
NS = 36


@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_batch_equals_events_alone(mode):
    evs = [S.pp_event(seed=7), S.min_bias_event(1003), S.central_event(seed=5, scale=0.1)]
    cl = np.concatenate([e.clusters for e in evs])
    rc = np.concatenate([e.row_counts for e in evs])
    ob = oracle.run(cl, rc, len(evs), evs[0].bz, XR, mode=mode)
    parts = [oracle.run(e.clusters, e.row_counts, 1, e.bz, XR, mode=mode) for e in evs]
    assert all(len(p["trk_t"]) > 50 for p in parts)
    off_n = np.cumsum([0] + [e.n for e in evs])
    off_t = np.cumsum([0] + [len(p["start"]) for p in parts])

    def cat(key, offs=None):
        out = []
        for i, p in enumerate(parts):
            a = p[key]
            if offs is not None:
                a = np.where(a >= 0, a + offs[i], a)
            out.append(a)
        return np.concatenate(out)

    for k in ("up_raw", "dn_raw", "up", "dn", "start", "tl_hits", "trk_hits"):
        np.testing.assert_array_equal(ob[k], cat(k, off_n), err_msg=k)
    for k in ("tl_n", "tl_alive", "trk_n", "tl_f"):
        np.testing.assert_array_equal(ob[k], cat(k), err_msg=k)
    np.testing.assert_array_equal(ob["trk_t"], cat("trk_t", off_t))
    np.testing.assert_array_equal(ob["tl_unit"], cat("tl_unit", [NS * i for i in range(len(evs))]))
