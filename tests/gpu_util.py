"""Helpers shared by the GPU parity tests: run both sides on the same input
and bring their per-stage results into one comparable form."""
import numpy as np

import oracle
from paper_1712_09430_gb300 import capi, synth as S
from paper_1712_09430_gb300.tracker import Tracker

XR = S.row_x()


def gpu_run(clusters, row_counts, n_events, bz=0.5, dumps=True, tracker=None, **params):
    own = tracker is None
    tr = tracker or Tracker(XR, bz=bz, **params)
    try:
        if not own and params:
            tr.set_params(**params)
        res = tr.track(clusters, row_counts, n_events)
        out = dict(tracks=res.tracks, hit_ids=res.hit_ids, hit_off=res.hit_off)
        if dumps:
            lr = tr.dump(capi.TPC_DUMP_LINKS_RAW)
            lc = tr.dump(capi.TPC_DUMP_LINKS)
            out.update(up_raw=lr[0], dn_raw=lr[1], up=lc[0], dn=lc[1])
            out["start"] = tr.dump(capi.TPC_DUMP_STARTS)
            out["tl_f"] = tr.dump(capi.TPC_DUMP_TRACKLETS)
            tn = tr.dump(capi.TPC_DUMP_TRACKLET_N)
            out["tl_n"], out["tl_alive"] = tn[0], tn[1]
            out["tl_hits"] = tr.dump(capi.TPC_DUMP_TRACKLET_HITS)
        return out
    finally:
        if own:
            tr.close()


def oracle_run(clusters, row_counts, n_events, bz=0.5, mode="f32", **params):
    p = oracle.default_params(**params) if params else None
    return oracle.run(clusters, row_counts, n_events, bz, XR, params=p, mode=mode)


def oracle_tl_hits_dense(o, n_rows=159):
    T = len(o["tl_n"])
    dense = np.full((T, n_rows), -1, np.int32)
    for t in range(T):
        h = o["tl_hits"][o["tl_hit_off"][t]:o["tl_hit_off"][t + 1]]
        dense[t, :len(h)] = h
    return dense


def assert_exact_equal(g, o):
    """Bit-exact parity of every stage: links, start hits, tracklets (cluster
    lists and filter outputs) and selected tracks."""
    for k in ("up_raw", "dn_raw", "up", "dn"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    np.testing.assert_array_equal(g["start"], o["start"], err_msg="start hits")
    np.testing.assert_array_equal(g["tl_n"], o["tl_n"], err_msg="tracklet cluster counts")
    np.testing.assert_array_equal(g["tl_alive"], o["tl_alive"], err_msg="tracklet alive")
    np.testing.assert_array_equal(g["tl_hits"], oracle_tl_hits_dense(o), err_msg="tracklet clusters")
    of = o["tl_f"].astype(np.float32)
    np.testing.assert_array_equal(g["tl_f"].view(np.uint32), of.view(np.uint32),
                                  err_msg="tracklet filter state (bits)")
    np.testing.assert_array_equal(g["tracks"]["tracklet"], o["trk_t"], err_msg="selected tracklets")
    np.testing.assert_array_equal(g["tracks"]["nhits"], o["trk_n"], err_msg="owned cluster counts")
    np.testing.assert_array_equal(g["hit_ids"], o["trk_hits"], err_msg="track clusters")
