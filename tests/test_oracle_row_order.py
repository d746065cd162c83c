"""Pin of the oracle's independence from the order of clusters in a row.

The method's rules never look at where a cluster sits in the input: every
tie (equal pair residuals in the neighbour finder, equal distances in the
tracklet search, equal selection keys) is decided by cluster id, and
tracklets are numbered in (event, sector, row, id) order.  So permuting the
clusters inside each row must leave every result the same once positions are
mapped back to cluster ids: links, start hits, tracklet clusters and filter
outputs, and tracks, bit for bit in both oracle modes.  The tiny lattice
events put clusters at identical positions, so their ties are decided by the
id rules and a rule that fell back on input order would show here."""
import numpy as np
import pytest

import oracle
from paper_1712_09430_gb300 import synth as S

XR = S.row_x()


def _ids(cl):
    return cl[:, 3].view(np.uint32).astype(np.int64)


def _permuted(cl, rc, seed):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(rc)])
    perm = np.concatenate([off[r] + rng.permutation(int(rc[r])) for r in range(len(rc))])
    return cl[perm]


def _links_by_id(o, ids, key):
    a = o[key]
    dst = np.where(a >= 0, ids[np.maximum(a, 0)], -1)
    return dict(zip(ids.tolist(), dst.tolist()))


def _check(cl, rc, n_events, bz, mode, seed):
    cl2 = _permuted(cl, rc, seed)
    o = oracle.run(cl, rc, n_events, bz, XR, mode=mode)
    o2 = oracle.run(cl2, rc, n_events, bz, XR, mode=mode)
    id1, id2 = _ids(cl), _ids(cl2)
    for k in ("up_raw", "dn_raw", "up", "dn"):
        assert _links_by_id(o, id1, k) == _links_by_id(o2, id2, k), k
    np.testing.assert_array_equal(id2[o2["start"]], id1[o["start"]])
    for k in ("tl_unit", "tl_n", "tl_alive", "tl_hit_off", "trk_t", "trk_n", "trk_hit_off"):
        np.testing.assert_array_equal(o2[k], o[k], err_msg=k)
    np.testing.assert_array_equal(o2["tl_f"], o["tl_f"])
    np.testing.assert_array_equal(id2[o2["tl_hits"]], id1[o["tl_hits"]])
    np.testing.assert_array_equal(id2[o2["trk_hits"]], id1[o["trk_hits"]])
    return o


@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_row_order_does_not_change_results_pp_and_central(mode):
    for ev in (S.pp_event(seed=7), S.central_event(seed=5, scale=0.2)):
        o = _check(ev.clusters, ev.row_counts, 1, ev.bz, mode, seed=1)
        assert len(o["trk_t"]) > 50


@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_row_order_does_not_change_results_with_ties(mode):
    cl, rc = S.tiny_lattice_events(200, seed=12)
    o = _check(cl, rc, 200, 0.5, mode, seed=3)
    assert len(o["up"]) == len(cl)
