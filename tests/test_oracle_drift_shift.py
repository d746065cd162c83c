"""Pin of reading T01 on the oracle: tracking on the drift coordinate.

In continuous readout (Sec. 3.3, Run 3 conditions) a collision's unknown
time shifts all of its clusters along z by sign(side) dz.  The tracker runs
on that drift coordinate and the collision offsets are estimated afterwards
from the refitted tracks (T02-T04), with no second, re-transformed tracking
pass.  That is sound only if a z shift changes nothing but z: neighbour links
compare z differences, and the filter's z block sees z only through residuals
and increments.  Here the oracle tracks the same event twice, once with every
cluster moved towards z = 0 by dz, and the two results are compared.  The one
cut on absolute z, |z| <= z_max, may end a track that reaches the endcap at a
different row; those tracklets are the only ones allowed to differ."""
import numpy as np
import pytest

import oracle
from paper_1712_09430_gb300 import synth as S

XR = S.row_x()
NR, NS = len(XR), 36
Z_MAX = 250.0


def _shifted(ev, dz):
    """Every cluster moved by dz towards z = 0: z - dz on side A, z + dz on
    side C (sectors 0-17 are side A)."""
    unit = np.repeat(np.arange(len(ev.row_counts)) // NR, ev.row_counts)
    side_a = (unit % NS) < NS // 2
    cl = ev.clusters.copy()
    cl[:, 2] = np.where(side_a, cl[:, 2] - dz, cl[:, 2] + dz).astype(np.float32)
    return cl, side_a


def _track_lists(o):
    off = o["trk_hit_off"]
    return [tuple(o["trk_hits"][off[m]:off[m + 1]]) for m in range(len(o["trk_t"]))]


@pytest.mark.parametrize("dz", [3.0, 17.0])
def test_pp_event_tracks_unchanged_by_a_drift_shift(dz):
    """A pp-like event (no track reaches the endcap cut differently): links,
    every tracklet's cluster count and every track's clusters are identical."""
    ev = S.pp_event(seed=7)
    o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR, mode="f64")
    cl, _ = _shifted(ev, dz)
    o2 = oracle.run(cl, ev.row_counts, 1, ev.bz, XR, mode="f64")
    assert len(o["trk_t"]) > 50
    for k in ("up_raw", "dn_raw", "up", "dn", "start", "tl_n", "trk_t"):
        np.testing.assert_array_equal(o2[k], o[k], err_msg=k)
    assert _track_lists(o2) == _track_lists(o)


# z and tan(lambda) agree up to the rounding of the shifted float32 inputs
# (FP64 mode) or of the float32 arithmetic itself (FP32_EXACT mode, the one
# the GPU's exact build reproduces bit for bit)
TOL = {"f64": 2e-6, "f32": 2e-4}


@pytest.mark.parametrize("mode", ["f64", "f32"])
@pytest.mark.parametrize("dz", [3.0, 17.0])
def test_dense_event_fits_move_only_along_z(dz, mode):
    """A denser event: links are identical; a tracklet whose results differ is
    one that reaches |z| near z_max inside the outer radius; every other
    tracklet has the same y, sin(phi) and q/pT bit for bit (the y block never
    sees z), z moved by the shift and the same tan(lambda)."""
    ev = S.central_event(seed=5, scale=0.2)
    o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR, mode=mode)
    cl, side_a = _shifted(ev, dz)
    o2 = oracle.run(cl, ev.row_counts, 1, ev.bz, XR, mode=mode)
    for k in ("up_raw", "dn_raw", "up", "dn", "start"):
        np.testing.assert_array_equal(o2[k], o[k], err_msg=k)
    f1, f2 = o["tl_f"], o2["tl_f"]
    # state columns: x y z sin(phi) tan(lambda) q/pT ...
    x0, z0, t = f1[:, 0], f1[:, 2], f1[:, 4]
    z_outer = z0 + t * (XR[-1] - x0) * 1.05      # generous: the arc is longer than the chord
    endcap = np.abs(z_outer) > Z_MAX - 10.0
    differ = (o2["tl_n"] != o["tl_n"]) | (o2["tl_alive"] != o["tl_alive"])
    assert not np.any(differ & ~endcap), np.flatnonzero(differ & ~endcap)[:10]
    ok = ~endcap & ~differ & (o["tl_n"] > 0)
    assert ok.sum() > 10000
    for c, name in ((1, "y"), (3, "sin(phi)"), (5, "q/pT")):
        np.testing.assert_array_equal(f2[ok, c], f1[ok, c], err_msg=name)
    shift = np.where(side_a[o["start"]], -dz, dz)
    np.testing.assert_allclose(f2[ok, 2] - f1[ok, 2], shift[ok], rtol=0, atol=TOL[mode], err_msg="z")
    np.testing.assert_allclose(f2[ok, 4], f1[ok, 4], rtol=0, atol=TOL[mode], err_msg="tan(lambda)")
    # the selected tracks away from the endcap keep their clusters
    keep = ~endcap[o["trk_t"]]
    l1, l2 = _track_lists(o), _track_lists(o2)
    t2 = {int(t): m for m, t in enumerate(o2["trk_t"])}
    for m in np.flatnonzero(keep):
        m2 = t2.get(int(o["trk_t"][m]))
        assert m2 is not None and l2[m2] == l1[m]
