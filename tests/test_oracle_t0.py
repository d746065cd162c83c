"""Pins of the continuous-readout oracle (oracle/tpc_refit.c, readings
T01-T05): per-collision drift offsets estimated from the tracks, because in a
time frame a cluster's z is known only once its collision's time is (Run 3
conditions, Sec. 3.3, item 3).  Pinned against the generator's exact
crossings of shifted collisions, hand-built grouping cases, and the truth of
a generated time frame run through the whole oracle chain."""
import math

import numpy as np

import oracle
from paper_1712_09430_gb300 import synth as S

XR = S.row_x()
BZ = 0.5


def _fit_row(x, p, status=0):
    f = np.zeros(oracle.N_FIT)
    f[0] = x
    f[1:6] = p
    f[23] = status
    return f


def test_track_offset_is_the_collision_shift():
    """A primary's exact state at its innermost crossing with z shifted by
    sign(side) dz (the drift coordinate) steps back to the beam line with
    y = 0 and u = dz, on both sides; a secondary from a displaced vertex
    fails the |y(0)| cut."""
    rng = np.random.default_rng(41)
    tr = S.gen_tracks(rng, 400, 0, pt_mean=1.0)
    cr = S.crossings(tr, BZ)
    fits, units, want = [], [], []
    for m in range(len(tr)):
        sel = np.flatnonzero(cr["track"] == m)
        if len(sel) == 0:
            continue
        i = sel[np.argmin(cr["row"][sel])]
        sec = int(cr["sector"][i])
        sgn = 1.0 if sec < 18 else -1.0
        dz = rng.uniform(-100, 100)
        p = [cr["y"][i], cr["z"][i] + sgn * dz, cr["sphi"][i], tr.tanl[m], tr.q[m] / tr.pt[m]]
        fits.append(_fit_row(XR[cr["row"][i]], p))
        units.append(sec)
        want.append(dz)
    o = np.argsort(units, kind="stable")
    fits, units, want = np.array(fits)[o], np.array(units)[o], np.array(want)[o]
    out = oracle.t0_tracks(units, fits, oracle.fit_params(BZ), oracle.t0_params(n_min=1000))
    assert len(want) > 200
    err = np.abs(out[:, 1] - want)
    assert np.all(err < 1e-6), err.max()
    # a secondary: vertex 20 cm off the beam line in y
    tr2 = S.Tracks(np.array([0.0]), np.array([20.0]), np.array([0.0]), np.array([0.1]),
                   np.array([2.0]), np.array([0.3]), np.array([1.0]))
    cr2 = S.crossings(tr2, BZ)
    i = np.argmin(cr2["row"])
    f2 = _fit_row(XR[cr2["row"][i]], [cr2["y"][i], cr2["z"][i], cr2["sphi"][i], 0.3, 0.5])
    out2 = oracle.t0_tracks(np.array([cr2["sector"][i]]), f2[None], oracle.fit_params(BZ),
                            oracle.t0_params(n_min=1))
    assert out2[0, 0] == -1


def _beam_fits(us, sides_c=None):
    """States on the beam line (x = 0, y = 0): u = z on side A, -z on side C."""
    fits, units = [], []
    for k, u in enumerate(us):
        side_c = bool(sides_c[k]) if sides_c is not None else k % 2 == 1
        fits.append(_fit_row(0.0, [0.0, -u if side_c else u, 0.0, 0.0, 0.0]))
        units.append(21 if side_c else 3)
    units = np.array(units)
    o = np.argsort(units, kind="stable")
    return units[o], np.array(fits)[o], np.array(us)[o]


def test_peak_rule_and_means():
    fp = oracle.fit_params(BZ)
    tp = oracle.t0_params(n_min=3, window=8, radius=1.0)
    a = [10.0, 10.1, 10.2, 10.05]                # a collision
    b = [12.6, 12.7, 12.8]                       # 2.6 cm higher: its own peak (beyond W = 2 cm)
    c = [20.0, 20.1, 20.2, 20.3, 21.3, 21.4, 21.5]   # two groups 1.3 cm apart: one peak
    d = [40.0, 40.1]                             # too few
    units, fits, us = _beam_fits(a + b + c + d)
    out = oracle.t0_tracks(units, fits, fp, tp)
    got = {round(float(u), 4): (int(k), D) for u, (k, _, D) in zip(us, out)}
    assert got[10.0][0] == 0 and got[12.7][0] == 1 and got[20.1][0] == 2
    assert got[40.0][0] == -1 and got[40.1][0] == -1
    # the suppressed group's tracks join the peak only within r = 1 cm of its centre
    assert got[21.3][0] in (-1, 2)
    assert sum(v[0] == 2 for v in got.values()) >= 4
    assert abs(got[10.1][1] - np.float32(sum(a) / 4)) < 1e-6
    assert abs(got[12.8][1] - np.float32(12.7)) < 1e-6
    # equal counts on a plateau: the lowest bin is the peak, one collision
    units, fits, us = _beam_fits([30.0, 30.0, 30.0, 31.0, 31.0, 31.0])
    out = oracle.t0_tracks(units, fits, fp, tp)
    assert set(out[:, 0].astype(int)) == {0}
    # failed fits and off-beam tracks are not candidates
    f = np.array([_fit_row(0.0, [0.0, 5.0, 0, 0, 0]) for _ in range(3)])
    f[1, 23] = 1
    f[2, 1] = 1.5
    out = oracle.t0_tracks(np.zeros(3, np.int32), f, fp, oracle.t0_params(n_min=1))
    assert out[0, 0] == 0 and out[1, 0] == -1 and out[2, 0] == -1
    # another event numbers its collisions from 0
    f = np.array([_fit_row(0.0, [0.0, z, 0, 0, 0]) for z in (5.0, 5.1, 5.2, 8.0, 8.1, 8.2)])
    out = oracle.t0_tracks(np.array([0, 0, 0, 36, 36, 36]), f, fp, tp)
    assert list(out[:, 0]) == [0, 0, 0, 0, 0, 0]


def test_time_frame_collisions_recovered():
    """The whole oracle chain (tracking, refit, offsets) on a time frame of
    12 overlaid collisions: most collisions with enough tracks are found at
    their true drift offset, and assigned tracks come from that collision."""
    ev = S.time_frame(seed=7, n_coll=12, scale=0.3)
    o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR)
    fp = oracle.fit_params(ev.bz)
    fits = oracle.refit_tracks(o, ev.clusters, ev.bz, fp=fp)
    unit = o["tl_unit"][o["trk_t"]]
    out = oracle.t0_tracks(unit, fits, fp)
    coll = out[:, 0].astype(int)
    assert (coll >= 0).mean() > 0.3
    # truth collision of each track (majority label)
    lab = ev.label
    truth = np.full(len(coll), -1)
    for m in range(len(coll)):
        h = o["trk_hits"][o["trk_hit_off"][m]:o["trk_hit_off"][m + 1]]
        v, c = np.unique(lab[h], return_counts=True)
        if v[np.argmax(c)] >= 0:
            truth[m] = ev.track_coll[v[np.argmax(c)]]
    found = 0
    for k in np.unique(coll[coll >= 0]):
        sel = coll == k
        D = out[sel, 2][0]
        tc = np.bincount(truth[sel][truth[sel] >= 0]).argmax()
        found += 1
        assert abs(D - ev.coll_dz[tc]) < 0.3, (D, ev.coll_dz[tc])
        assert np.mean(truth[sel] == tc) > 0.9
    # every collision with many primaries reconstructed is found
    big = [c for c in range(len(ev.coll_dz)) if np.sum(truth == c) > 300]
    assert found >= len(big) >= 3


def test_assignment_tie_centre_and_range_edge():
    """T03/T04: bin centres are -z_max + (b + 1/2) w; a candidate exactly r
    from two collisions' centres joins the lower one; the histogram covers
    [-z_max, z_max), so candidates at u = z_max form no collision."""
    fp = oracle.fit_params(BZ)
    tp = oracle.t0_params(n_min=3, window=2, radius=1.0)
    a = [10.125] * 4                 # bin 1040, centre 10.125
    b = [12.125] * 4                 # bin 1048, centre 12.125: a second peak (8 bins > W = 2)
    units, fits, us = _beam_fits(a + b + [11.125])
    out = oracle.t0_tracks(units, fits, fp, tp)
    got = {float(u): int(k) for u, (k, _, _) in zip(us, out)}
    assert got[10.125] == 0 and got[12.125] == 1
    assert got[11.125] == 0          # 1.0 cm from both centres: the lower collision
    # the range is half-open
    units, fits, us = _beam_fits([250.0] * 4)
    out = oracle.t0_tracks(units, fits, fp, oracle.t0_params(n_min=3))
    assert np.all(out[:, 0] == -1)
    units, fits, us = _beam_fits([-250.0] * 4)
    out = oracle.t0_tracks(units, fits, fp, oracle.t0_params(n_min=3))
    assert np.all(out[:, 0] == 0)


def test_smoothing_spans_five_bins():
    """T03: counts and scores are taken over b-2..b+2 with weights 1 2 3 2 1.
    Three candidates in bin 1040 and two in bin 1042 (n_min = 5): only the
    five-bin sum reaches n_min at bin 1040, which is the peak (score 11 against
    10 at bin 1041), so with r = 0.3 cm the two candidates 0.5 cm above its
    centre join no collision."""
    fp = oracle.fit_params(BZ)
    tp = oracle.t0_params(n_min=5, radius=0.3)
    units, fits, us = _beam_fits([10.125] * 3 + [10.625] * 2)
    out = oracle.t0_tracks(units, fits, fp, tp)
    got = [(float(u), int(k)) for u, (k, _, _) in zip(us, out)]
    assert sorted(got) == [(10.125, 0)] * 3 + [(10.625, -1)] * 2
