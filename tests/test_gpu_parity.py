"""GPU (CUDA, through the C ABI) against the CPU oracle.

Exact mode (kernels built with -fmad=false) against the FP32_EXACT oracle:
every stage bit-exact: raw and cleaned links, start hits, tracklet cluster
lists, tracklet filter states, selected tracks and their clusters.
Production mode against the FP64 oracle: efficiency, clone and fake rates
within 0.2 percentage points; parameters of tracks with identical cluster
lists within 1e-4 relative + 1e-3 absolute (cm for y and z).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import qa  # noqa: E402
from gpu_util import XR, assert_exact_equal, gpu_run, oracle_run  # noqa: E402
from paper_1712_09430_gb300 import capi, synth as S  # noqa: E402
from paper_1712_09430_gb300.tracker import Tracker, TrackerError  # noqa: E402


@pytest.fixture(scope="module")
def events():
    return {
        "c1": S.single_sector(),
        "c2": S.pp_event(),
        "c3s": S.central_event(seed=3, scale=0.1),
        "tf": S.time_frame(seed=4, n_coll=4, scale=0.3),
        "lowB": S.make_event(21, 300, 60, pt_mean=0.3, noise_frac=0.2, bz=0.2),
        "negB": S.make_event(23, 300, 60, pt_mean=0.4, noise_frac=0.1, bz=-0.5),  # reversed field
        "zeroB": S.make_event(25, 300, 60, pt_mean=0.5, noise_frac=0.1, bz=0.0),  # straight tracks
    }


@pytest.mark.parametrize("name", ["c1", "c2", "c3s", "tf", "lowB", "negB", "zeroB"])
def test_exact_parity_every_stage(events, name):
    ev = events[name]
    g = gpu_run(ev.clusters, ev.row_counts, 1, bz=ev.bz, exact_fp32=1)
    o = oracle_run(ev.clusters, ev.row_counts, 1, bz=ev.bz, mode="f32")
    assert len(o["trk_t"]) > 0
    assert_exact_equal(g, o)


def test_exact_parity_batch_with_an_empty_event(events):
    """An event without clusters between two others: its 36 units are empty
    in every stage, the schedule blocks and the selection skip them."""
    empty = np.zeros(36 * 159, np.int32)
    evs = [events["c2"], events["c3s"]]
    cl = np.concatenate([evs[0].clusters, evs[1].clusters])
    rc = np.concatenate([evs[0].row_counts, empty, evs[1].row_counts])
    g = gpu_run(cl, rc, 3, exact_fp32=1, use_graph=1)
    o = oracle_run(cl, rc, 3, mode="f32")
    assert_exact_equal(g, o)
    assert not np.any(g["tracks"]["event"] == 1)


def test_exact_parity_multi_event_batch(events):
    evs = [events["c2"], events["c3s"], events["c1"], S.pp_event(seed=9)]
    cl, rc = S.concat_events(evs)
    g = gpu_run(cl, rc, len(evs), exact_fp32=1)
    o = oracle_run(cl, rc, len(evs), mode="f32")
    assert_exact_equal(g, o)
    # each event alone gives the same tracks (units are independent)
    off_cl = 0
    for e_i, ev in enumerate(evs):
        ge = gpu_run(ev.clusters, ev.row_counts, 1, exact_fp32=1, dumps=False)
        gb = g["tracks"][g["tracks"]["event"] == e_i]
        assert len(gb) == len(ge["tracks"])
        hits_b = np.concatenate([g["hit_ids"][t["hit_off"]:t["hit_off"] + t["nhits"]] for t in gb]) \
            if len(gb) else np.zeros(0, np.int32)
        np.testing.assert_array_equal(hits_b - off_cl, ge["hit_ids"])
        for f in ("sector", "nhits", "ndf", "p", "cov_y", "cov_z", "chi2", "x"):
            np.testing.assert_array_equal(gb[f], ge["tracks"][f])
        off_cl += ev.n


@pytest.mark.parametrize("over", [dict(bin_target=0.5), dict(bin_target=8.0, threads_per_row=32),
                                  dict(bin_target=2.0, threads_per_row=256),
                                  dict(plain_per_sector=1), dict(use_graph=1),
                                  dict(plain_per_sector=2, n_queues=8),
                                  dict(plain_per_sector=2, n_queues=3, use_graph=1),
                                  dict(tracklets_per_warp=4), dict(schedule=1),
                                  dict(tracklets_per_warp=16, schedule=1), dict(schedule=2),
                                  dict(tracklets_per_warp=8, schedule=2),
                                  dict(lanes_per_hit=2), dict(lanes_per_hit=4, threads_per_row=256),
                                  dict(lanes_per_hit=8, threads_per_row=32, bin_target=8.0),
                                  dict(lanes_per_hit=4, plain_per_sector=2, n_queues=4)])
def test_execution_params_do_not_change_results(events, over):
    ev = events["c3s"]
    base = gpu_run(ev.clusters, ev.row_counts, 1, exact_fp32=1)
    g = gpu_run(ev.clusters, ev.row_counts, 1, exact_fp32=1, **over)
    for k in ("up_raw", "dn_raw", "start", "tl_n", "tl_hits"):
        np.testing.assert_array_equal(g[k], base[k], err_msg=k)
    np.testing.assert_array_equal(g["tl_f"].view(np.uint32), base["tl_f"].view(np.uint32))
    np.testing.assert_array_equal(g["hit_ids"], base["hit_ids"])


def test_neighbour_forms_agree_in_production_build(events):
    """The production build too gives the same links and tracks whichever
    number of lanes shares a hit in the neighbour finder (the pair residual
    rounds alike in every form)."""
    ev = events["c3s"]
    base = gpu_run(ev.clusters, ev.row_counts, 1, exact_fp32=0)
    for lh in (2, 4, 8):
        g = gpu_run(ev.clusters, ev.row_counts, 1, exact_fp32=0, lanes_per_hit=lh)
        for k in ("up_raw", "dn_raw", "up", "dn", "start"):
            np.testing.assert_array_equal(g[k], base[k], err_msg=f"{k} lanes_per_hit={lh}")
        np.testing.assert_array_equal(g["hit_ids"], base["hit_ids"])


def test_graph_replay_repeats(events):
    ev = events["c3s"]
    with Tracker(XR, bz=ev.bz, exact_fp32=1, use_graph=1) as tr:
        r1 = tr.track(ev.clusters, ev.row_counts, 1)
        r2 = tr.track(ev.clusters, ev.row_counts, 1)
        r3 = tr.track(ev.clusters, ev.row_counts, 1)
    for r in (r2, r3):
        np.testing.assert_array_equal(r.hit_ids, r1.hit_ids)
        np.testing.assert_array_equal(r.tracks.view(np.uint8), r1.tracks.view(np.uint8))


def _labels_batch(evs):
    return np.concatenate([np.where(e.label >= 0, e.label + i * 10_000_000, -1)
                           for i, e in enumerate(evs)])


def test_production_vs_fp64(events):
    evs = [events["c3s"], events["c2"], events["tf"]]
    cl, rc = S.concat_events(evs)
    g = gpu_run(cl, rc, len(evs), exact_fp32=0)
    o = oracle_run(cl, rc, len(evs), mode="f64")
    lab = _labels_batch(evs)
    qg = qa.qa(lab, rc, g["hit_off"], g["hit_ids"])
    qo = qa.qa(lab, rc, o["trk_hit_off"], o["trk_hits"])
    for key in ("eff", "clone", "fake"):
        assert abs(qg[key] - qo[key]) <= 0.002, (key, qg[key], qo[key])
    # parameters of tracks found with identical cluster lists
    ok = {}
    for m, t in enumerate(o["trk_t"]):
        h = o["trk_hits"][o["trk_hit_off"][m]:o["trk_hit_off"][m + 1]]
        ok[(int(o["start"][t]), tuple(h.tolist()))] = o["tl_f"][t]
    n_cmp = 0
    gst = g["start"]
    for m, tr in enumerate(g["tracks"]):
        h = g["hit_ids"][tr["hit_off"]:tr["hit_off"] + tr["nhits"]]
        key = (int(gst[tr["tracklet"]]), tuple(h.tolist()))
        if key not in ok:
            continue
        f = ok[key]
        got = np.array([tr["x"], *tr["p"]], np.float64)
        want = f[0:6]
        tol = 1e-3 + 1e-4 * np.abs(want)
        assert np.all(np.abs(got - want) <= tol), (got, want)
        n_cmp += 1
    assert n_cmp >= 0.9 * len(g["tracks"])


def test_full_size_bench_configuration_sampled_vs_fp64():
    """The configuration the benchmark times: eight full central events in one
    call (16.4 M clusters), production build, graph replay, the default
    (block) schedule.  The FP64 oracle tracks a sample of 24 of the 288
    (event, sector) units, each unit as an event of its own (units are
    independent); the GPU batch's tracks of those units reach the oracle's
    QA rates within 0.2 pp, and tracks with identical cluster lists agree in
    their parameters within 1e-4 relative + 1e-3 absolute."""
    evs = [S.central_event(seed=3 + i) for i in range(8)]
    cl, rc = S.concat_events(evs)
    lab = _labels_batch(evs)
    with Tracker(XR, use_graph=1, exact_fp32=0) as tr:
        tr.track(cl, rc, 8)
        r = tr.track(cl, rc, 8)   # a graph replay
        gstart = tr.dump(capi.TPC_DUMP_STARTS)
    units = np.sort(np.random.default_rng(11).choice(8 * 36, 24, replace=False))
    ucnt = rc.reshape(-1, 159)
    uoff = np.r_[0, np.cumsum(ucnt.sum(1))]
    # the sample as a batch of one-unit events
    parts, rcs, labs, base = [], [], [], {}
    pos = 0
    for k, u in enumerate(units):
        parts.append(cl[uoff[u]:uoff[u + 1]])
        labs.append(np.where(lab[uoff[u]:uoff[u + 1]] >= 0, lab[uoff[u]:uoff[u + 1]] + k * 10_000_000, -1))
        r1 = np.zeros(36 * 159, np.int32)
        r1[(u % 36) * 159:(u % 36 + 1) * 159] = ucnt[u]
        rcs.append(r1)
        base[int(u)] = (k, pos - uoff[u])   # sample event, position shift
        pos += len(parts[-1])
    cl_s, rc_s, lab_s = np.concatenate(parts), np.concatenate(rcs), np.concatenate(labs)
    o = oracle_run(cl_s, rc_s, len(units), mode="f64")
    # the GPU tracks of the sampled units, in the sample's numbering
    sel = [m for m, t in enumerate(r.tracks) if int(t["event"]) * 36 + int(t["sector"]) in base]
    g_off, g_hits, g_keys = [0], [], []
    for m in sel:
        t = r.tracks[m]
        _, shift = base[int(t["event"]) * 36 + int(t["sector"])]
        h = r.hits_of(m) + shift
        g_hits.append(h)
        g_off.append(g_off[-1] + len(h))
        g_keys.append((int(gstart[t["tracklet"]]) + shift, tuple(h.tolist())))
    g_hits = np.concatenate(g_hits)
    assert len(sel) > 2000
    qg = qa.qa(lab_s, rc_s, np.array(g_off), g_hits)
    qo = qa.qa(lab_s, rc_s, o["trk_hit_off"], o["trk_hits"])
    for key in ("eff", "clone", "fake"):
        assert abs(qg[key] - qo[key]) <= 0.002, (key, qg[key], qo[key])
    want = {}
    for m, t in enumerate(o["trk_t"]):
        h = o["trk_hits"][o["trk_hit_off"][m]:o["trk_hit_off"][m + 1]]
        want[(int(o["start"][t]), tuple(h.tolist()))] = o["tl_f"][t][0:6]
    n_cmp = 0
    for m, key in zip(sel, g_keys):
        if key not in want:
            continue
        t = r.tracks[m]
        got = np.array([t["x"], *t["p"]], np.float64)
        assert np.all(np.abs(got - want[key]) <= 1e-3 + 1e-4 * np.abs(want[key])), (got, want[key])
        n_cmp += 1
    assert n_cmp >= 0.9 * len(sel)


# ------------------------------------------------------------------ edges

def test_tiny_lattice_events_exact():
    """1000 tiny seeded events in one call (a patch of 3-30 rows in a random
    sector, up to 50 clusters a row on a 0.05 cm lattice: duplicate positions
    and exact distance ties are common): every stage equals the brute-force
    oracle bit for bit, through the search grid at a fine and a coarse bin
    size."""
    cl, rc = S.tiny_lattice_events(1000, seed=12)
    o = oracle_run(cl, rc, 1000, mode="f32")
    assert len(o["trk_t"]) > 0
    # lanes_per_hit > 1: the warp-cooperative neighbour search, whose windows
    # here often hold more down candidates than its per-group list (rescan)
    for bt, lh in ((0.25, 1), (4.0, 1), (0.25, 4), (4.0, 8), (0.25, 2)):
        g = gpu_run(cl, rc, 1000, exact_fp32=1, bin_target=bt, lanes_per_hit=lh)
        assert_exact_equal(g, o)


def test_empty_inputs():
    rc = np.zeros(36 * 159, np.int32)
    g = gpu_run(np.zeros((0, 4), np.float32), rc, 1, dumps=False)
    assert len(g["tracks"]) == 0
    g = gpu_run(np.zeros((0, 4), np.float32), np.zeros(0, np.int32), 0, dumps=False)
    assert len(g["tracks"]) == 0


def test_ragged_sparse_rows():
    # a handful of clusters on scattered rows, single-cluster rows, no tracks
    rng = np.random.default_rng(3)
    rc = np.zeros(36 * 159, np.int32)
    idx = rng.choice(36 * 159, 50, replace=False)
    rc[idx] = rng.integers(1, 3, 50)
    n = int(rc.sum())
    rows = np.repeat(np.arange(36 * 159), rc) % 159
    secs = np.repeat(np.arange(36 * 159), rc) // 159
    cl = np.zeros((n, 4), np.float32)
    cl[:, 0] = XR[rows]
    cl[:, 1] = rng.uniform(-5, 5, n)
    cl[:, 2] = np.where(secs < 18, 1, -1) * rng.uniform(0, 250, n)
    cl.view(np.uint32)[:, 3] = np.arange(n)
    g = gpu_run(cl, rc, 1, exact_fp32=1)
    o = oracle_run(cl, rc, 1, mode="f32")
    assert_exact_equal(g, o)


def test_dense_row_at_limit():
    # one row at the maximum cluster count and its neighbours dense too
    rng = np.random.default_rng(4)
    rc = np.zeros(36 * 159, np.int32)
    rc[80:83] = [2000, capi.TPC_MAX_ROW_CLUSTERS, 2000]
    n = int(rc.sum())
    rows = np.repeat(np.arange(36 * 159), rc) % 159
    cl = np.zeros((n, 4), np.float32)
    cl[:, 0] = XR[rows]
    cl[:, 1] = rng.uniform(-25, 25, n)
    cl[:, 2] = rng.uniform(0, 250, n)
    cl.view(np.uint32)[:, 3] = rng.permutation(n)
    g = gpu_run(cl, rc, 1, exact_fp32=1)
    o = oracle_run(cl, rc, 1, mode="f32")
    assert_exact_equal(g, o)


def _uniform_rows(unit_rows, per_row, seed, n_tracks=40):
    """per_row clusters on each of the first n rows of each unit: n_tracks
    straight tracks through those rows, the rest uniform noise."""
    rng = np.random.default_rng(seed)
    rc = np.zeros(36 * 159, np.int32)
    for u, n_rows in unit_rows.items():
        rc[u * 159:u * 159 + n_rows] = per_row
    n = int(rc.sum())
    rr = np.repeat(np.arange(36 * 159), rc)
    rows, secs = rr % 159, rr // 159
    cl = np.zeros((n, 4), np.float32)
    cl[:, 0] = XR[rows]
    half = XR[rows] * np.tan(np.radians(10.0))
    cl[:, 1] = rng.uniform(-1, 1, n) * half
    cl[:, 2] = np.where(secs < 18, 1, -1) * rng.uniform(0, 250, n)
    # the first n_tracks clusters of every row lie on straight tracks
    first = np.r_[0, np.cumsum(rc)[:-1]]
    for u in unit_rows:
        sgn = 1.0 if u < 18 else -1.0
        y0 = rng.uniform(-10, 10, n_tracks)
        ty = rng.uniform(-0.05, 0.05, n_tracks)
        z0 = rng.uniform(20, 230, n_tracks)
        tz = rng.uniform(-0.1, 0.1, n_tracks)
        for r in range(unit_rows[u]):
            i0 = first[u * 159 + r]
            dx = XR[r] - XR[0]
            cl[i0:i0 + n_tracks, 1] = y0 + ty * dx
            cl[i0:i0 + n_tracks, 2] = sgn * (z0 + tz * dx)
    cl.view(np.uint32)[:, 3] = rng.permutation(n)
    return cl, rc


def test_graph_not_replayed_for_a_larger_unit():
    """Two batches alike in cluster count, rows and row maxima whose largest
    (event, sector) unit differs: the second must not replay the first's
    graph, whose ownership launch is sized for the smaller unit."""
    a = _uniform_rows({0: 10, 1: 10}, 1000, 11)
    b = _uniform_rows({0: 20}, 1000, 12)
    assert len(a[0]) == len(b[0])
    with Tracker(XR, use_graph=1, exact_fp32=1) as tr:
        tr.track(*a, 1)
        got = tr.track(*b, 1)
    with Tracker(XR, use_graph=0, exact_fp32=1) as tr:
        want = tr.track(*b, 1)
    assert len(want.tracks) > 0
    np.testing.assert_array_equal(got.tracks.view(np.uint8), want.tracks.view(np.uint8))
    np.testing.assert_array_equal(got.hit_ids, want.hit_ids)


def test_invalid_inputs_are_rejected(events):
    ev = events["c2"]
    with Tracker(XR, bz=ev.bz) as tr:
        bad = ev.clusters.copy()
        bad[17, 1] = np.nan
        with pytest.raises(TrackerError) as e:
            tr.track(bad, ev.row_counts, 1)
        assert e.value.code == capi.TPC_ERR_INVALID
        bad = ev.clusters.copy()
        bad[5, 0] += 0.5
        with pytest.raises(TrackerError) as e:
            tr.track(bad, ev.row_counts, 1)
        assert e.value.code == capi.TPC_ERR_INVALID
        rc = ev.row_counts.copy()
        rc[0] = capi.TPC_MAX_ROW_CLUSTERS + 1
        with pytest.raises(TrackerError) as e:
            tr.track(np.zeros((int(rc.sum()), 4), np.float32), rc, 1)
        assert e.value.code == capi.TPC_ERR_INVALID
        rc = ev.row_counts.copy()
        rc[3] = -1
        with pytest.raises(TrackerError):
            tr.track(ev.clusters, rc, 1)
        # the tracker is still usable
        r = tr.track(ev.clusters, ev.row_counts, 1)
        assert len(r.tracks) > 0


def test_output_truncation_and_fetch(events):
    ev = events["c3s"]
    with Tracker(XR, bz=ev.bz) as tr:
        full = tr.track(ev.clusters, ev.row_counts, 1)
        with pytest.raises(TrackerError) as e:
            tr.track(ev.clusters, ev.row_counts, 1, cap_tracks=5, cap_hits=50)
        assert e.value.code == capi.TPC_ERR_OUTPUT_TRUNCATED
        # default path: short estimate, then fetch the rest without recompute
        tr._est_tracks, tr._est_hits = 3, 10
        r = tr.track(ev.clusters, ev.row_counts, 1)
        np.testing.assert_array_equal(r.hit_ids, full.hit_ids)


def test_device_input_equals_host_input(events):
    ev = events["c3s"]
    dev = torch.from_numpy(ev.clusters).cuda()
    with Tracker(XR, bz=ev.bz) as tr:
        a = tr.track(ev.clusters, ev.row_counts, 1)
        b = tr.track(dev, ev.row_counts, 1)
    np.testing.assert_array_equal(a.hit_ids, b.hit_ids)
    np.testing.assert_array_equal(a.tracks.view(np.uint8), b.tracks.view(np.uint8))


def test_full_size_central_batch_exact():
    """The benchmark's workload size (full central events, batched launch,
    graph replay) against the FP32 oracle, every stage."""
    evs = [S.central_event(seed=3 + i) for i in range(2)]
    cl, rc = S.concat_events(evs)
    o = oracle_run(cl, rc, len(evs), mode="f32")
    for lh in (1, 4):  # one thread per hit, and four lanes sharing a hit
        g = gpu_run(cl, rc, len(evs), exact_fp32=1, use_graph=1, lanes_per_hit=lh)
        assert_exact_equal(g, o)


def test_block_schedule_full_size():
    """Schedule 2 on two full central events: blocks of about 2 M clusters
    (37 and 35 of the 72 units, the last one ragged) give the same tracks as
    the canonical order."""
    evs = [S.central_event(seed=3 + i) for i in range(2)]
    cl, rc = S.concat_events(evs)
    with Tracker(XR, exact_fp32=1, use_graph=1, schedule=0) as tr:
        a = tr.track(cl, rc, 2)
    with Tracker(XR, exact_fp32=1, use_graph=1, schedule=2) as tr:
        b = tr.track(cl, rc, 2)
    assert len(a.tracks) > 40000
    np.testing.assert_array_equal(a.tracks.view(np.uint8), b.tracks.view(np.uint8))
    np.testing.assert_array_equal(a.hit_ids, b.hit_ids)


def test_full_size_time_frame_exact():
    """The full 50-collision continuous-readout time frame (5.5 M clusters as
    one event; rows of up to ~1,500 clusters, hundreds of start hits in a
    row) against the FP32 oracle, every stage, batched launch with graph
    replay."""
    ev = S.time_frame(seed=4)
    assert int(ev.row_counts.max()) > 1000
    o = oracle_run(ev.clusters, ev.row_counts, 1, mode="f32")
    for lh in (1, 8):
        g = gpu_run(ev.clusters, ev.row_counts, 1, exact_fp32=1, use_graph=1, lanes_per_hit=lh)
        assert_exact_equal(g, o)


def test_work_counts_only_on_request(events):
    """The constructor's work counts (the byte model of the roofline) are
    compiled in only with params.count_work = 1; counting does not change
    the results, and the counts are consistent with the tracklets."""
    ev = events["c3s"]
    with Tracker(XR, exact_fp32=1, use_graph=1) as tr:
        a = tr.track(ev.clusters, ev.row_counts, 1)
        with pytest.raises(TrackerError):
            tr.dump(capi.TPC_DUMP_TRACKLET_WORK)
        tr.set_params(count_work=1)
        b = tr.track(ev.clusters, ev.row_counts, 1)
        w = tr.dump(capi.TPC_DUMP_TRACKLET_WORK)
        n = tr.dump(capi.TPC_DUMP_TRACKLET_N)[0]
    np.testing.assert_array_equal(a.tracks.view(np.uint8), b.tracks.view(np.uint8))
    np.testing.assert_array_equal(a.hit_ids, b.hit_ids)
    steps, bin_rows, cand, chain = w
    assert len(steps) == len(n) > 0
    assert np.all(steps >= n) and np.all(bin_rows >= steps) and np.all(chain >= 3)
    assert cand.sum() >= n.sum()


def test_autotune_keeps_results_and_caches(events, tmp_path):
    from paper_1712_09430_gb300 import autotune
    ev = events["c3s"]
    with Tracker(XR, bz=ev.bz, exact_fp32=1, bin_target=4.0, threads_per_row=32) as tr:
        before = tr.track(ev.clusters, ev.row_counts, 1)
        cache = str(tmp_path / "tune.json")
        fields, ms = autotune.tune(tr, ev.clusters, ev.row_counts, 1, reps=2, cache_path=cache)
        assert ms > 0 and set(fields) == set(autotune.FIELDS)
        after = tr.track(ev.clusters, ev.row_counts, 1)
        np.testing.assert_array_equal(after.tracks.view(np.uint8), before.tracks.view(np.uint8))
        np.testing.assert_array_equal(after.hit_ids, before.hit_ids)
    with Tracker(XR, bz=ev.bz, exact_fp32=1) as tr2:   # a cached choice applies without timing
        f2, _ = autotune.tune(tr2, ev.clusters, ev.row_counts, 1, cache_path=cache)
        assert f2 == fields and tr2.params.bin_target == fields["bin_target"]


def test_time_frame_uneven_slices_exact():
    """Continuous-readout time frame cut into uneven slices (different
    numbers of collisions per slice), all slices in one call."""
    tf = [S.time_frame(seed=70 + i, n_coll=n, scale=0.5) for i, n in enumerate((2, 5, 9))]
    cl, rc = S.concat_events(tf)
    g = gpu_run(cl, rc, len(tf), exact_fp32=1, use_graph=1)
    o = oracle_run(cl, rc, len(tf), mode="f32")
    assert_exact_equal(g, o)


def test_order_inside_rows_and_repeat_calls_do_not_change_results(events):
    """Clusters may come in any order inside a row (ties break by id), and
    the dynamic work distribution never shows in the output."""
    ev = events["c3s"]
    rng = np.random.default_rng(17)
    perm = np.arange(ev.n)
    off = np.concatenate([[0], np.cumsum(ev.row_counts)])
    for a, b in zip(off[:-1], off[1:]):
        if b - a > 1:
            perm[a:b] = a + rng.permutation(b - a)
    shuffled = ev.clusters[perm]
    with Tracker(XR, bz=ev.bz) as tr:
        r1 = tr.track(ev.clusters, ev.row_counts, 1)
        r2 = tr.track(ev.clusters, ev.row_counts, 1)
        r3 = tr.track(shuffled, ev.row_counts, 1)
    np.testing.assert_array_equal(r1.tracks.view(np.uint8), r2.tracks.view(np.uint8))
    np.testing.assert_array_equal(r1.hit_ids, r2.hit_ids)
    # same tracks; hit ids refer to positions, so map the shuffled ones back
    np.testing.assert_array_equal(r3.tracks.view(np.uint8), r1.tracks.view(np.uint8))
    np.testing.assert_array_equal(perm[r3.hit_ids], r1.hit_ids)
