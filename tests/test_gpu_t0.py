"""Continuous readout on the GPU (k_t0_*, through the C ABI) against the
oracle (oracle/tpc_refit.c, readings T01-T05): per-collision drift offsets of
a time frame estimated from its refitted tracks (Sec. 3.3, Run 3
conditions).  The oracle works on the GPU's own refitted tracks, so the
comparison isolates the offset estimation.  Exact mode: identical
collisions and bit-identical u and offsets.  Production mode against FP64:
the same collisions for all but near-boundary estimates."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import XR  # noqa: E402
from paper_1712_09430_gb300 import synth as S  # noqa: E402
from paper_1712_09430_gb300.tracker import Tracker, TrackerError  # noqa: E402


@pytest.fixture(scope="module")
def frames():
    return {
        "tf12": S.time_frame(seed=7, n_coll=12, scale=0.3),
        "tf4": S.time_frame(seed=4, n_coll=4, scale=0.3),
        "tf30": S.time_frame(seed=9, n_coll=30, scale=0.2),
    }


def gpu_t0(cl, rc, n_events=1, **params):
    with Tracker(XR, refit=1, t0=1, **params) as tr:
        return tr.track(cl, rc, n_events)


def fit_matrix(f):
    return np.concatenate([f["x"][:, None], f["p"], f["cov"], f["chi2"][:, None],
                           f["ndf"][:, None], f["status"][:, None]], axis=1).astype(np.float64)


def oracle_t0(r, mode):
    unit = r.tracks["event"].astype(np.int32) * 36 + r.tracks["sector"]
    return oracle.t0_tracks(unit, fit_matrix(r.fits), oracle.fit_params(0.5), mode=mode)


@pytest.mark.parametrize("name", ["tf12", "tf4", "tf30"])
def test_t0_exact_parity(frames, name):
    ev = frames[name]
    r = gpu_t0(ev.clusters, ev.row_counts, exact_fp32=1)
    o = oracle_t0(r, "f32")
    np.testing.assert_array_equal(r.t0s["collision"], o[:, 0].astype(np.int32))
    np.testing.assert_array_equal(r.t0s["u"].view(np.uint32), o[:, 1].astype(np.float32).view(np.uint32))
    np.testing.assert_array_equal(r.t0s["dz"].view(np.uint32), o[:, 2].astype(np.float32).view(np.uint32))
    assert (r.t0s["collision"] >= 0).sum() > 100


def test_t0_finds_the_collisions(frames):
    """Quality (not parity): every collision found sits at a true drift
    offset (within 0.3 cm), and its tracks come from that collision."""
    ev = frames["tf12"]
    r = gpu_t0(ev.clusters, ev.row_counts, exact_fp32=0)
    coll = r.t0s["collision"]
    lab = ev.label
    truth = np.full(len(coll), -1)
    for m in range(len(coll)):
        v, c = np.unique(lab[r.hits_of(m)], return_counts=True)
        if v[np.argmax(c)] >= 0:
            truth[m] = ev.track_coll[v[np.argmax(c)]]
    ks = np.unique(coll[coll >= 0])
    assert len(ks) >= 3
    for k in ks:
        sel = coll == k
        tc = np.bincount(truth[sel][truth[sel] >= 0]).argmax()
        assert abs(r.t0s["dz"][sel][0] - ev.coll_dz[tc]) < 0.3
        assert np.mean(truth[sel] == tc) > 0.9


def test_t0_production_vs_fp64(frames):
    for name in ("tf12", "tf30"):
        ev = frames[name]
        r = gpu_t0(ev.clusters, ev.row_counts, exact_fp32=0)
        o = oracle_t0(r, "f64")
        agree = np.mean(r.t0s["collision"] == o[:, 0])
        assert agree > 0.995, (name, agree)
        both = (o[:, 0] >= 0) & (r.t0s["collision"] == o[:, 0])
        assert np.all(np.abs(r.t0s["dz"][both] - o[both, 2]) < 1e-3)
        cand = o[:, 1] != 0
        assert np.all(np.abs(r.t0s["u"][cand] - o[cand, 1]) < 1e-3 + 1e-5 * np.abs(o[cand, 1]))


def test_t0_batch_of_frames_equals_alone(frames):
    evs = [frames["tf4"], frames["tf12"]]
    cl, rc = S.concat_events(evs)
    r = gpu_t0(cl, rc, len(evs), exact_fp32=1)
    for e_i, ev in enumerate(evs):
        a = gpu_t0(ev.clusters, ev.row_counts, exact_fp32=1)
        np.testing.assert_array_equal(r.t0s[r.tracks["event"] == e_i].view(np.uint8), a.t0s.view(np.uint8))


@pytest.mark.parametrize("over", [dict(plain_per_sector=1), dict(use_graph=1), dict(merge=1)])
def test_t0_same_in_every_launch_form(frames, over):
    ev = frames["tf4"]
    a = gpu_t0(ev.clusters, ev.row_counts, exact_fp32=1)
    b = gpu_t0(ev.clusters, ev.row_counts, exact_fp32=1, **over)
    np.testing.assert_array_equal(a.t0s.view(np.uint8), b.t0s.view(np.uint8))


def test_t0_serving_equals_alone(frames):
    pool = [frames["tf4"], frames["tf12"], frames["tf30"]]
    with Tracker(XR, refit=1, t0=1) as alone:
        ref = [alone.track(e.clusters, e.row_counts, 1) for e in pool]
    with Tracker(XR, refit=1, t0=1) as tr:
        tr.stream_configure(arena_bytes=4 << 30, max_batch_events=2, max_inflight=2)
        tickets = [tr.submit(e.clusters, e.row_counts, 1) for e in pool]
        got = {}
        while len(got) < len(tickets):
            for i, t in enumerate(tickets):
                if i not in got:
                    res = tr.poll(t, timeout_us=200)
                    if res is not None:
                        got[i] = res
    for i, res in got.items():
        np.testing.assert_array_equal(res.t0s.view(np.uint8), ref[i].t0s.view(np.uint8))


def test_t0_needs_refit():
    with pytest.raises(TrackerError):
        Tracker(XR, refit=0, t0=1)


def test_t0_full_size_time_frame_exact():
    """The full 50-collision time frame (5.5 M clusters) in the exact build:
    the oracle's collision offsets on the GPU's refitted tracks agree bit for
    bit."""
    ev = S.time_frame(seed=4)
    r = gpu_t0(ev.clusters, ev.row_counts, exact_fp32=1)
    o = oracle_t0(r, "f32")
    np.testing.assert_array_equal(r.t0s["collision"], o[:, 0].astype(np.int32))
    np.testing.assert_array_equal(r.t0s["dz"].view(np.uint32), o[:, 2].astype(np.float32).view(np.uint32))
    assert len(np.unique(r.t0s["collision"][r.t0s["collision"] >= 0])) >= 20
