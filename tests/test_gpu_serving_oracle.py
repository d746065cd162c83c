"""Serving results against the CPU oracle (Sec. 3.2: several events in
flight on one GPU; each must come out as if it had been tracked alone).

A mixed pool of requests -- pp events, min-bias events, a reduced central
event, a small continuous-readout time frame and one request that holds
three events -- is streamed through tpc_stream_submit/poll and
tpc_stream_poll_view with two batches in flight and a cluster limit that
makes batches mix large and small requests.  Every ticket's result is then
compared with the oracle run on that request alone:

* exact build against the FP32_EXACT oracle, bit for bit: the selected
  tracklets, request-relative event and sector, owned cluster counts,
  request-relative cluster positions, the 16 filter outputs and ndf; with
  the final refit, merge links and collision offsets switched on, the
  oracle's own chain (refit of its tracks, merging of its refits, offsets
  of its refits) gives the same bits as the streamed views;
* production build against the FP64 oracle: efficiency, clone and fake
  rates over the whole pool within 0.2 percentage points, and the
  parameters of tracks with identical cluster lists within 1e-4 relative +
  1e-3 absolute.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import qa  # noqa: E402
from gpu_util import XR  # noqa: E402
from paper_1712_09430_gb300 import synth as S  # noqa: E402
from paper_1712_09430_gb300.tracker import Tracker  # noqa: E402


class Req:
    def __init__(self, events):
        self.events = events
        if len(events) == 1:
            self.clusters, self.row_counts = events[0].clusters, events[0].row_counts
        else:
            self.clusters, self.row_counts = S.concat_events(events)
        self.n_events = len(events)
        self.labels = np.concatenate([np.where(e.label >= 0, e.label + i * 10_000_000, -1)
                                      for i, e in enumerate(events)])


@pytest.fixture(scope="module")
def pool():
    reqs = [Req([S.pp_event(seed=80 + i)]) for i in range(3)]
    reqs += [Req([S.min_bias_event(seed=1100 + i)]) for i in range(4)]
    reqs += [Req([S.central_event(seed=90, scale=0.1)])]
    reqs += [Req([S.time_frame(seed=91, n_coll=3, scale=0.2)])]
    reqs += [Req([S.pp_event(seed=92), S.min_bias_event(seed=1110), S.pp_event(seed=93)])]
    return reqs


def _stream(pool, exact, refit):
    """Each request twice, in a seeded random order, through the request
    loop; results taken alternately by poll and by poll_view.  Returns
    [(request index, Result)] and the loop's counters."""
    order = np.random.default_rng(7).permutation(np.repeat(np.arange(len(pool)), 2))
    biggest = max(r.clusters.shape[0] for r in pool)
    opts = dict(refit=1, merge=1, t0=1) if refit else {}
    got = []
    with Tracker(XR, exact_fp32=exact, **opts) as tr:
        # two batches in flight, up to 4 events each, and room for about one
        # and a half of the largest requests: large and small requests mix
        tr.stream_configure(arena_bytes=4 << 30, max_batch_events=4, max_inflight=2,
                            max_batch_clusters=int(biggest * 1.5))
        pending = {}
        k = 0

        def collect(block_s):
            t_end = time.time() + block_s
            while pending:
                for t in list(pending):
                    i, view = pending[t]
                    if view:
                        r = tr.poll_view(t, timeout_us=100)
                        if r is not None:
                            r = _copy(r)
                            tr.release(t)
                    else:
                        r = tr.poll(t, timeout_us=100)
                    if r is not None:
                        got.append((i, r))
                        del pending[t]
                if time.time() > t_end:
                    return

        for i in order:
            q = pool[i]
            t = tr.submit(q.clusters, q.row_counts, q.n_events)
            t_end = time.time() + 60
            while t is None:  # not admitted now: take results, then retry
                collect(0.001)
                t = tr.submit(q.clusters, q.row_counts, q.n_events)
                assert time.time() < t_end, "admission timed out"
            pending[t] = (int(i), k % 2 == 1)
            k += 1
        t_end = time.time() + 120
        while pending:
            collect(0.01)
            assert time.time() < t_end, "poll timed out"
        stats = tr.stream_stats()
    return got, stats


def _copy(r):
    """A view's arrays copied out before the ticket is released."""
    from paper_1712_09430_gb300.tracker import Result
    c = (lambda a: None if a is None else np.array(a, copy=True))
    return Result(c(r.tracks), c(r.hit_ids), c(r.fits), c(r.merges), c(r.t0s))


def _fit_matrix(f):
    return np.concatenate([f["x"][:, None], f["p"], f["cov"], f["chi2"][:, None],
                           f["ndf"][:, None], f["status"][:, None]], axis=1).astype(np.float64)


def _bits(a):
    return (np.asarray(a, np.float64).astype(np.float32) + np.float32(0)).view(np.uint32)


@pytest.fixture(scope="module")
def exact_stream(pool):
    return _stream(pool, exact=1, refit=True)


@pytest.fixture(scope="module")
def oracle_f32(pool):
    return [oracle.run(q.clusters, q.row_counts, q.n_events, 0.5, XR, mode="f32") for q in pool]


def test_stream_formed_mixed_batches(pool, exact_stream):
    got, st = exact_stream
    assert len(got) == 2 * len(pool)
    assert st["batches"] >= 2 and st["max_batch_events"] >= 2


def test_streamed_tracks_equal_fp32_oracle_bit_for_bit(pool, exact_stream, oracle_f32):
    got, _ = exact_stream
    for i, r in got:
        o = oracle_f32[i]
        t = r.tracks
        M = len(o["trk_t"])
        assert len(t) == M, (i, len(t), M)
        if M == 0:
            continue
        np.testing.assert_array_equal(t["tracklet"], o["trk_t"], err_msg=f"request {i}: tracklets")
        unit = o["tl_unit"][o["trk_t"]]
        np.testing.assert_array_equal(t["event"], unit // 36, err_msg=f"request {i}: event")
        np.testing.assert_array_equal(t["sector"], unit % 36, err_msg=f"request {i}: sector")
        np.testing.assert_array_equal(t["nhits"], o["trk_n"], err_msg=f"request {i}: owned counts")
        np.testing.assert_array_equal(t["hit_off"], o["trk_hit_off"][:-1], err_msg=f"request {i}: hit_off")
        np.testing.assert_array_equal(r.hit_ids, o["trk_hits"], err_msg=f"request {i}: clusters")
        f = o["tl_f"][o["trk_t"]]
        g = np.concatenate([t["x"][:, None], t["p"], t["cov_y"], t["cov_z"], t["chi2"][:, None]], axis=1)
        np.testing.assert_array_equal(g.view(np.uint32), _bits(f), err_msg=f"request {i}: filter outputs")
        np.testing.assert_array_equal(t["ndf"], 2 * o["tl_n"][o["trk_t"]] - 5, err_msg=f"request {i}: ndf")


def test_streamed_refit_merge_offsets_equal_oracle_chain(pool, exact_stream, oracle_f32):
    """The oracle's own Phase-II chain on its own tracks: refit (tpc_refit.c),
    merging of those refits, collision offsets of those refits."""
    got, _ = exact_stream
    fp = oracle.fit_params(0.5)
    n_links = n_coll = 0
    for i, r in got:
        o = oracle_f32[i]
        q = pool[i]
        M = len(o["trk_t"])
        if M == 0:
            continue
        fits = oracle.refit_tracks(o, q.clusters, 0.5, mode="f32", fp=fp)
        g = _fit_matrix(r.fits)
        np.testing.assert_array_equal(_bits(g[:, :22]), _bits(fits[:, :22]), err_msg=f"request {i}: refit")
        np.testing.assert_array_equal(g[:, 22:].astype(np.int64), fits[:, 22:].astype(np.int64),
                                      err_msg=f"request {i}: refit ndf/status")
        unit = o["tl_unit"][o["trk_t"]].astype(np.int32)
        x_last = q.clusters[o["trk_hits"][o["trk_hit_off"][1:] - 1], 0].astype(np.float64)
        nxt, chi = oracle.merge_tracks(unit, fits, x_last, fp, mode="f32")
        np.testing.assert_array_equal(r.merges["next"], nxt, err_msg=f"request {i}: merge links")
        np.testing.assert_array_equal(r.merges["chi2"].view(np.uint32), _bits(chi), err_msg=f"request {i}: merge chi2")
        t0 = oracle.t0_tracks(unit, fits, fp, mode="f32")
        np.testing.assert_array_equal(r.t0s["collision"], t0[:, 0].astype(np.int32),
                                      err_msg=f"request {i}: collisions")
        np.testing.assert_array_equal(r.t0s["u"].view(np.uint32), _bits(t0[:, 1]), err_msg=f"request {i}: u")
        np.testing.assert_array_equal(r.t0s["dz"].view(np.uint32), _bits(t0[:, 2]), err_msg=f"request {i}: dz")
        n_links += int((nxt >= 0).sum())
        n_coll += int((t0[:, 0] >= 0).sum())
    assert n_links > 0 and n_coll > 0


def test_streamed_production_vs_fp64_oracle(pool):
    got, _ = _stream(pool, exact=0, refit=False)
    o64 = [oracle.run(q.clusters, q.row_counts, q.n_events, 0.5, XR, mode="f64") for q in pool]
    # pool the requests (each streamed twice) into one QA sample
    parts_g, parts_o = [], []
    labels, rcs = [], []
    shift = 0
    lab_shift = 0
    for i, r in got:
        q, o = pool[i], o64[i]
        labels.append(np.where(q.labels >= 0, q.labels + lab_shift, -1))
        rcs.append(q.row_counts)
        parts_g.append((r.hit_off, r.hit_ids + shift))
        parts_o.append((o["trk_hit_off"], o["trk_hits"] + shift))
        shift += q.clusters.shape[0]
        lab_shift += 100_000_000
    lab = np.concatenate(labels)
    rc = np.concatenate(rcs)

    def join(parts):
        offs, hits, base = [np.zeros(1, np.int64)], [], 0
        for off, h in parts:
            offs.append(np.asarray(off[1:], np.int64) + base)
            hits.append(h)
            base += len(h)
        return np.concatenate(offs), np.concatenate(hits)
    qg = qa.qa(lab, rc, *join(parts_g))
    qo = qa.qa(lab, rc, *join(parts_o))
    assert qg["n_reconstructable"] > 1000
    for key in ("eff", "clone", "fake"):
        assert abs(qg[key] - qo[key]) <= 0.002, (key, qg[key], qo[key])
    n_cmp = n_all = 0
    for i, r in got:
        o = o64[i]
        want = {}
        for m, t in enumerate(o["trk_t"]):
            h = o["trk_hits"][o["trk_hit_off"][m]:o["trk_hit_off"][m + 1]]
            want[tuple(h.tolist())] = o["tl_f"][t][0:6]
        for m in range(len(r.tracks)):
            n_all += 1
            key = tuple(r.hits_of(m).tolist())
            if key not in want:
                continue
            t = r.tracks[m]
            got_p = np.array([t["x"], *t["p"]], np.float64)
            w = want[key]
            assert np.all(np.abs(got_p - w) <= 1e-3 + 1e-4 * np.abs(w)), (i, m, got_p, w)
            n_cmp += 1
    assert n_cmp >= 0.9 * n_all
