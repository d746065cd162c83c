"""Track merging on the GPU (k_merge_*, through the C ABI) against the
merging oracle (oracle/tpc_refit.c): Sec. 2 Phase II step 3, segments linked
inside a sector across a gap and across sector borders by comparing their
refitted parameters with the covariances.

The oracle links the GPU's own refitted tracks, so the comparison isolates
the merging.  Exact mode against the FP32_EXACT oracle: identical links and
bit-identical link chi2.  Production mode against FP64: the same links for
all but a tiny fraction of near-threshold or near-tie pairs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import XR  # noqa: E402
from paper_1712_09430_gb300 import synth as S  # noqa: E402
from paper_1712_09430_gb300.tracker import Tracker  # noqa: E402


@pytest.fixture(scope="module")
def events():
    return {
        "c2": S.pp_event(),
        "c3s": S.central_event(seed=3, scale=0.1),
        "tf": S.time_frame(seed=4, n_coll=4, scale=0.3),
        "lowB": S.make_event(21, 300, 60, pt_mean=0.3, noise_frac=0.2, bz=0.2),
        "lowpt": S.make_event(22, 400, 0, pt_mean=0.25, noise_frac=0.05),
        "negB": S.make_event(24, 400, 0, pt_mean=0.25, noise_frac=0.05, bz=-0.5),  # reversed field
        "zeroB": S.make_event(25, 300, 60, pt_mean=0.5, noise_frac=0.1, bz=0.0),  # straight tracks
    }


def gpu_merge(cl, rc, n_events=1, bz=0.5, **params):
    with Tracker(XR, bz=bz, refit=1, merge=1, **params) as tr:
        return tr.track(cl, rc, n_events)


def fit_matrix(f):
    return np.concatenate([f["x"][:, None], f["p"], f["cov"], f["chi2"][:, None],
                           f["ndf"][:, None], f["status"][:, None]], axis=1).astype(np.float64)


def oracle_merge(r, clusters, bz, mode):
    t = r.tracks
    unit = t["event"].astype(np.int32) * 36 + t["sector"]
    last = np.array([r.hits_of(m)[-1] for m in range(len(t))], np.int64)
    x_last = clusters[last, 0].astype(np.float64)
    return oracle.merge_tracks(unit, fit_matrix(r.fits), x_last, oracle.fit_params(bz), mode=mode)


@pytest.mark.parametrize("name", ["c2", "c3s", "tf", "lowB", "lowpt", "negB", "zeroB"])
def test_merge_exact_parity(events, name):
    ev = events[name]
    r = gpu_merge(ev.clusters, ev.row_counts, bz=ev.bz, exact_fp32=1)
    nxt, chi = oracle_merge(r, ev.clusters, ev.bz, "f32")
    np.testing.assert_array_equal(r.merges["next"], nxt)
    np.testing.assert_array_equal(r.merges["chi2"].view(np.uint32),
                                  chi.astype(np.float32).view(np.uint32))
    if name in ("c3s", "lowpt", "tf", "negB", "zeroB"):
        assert (nxt >= 0).sum() > 0


def test_merge_exact_parity_tiny_lattice_events():
    """1000 tiny one-sector events in one call: links (none expected across
    these short patches) and their chi2 equal the oracle's."""
    cl, rc = S.tiny_lattice_events(1000, seed=13)
    r = gpu_merge(cl, rc, n_events=1000, exact_fp32=1)
    nxt, chi = oracle_merge(r, cl, 0.5, "f32")
    np.testing.assert_array_equal(r.merges["next"], nxt)
    np.testing.assert_array_equal(r.merges["chi2"].view(np.uint32),
                                  chi.astype(np.float32).view(np.uint32))


def test_merge_links_mostly_join_one_mc_track(events):
    """Quality (not parity): the segments a link joins mostly come from the
    same generated track, and a good share of tracks crossing a sector
    border get linked."""
    ev = events["lowpt"]
    r = gpu_merge(ev.clusters, ev.row_counts, exact_fp32=0)
    lab = ev.label

    def major(m):
        h = r.hits_of(m)
        v, c = np.unique(lab[h], return_counts=True)
        return v[np.argmax(c)]
    links = [(a, b) for a, b in enumerate(r.merges["next"]) if b >= 0]
    assert len(links) > 20
    same = np.mean([major(a) == major(b) and major(a) >= 0 for a, b in links])
    assert same > 0.95, same
    cross = [(a, b) for a, b in links if r.tracks["sector"][a] != r.tracks["sector"][b]]
    assert len(cross) > 10


def test_merge_production_vs_fp64(events):
    for name in ("c3s", "lowpt", "tf"):
        ev = events[name]
        r = gpu_merge(ev.clusters, ev.row_counts, bz=ev.bz, exact_fp32=0)
        nxt, chi = oracle_merge(r, ev.clusters, ev.bz, "f64")
        agree = np.mean(r.merges["next"] == nxt)
        assert agree > 0.995, (name, agree)
        both = (nxt >= 0) & (r.merges["next"] == nxt)
        assert np.all(np.abs(r.merges["chi2"][both] - chi[both]) <= 1e-3 * chi[both] + 1e-3)


@pytest.mark.parametrize("over", [dict(plain_per_sector=1), dict(plain_per_sector=2, n_queues=3),
                                  dict(use_graph=1)])
def test_merge_same_in_every_launch_form(events, over):
    ev = events["c3s"]
    a = gpu_merge(ev.clusters, ev.row_counts, exact_fp32=1)
    b = gpu_merge(ev.clusters, ev.row_counts, exact_fp32=1, **over)
    np.testing.assert_array_equal(a.merges.view(np.uint8), b.merges.view(np.uint8))


def test_merge_multi_event_batch_equals_alone(events):
    evs = [events["c2"], events["c3s"], events["lowpt"]]
    cl, rc = S.concat_events(evs)
    r = gpu_merge(cl, rc, len(evs), exact_fp32=1)
    base = 0
    for e_i, ev in enumerate(evs):
        a = gpu_merge(ev.clusters, ev.row_counts, exact_fp32=1)
        sel = np.flatnonzero(r.tracks["event"] == e_i)
        got = r.merges[sel].copy()
        got["next"] = np.where(got["next"] >= 0, got["next"] - base, -1)
        np.testing.assert_array_equal(got.view(np.uint8), a.merges.view(np.uint8))
        base += len(sel)


def test_merge_serving_equals_alone(events):
    pool = [events["c2"], events["c3s"], events["lowpt"], events["lowB"]]
    with Tracker(XR, refit=1, merge=1) as alone:
        ref = [alone.track(e.clusters, e.row_counts, 1) for e in pool]
    with Tracker(XR, refit=1, merge=1) as tr:
        tr.stream_configure(arena_bytes=2 << 30, max_batch_events=3, max_inflight=2)
        tickets = [tr.submit(e.clusters, e.row_counts, 1) for e in pool]
        got = {}
        while len(got) < len(tickets):
            for i, t in enumerate(tickets):
                if i not in got:
                    v = tr.poll_view(t, timeout_us=200)
                    if v is not None:
                        got[i] = v.merges.copy()
                        tr.release(t)
    for i, m in got.items():
        np.testing.assert_array_equal(m.view(np.uint8), ref[i].merges.view(np.uint8))


def test_merge_needs_refit():
    from paper_1712_09430_gb300.tracker import TrackerError
    with pytest.raises(TrackerError):
        Tracker(XR, refit=0, merge=1)


def test_merge_full_size_central_exact():
    """Two full central events (4.1 M clusters), exact build: the merging
    oracle on the GPU's refitted tracks gives the same links."""
    evs = [S.central_event(seed=3), S.central_event(seed=4)]
    cl, rc = S.concat_events(evs)
    r = gpu_merge(cl, rc, 2, exact_fp32=1)
    assert len(r.tracks) > 40000
    nxt, chi = oracle_merge(r, cl, 0.5, "f32")
    np.testing.assert_array_equal(r.merges["next"], nxt)
    np.testing.assert_array_equal(r.merges["chi2"].view(np.uint32), chi.astype(np.float32).view(np.uint32))
    assert (nxt >= 0).sum() > 100
