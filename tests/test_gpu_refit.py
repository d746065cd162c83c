"""Final track fit on the GPU (k_refit, through the C ABI) against the refit
oracle (oracle/tpc_refit.c): the full Kalman filter refit of Sec. 2 ("Track
fit", Table 1 row 4) with the polynomial field.

The oracle refits the GPU's own tracks (start state, cluster lists, input
clusters), so the comparison isolates the refit.  Exact mode (-fmad=false)
against the FP32_EXACT oracle: bit-exact (signed zeros normalised).
Production mode against the FP64 oracle: parameters within 1e-4 relative +
1e-3 absolute (cm for y and z, else units of the parameter); covariance
diagonal within 1 %, chi2 within 1e-3 relative."""
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

FIELD = (2e-5, -4e-8, -8e-8, 1e-10, 1e-13)
FIELD32 = tuple(float(np.float32(b)) for b in FIELD)  # the values the GPU sees


@pytest.fixture(scope="module")
def events():
    return {
        "c1": S.single_sector(),
        "c2": S.pp_event(),
        "c3s": S.central_event(seed=3, scale=0.1),
        "tf": S.time_frame(seed=4, n_coll=4, scale=0.3),
        "lowB": S.make_event(21, 300, 60, pt_mean=0.3, noise_frac=0.2, bz=0.2),
        "negB": S.make_event(23, 300, 60, pt_mean=0.4, noise_frac=0.1, bz=-0.5),
        "zeroB": S.make_event(25, 300, 60, pt_mean=0.5, noise_frac=0.1, bz=0.0),  # straight tracks
    }


def gpu_fits(ev_cl, ev_rc, n_events=1, bz=0.5, **params):
    with Tracker(XR, bz=bz, refit=1, **params) as tr:
        r = tr.track(ev_cl, ev_rc, n_events)
        ms = tr.stage_times()
    return r, ms


def oracle_fits(r, clusters, bz, field=None, mode="f32", tracks=None, hits=None):
    """The oracle refit of the GPU's tracks (all of r, or the given tracks
    with their concatenated cluster lists)."""
    t = r.tracks if tracks is None else tracks
    h = r.hit_ids if hits is None else hits
    st6 = np.concatenate([t["x"][:, None], t["p"]], axis=1).astype(np.float64)
    off = np.zeros(len(t) + 1, np.int64)
    off[1:] = np.cumsum(t["nhits"])
    if tracks is None:
        assert np.array_equal(off[:-1], t["hit_off"])
    fp = oracle.fit_params(bz, field=field)
    return oracle.refit_lists(st6, off, h, clusters, fp, mode=mode)


def fit_matrix(f):
    """Structured fits -> float64 [M, 24] in the oracle's layout."""
    return np.concatenate([f["x"][:, None], f["p"], f["cov"], f["chi2"][:, None],
                           f["ndf"][:, None], f["status"][:, None]], axis=1).astype(np.float64)


def assert_bits_equal(g, o):
    a = (g[:, :22].astype(np.float32) + np.float32(0)).view(np.uint32)
    b = (o[:, :22].astype(np.float32) + np.float32(0)).view(np.uint32)
    bad = np.argwhere(a != b)
    assert len(bad) == 0, (len(bad), bad[:5], g[bad[0][0]], o[bad[0][0]])
    np.testing.assert_array_equal(g[:, 22:], o[:, 22:])


@pytest.mark.parametrize("name", ["c1", "c2", "c3s", "tf", "lowB", "negB", "zeroB"])
def test_refit_exact_parity(events, name):
    ev = events[name]
    r, ms = gpu_fits(ev.clusters, ev.row_counts, bz=ev.bz, exact_fp32=1)
    assert len(r.tracks) > 0 and r.fits is not None and len(r.fits) == len(r.tracks)
    o = oracle_fits(r, ev.clusters, ev.bz, mode="f32")
    assert_bits_equal(fit_matrix(r.fits), o)
    assert np.mean(r.fits["status"] == 0) > 0.95
    assert ms[6] > 0.0


def test_refit_exact_parity_tiny_lattice_events():
    """1000 tiny events in one call (short tracks of 10-30 clusters on a
    0.05 cm lattice): every fit equals the oracle's bit for bit."""
    cl, rc = S.tiny_lattice_events(1000, seed=13)
    r, _ = gpu_fits(cl, rc, n_events=1000, exact_fp32=1)
    assert len(r.tracks) > 0
    assert_bits_equal(fit_matrix(r.fits), oracle_fits(r, cl, 0.5, mode="f32"))


def test_refit_exact_parity_polynomial_field(events):
    ev = events["c3s"]
    r, _ = gpu_fits(ev.clusters, ev.row_counts, bz=ev.bz, exact_fp32=1, field=FIELD32)
    o = oracle_fits(r, ev.clusters, ev.bz, field=FIELD32, mode="f32")
    assert_bits_equal(fit_matrix(r.fits), o)
    # the field terms matter: the uniform-field refit differs
    u = oracle_fits(r, ev.clusters, ev.bz, mode="f32")
    assert np.mean(u[:, 5] != o[:, 5]) > 0.9


def test_refit_tracks_unchanged_by_refit(events):
    """The refit is a stage after selection: tracks and clusters are the
    same with and without it."""
    ev = events["c3s"]
    with Tracker(XR, exact_fp32=1) as tr:
        a = tr.track(ev.clusters, ev.row_counts, 1)
        assert a.fits is None
        ms = tr.stage_times()
        assert ms[6] < 0.05  # no refit launched: two adjacent events
        tr.set_params(refit=1)
        b = tr.track(ev.clusters, ev.row_counts, 1)
    np.testing.assert_array_equal(a.tracks.view(np.uint8), b.tracks.view(np.uint8))
    np.testing.assert_array_equal(a.hit_ids, b.hit_ids)


def test_refit_production_vs_fp64(events):
    for name in ("c3s", "tf", "lowB"):
        ev = events[name]
        r, _ = gpu_fits(ev.clusters, ev.row_counts, bz=ev.bz, exact_fp32=0, field=FIELD32)
        o = oracle_fits(r, ev.clusters, ev.bz, field=FIELD32, mode="f64")
        g = fit_matrix(r.fits)
        ok = (g[:, 23] == 0) & (o[:, 23] == 0)
        assert ok.mean() > 0.95
        np.testing.assert_array_equal(g[:, 23], o[:, 23])
        dp = np.abs(g[ok, 1:6] - o[ok, 1:6])
        assert np.all(dp <= 1e-4 * np.abs(o[ok, 1:6]) + 1e-3), (name, dp.max(axis=0))
        assert np.all(np.abs(g[ok, 0] - o[ok, 0]) == 0)
        diag = [6, 8, 11, 15, 20]
        rel = np.abs(g[ok][:, diag] - o[ok][:, diag]) / o[ok][:, diag]
        assert np.all(rel < 1e-2), (name, rel.max(axis=0))
        assert np.all(np.abs(g[ok, 21] - o[ok, 21]) <= 1e-3 * o[ok, 21] + 1e-3)


@pytest.mark.parametrize("over", [dict(plain_per_sector=1), dict(plain_per_sector=2, n_queues=4),
                                  dict(use_graph=1)])
def test_refit_same_in_every_launch_form(events, over):
    ev = events["c3s"]
    base, _ = gpu_fits(ev.clusters, ev.row_counts, exact_fp32=1)
    r, _ = gpu_fits(ev.clusters, ev.row_counts, exact_fp32=1, **over)
    np.testing.assert_array_equal(fit_matrix(r.fits), fit_matrix(base.fits))


def test_refit_multi_event_batch_equals_alone(events):
    evs = [events["c2"], events["c3s"], events["c1"]]
    cl, rc = S.concat_events(evs)
    r, _ = gpu_fits(cl, rc, len(evs), exact_fp32=1)
    for e_i, ev in enumerate(evs):
        a, _ = gpu_fits(ev.clusters, ev.row_counts, exact_fp32=1)
        sel = r.tracks["event"] == e_i
        np.testing.assert_array_equal(fit_matrix(r.fits[sel]), fit_matrix(a.fits))


def test_refit_graph_repeat_and_device_input(events):
    ev = events["tf"]
    with Tracker(XR, refit=1, use_graph=1) as tr:
        a = tr.track(ev.clusters, ev.row_counts, 1)
        b = tr.track(ev.clusters, ev.row_counts, 1)
        d = tr.track(torch.from_numpy(ev.clusters).cuda(), ev.row_counts, 1)
    np.testing.assert_array_equal(fit_matrix(a.fits), fit_matrix(b.fits))
    np.testing.assert_array_equal(fit_matrix(a.fits), fit_matrix(d.fits))


def test_refit_empty_and_tiny_inputs():
    rc = np.zeros(36 * 159, np.int32)
    with Tracker(XR, refit=1) as tr:
        r = tr.track(np.zeros((0, 4), np.float32), rc, 1)
        assert len(r.tracks) == 0 and len(r.fits) == 0


def test_refit_serving_equals_alone(events):
    pool = [events["c2"], events["c3s"], events["lowB"], events["c1"]]
    with Tracker(XR, refit=1) as alone:
        ref = [alone.track(e.clusters, e.row_counts, 1) for e in pool]
    with Tracker(XR, refit=1) as tr:
        tr.stream_configure(arena_bytes=2 << 30, max_batch_events=3, max_inflight=2)
        tickets = [tr.submit(e.clusters, e.row_counts, 1) for e in pool]
        assert all(t is not None for t in tickets)
        got = {}
        while len(got) < len(tickets):
            for i, t in enumerate(tickets):
                if i not in got:
                    res = tr.poll(t, timeout_us=200)
                    if res is not None:
                        got[i] = res
    for i, res in got.items():
        np.testing.assert_array_equal(fit_matrix(res.fits), fit_matrix(ref[i].fits))


def test_refit_full_size_central_sampled():
    """Two full central events in the production build: the oracle (FP64)
    refits a sample of the GPU's tracks one by one; all within tolerance."""
    evs = [S.central_event(seed=3), S.central_event(seed=4)]
    cl, rc = S.concat_events(evs)
    r, ms = gpu_fits(cl, rc, 2)
    assert len(r.fits) > 20000
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(len(r.tracks), 3000, replace=False))

    hits = np.concatenate([r.hits_of(m) for m in idx])
    o = oracle_fits(r, cl, 0.5, mode="f64", tracks=r.tracks[idx], hits=hits)
    g = fit_matrix(r.fits[idx])
    ok = (g[:, 23] == 0) & (o[:, 23] == 0)
    assert ok.mean() > 0.95
    dp = np.abs(g[ok, 1:6] - o[ok, 1:6])
    assert np.all(dp <= 1e-4 * np.abs(o[ok, 1:6]) + 1e-3), dp.max(axis=0)
