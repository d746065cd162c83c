"""Serving: the request loop with continuous batching (tpc_stream_submit/poll).

Each result must be the same alone (tpc_track_sectors on that event) and in
the mix (batched with whatever else was pending), bit for bit: the units of a
batch are independent and every output slot is indexed canonically.
Admission by free arena memory, time-outs and host-side fault injection are
covered without touching the GPU's own state.
"""
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1712_09430_gb300 import capi, synth as S  # noqa: E402
from paper_1712_09430_gb300.tracker import Tracker, TrackerError  # noqa: E402

XR = S.row_x()


@pytest.fixture(scope="module")
def pool():
    evs = [S.pp_event(seed=40 + i) for i in range(4)]
    evs += [S.min_bias_event(seed=1000 + i) for i in range(6)]
    evs += [S.central_event(seed=60, scale=0.1), S.time_frame(seed=61, n_coll=3, scale=0.2)]
    return evs


def _same(a, b):
    np.testing.assert_array_equal(a.tracks.view(np.uint8), b.tracks.view(np.uint8))
    np.testing.assert_array_equal(a.hit_ids, b.hit_ids)


def _drain(tr, tickets, timeout_s=60):
    out = {}
    t_end = time.time() + timeout_s
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            r = tr.poll(t, timeout_us=200)
            if r is not None:
                out[t] = r
        assert time.time() < t_end, "poll timed out"
    return out


@pytest.mark.parametrize("exact,no_copy,policy", [(1, False, None), (0, False, None), (0, True, None),
                                                   (1, False, (600_000, 3000)), (0, True, (1 << 20, 500))])
def test_stream_results_equal_alone(pool, exact, no_copy, policy):
    """Every streamed result equals the synchronous call on its event alone,
    also when the batching policy holds requests back to form larger batches
    while another batch runs."""
    with Tracker(XR, exact_fp32=exact) as alone:
        ref = [alone.track(e.clusters, e.row_counts, 1) for e in pool]
    with Tracker(XR, exact_fp32=exact) as tr:
        tr.stream_configure(arena_bytes=4 << 30, max_batch_events=5, max_inflight=2, no_copy=no_copy)
        if policy:
            tr.stream_set_batching(*policy)
        order = np.random.default_rng(1).permutation(np.repeat(np.arange(len(pool)), 2))
        tickets, which, res = [], {}, {}
        for i in order:
            e = pool[i]
            t = tr.submit(e.clusters, e.row_counts, 1)
            while t is None:                   # not admitted now: collect results, retry
                for tk in tickets:
                    if tk not in res:
                        r = tr.poll(tk, 0)
                        if r is not None:
                            res[tk] = r
                time.sleep(0.0005)
                t = tr.submit(e.clusters, e.row_counts, 1)
            tickets.append(t)
            which[t] = i
        res.update(_drain(tr, [t for t in tickets if t not in res]))
    for t, r in res.items():
        _same(r, ref[which[t]])


def test_stream_multi_event_request(pool):
    evs = pool[:3]
    cl, rc = S.concat_events(evs)
    with Tracker(XR, exact_fp32=1) as tr:
        whole = tr.track(cl, rc, len(evs))
        tr.stream_configure(arena_bytes=2 << 30, max_batch_events=8, max_inflight=2)
        t1 = tr.submit(pool[5].clusters, pool[5].row_counts, 1)
        t2 = tr.submit(cl, rc, len(evs))
        res = _drain(tr, [t1, t2])
    _same(res[t2], whole)


def test_admission_by_free_arena_memory(pool):
    ev = pool[10]  # the largest request in the pool
    with Tracker(XR) as probe:
        probe.track(ev.clusters, ev.row_counts, 1)
    with Tracker(XR) as tr:
        # an arena that holds one such request but not two
        tr.stream_configure(arena_bytes=int(ev.n * 330 * 1.5) + (8 << 20), max_batch_events=4,
                            max_inflight=2)
        t1 = tr.submit(ev.clusters, ev.row_counts, 1)
        assert t1 is not None
        t2 = tr.submit(ev.clusters, ev.row_counts, 1)
        assert t2 is None                      # TPC_BUSY: not admitted now
        r1 = _drain(tr, [t1])[t1]
        t2 = tr.submit(ev.clusters, ev.row_counts, 1)
        assert t2 is not None                  # admitted once memory was freed
        r2 = _drain(tr, [t2])[t2]
    _same(r1, r2)


def test_poll_pending_and_unknown_ticket(pool):
    ev = pool[10]
    with Tracker(XR) as tr:
        tr.stream_configure(arena_bytes=2 << 30)
        t = tr.submit(ev.clusters, ev.row_counts, 1)
        # a central-size event cannot be done within microseconds of submission
        assert tr.poll(t, timeout_us=0) is None
        assert _drain(tr, [t])[t] is not None
        with pytest.raises(TrackerError) as e:
            tr.poll(t, 0)                      # released after its result was taken
        assert e.value.code == capi.TPC_ERR_UNKNOWN_TICKET


def test_fault_injection_admission_and_allocation(pool):
    ev = pool[0]
    os.environ["TPC_FAULT_ADMIT"] = "1"
    try:
        with Tracker(XR) as tr:
            tr.stream_configure(arena_bytes=256 << 20)
            assert tr.submit(ev.clusters, ev.row_counts, 1) is None
            os.environ["TPC_FAULT_ADMIT"] = "0"
            t = tr.submit(ev.clusters, ev.row_counts, 1)
            assert t is not None and _drain(tr, [t])[t] is not None
    finally:
        os.environ.pop("TPC_FAULT_ADMIT", None)
    os.environ["TPC_FAULT_ALLOC"] = "1"
    try:
        with Tracker(XR) as tr:
            tr.stream_configure(arena_bytes=256 << 20)
            with pytest.raises(TrackerError) as e:
                tr.submit(ev.clusters, ev.row_counts, 1)
            assert e.value.code == capi.TPC_ERR_NOMEM
    finally:
        os.environ.pop("TPC_FAULT_ALLOC", None)


def test_stream_rejects_invalid_input(pool):
    ev = pool[1]
    bad = ev.clusters.copy()
    bad[3, 2] = np.inf
    with Tracker(XR) as tr:
        tr.stream_configure(arena_bytes=256 << 20)
        t = tr.submit(bad, ev.row_counts, 1)
        with pytest.raises(TrackerError) as e:
            _drain(tr, [t])
        assert e.value.code == capi.TPC_ERR_INVALID
        # the loop keeps serving
        t = tr.submit(ev.clusters, ev.row_counts, 1)
        assert _drain(tr, [t])[t] is not None


def test_stream_poll_view_equals_poll_and_release(pool):
    evs = pool[:6]
    with Tracker(XR, exact_fp32=1) as a:
        a.stream_configure(arena_bytes=2 << 30, max_batch_events=4, max_inflight=2)
        ta = [a.submit(e.clusters, e.row_counts, 1) for e in evs]
        res = _drain(a, ta)
        ref = [res[t] for t in ta]
    with Tracker(XR, exact_fp32=1) as tr:
        tr.stream_configure(arena_bytes=2 << 30, max_batch_events=4, max_inflight=2)
        tickets = [tr.submit(e.clusters, e.row_counts, 1) for e in evs]
        seen = set()
        t_end = time.time() + 60
        while len(seen) < len(tickets):
            for i, t in enumerate(tickets):
                if i not in seen:
                    v = tr.poll_view(t, timeout_us=200)
                    if v is not None:
                        _same(v, ref[i])
                        tr.release(t)
                        seen.add(i)
            assert time.time() < t_end
        with pytest.raises(TrackerError) as e:
            tr.release(tickets[0])
        assert e.value.code == capi.TPC_ERR_UNKNOWN_TICKET


def test_stream_release_of_pending_ticket_is_refused(pool):
    ev = pool[10]
    with Tracker(XR) as tr:
        tr.stream_configure(arena_bytes=2 << 30)
        t = tr.submit(ev.clusters, ev.row_counts, 1)
        # a central-size event cannot be done within microseconds of submission
        with pytest.raises(TrackerError) as e:
            tr.release(t)
        assert e.value.code == capi.TPC_ERR_INVALID
        assert _drain(tr, [t])[t] is not None


def test_poll_any_returns_each_result_once(pool):
    """tpc_stream_poll_any hands out finished tickets in the order their
    batches finished, each once, with the same results as tracked alone;
    a ticket already taken by a per-ticket poll is skipped."""
    evs = pool[:6]
    with Tracker(XR, exact_fp32=1) as alone:
        ref = [alone.track(e.clusters, e.row_counts, 1) for e in evs]
    with Tracker(XR, exact_fp32=1) as tr:
        tr.stream_configure(arena_bytes=2 << 30, max_batch_events=3, max_inflight=2)
        tickets = {tr.submit(e.clusters, e.row_counts, 1): i for i, e in enumerate(evs)}
        first = next(iter(tickets))
        _same(_drain(tr, [first])[first], ref[tickets[first]])
        seen = set()
        t_end = time.time() + 60
        while len(seen) < len(tickets) - 1:
            got = tr.poll_any(200)
            if got is None:
                assert time.time() < t_end, "poll_any timed out"
                continue
            t, r = got
            assert t in tickets and t != first and t not in seen
            _same(r, ref[tickets[t]])
            tr.release(t)
            seen.add(t)
        assert tr.poll_any(0) is None


@pytest.mark.parametrize("cap", [0, 1])
def test_batches_respect_the_cluster_limit(cap):
    """Requests queued behind a running batch join the next one up to the
    event and cluster limits: with room for one event's clusters every
    later request runs alone; without a cluster limit they run together.
    Results are unchanged either way."""
    evs = [S.central_event(seed=70 + i, scale=0.5) for i in range(4)]
    limit = int(max(e.n for e in evs) * 1.5) if cap else 0
    with Tracker(XR) as alone:
        ref = [alone.track(e.clusters, e.row_counts, 1) for e in evs]
    pinned = [torch.from_numpy(e.clusters).pin_memory() for e in evs]  # fast submits: no copy
    with Tracker(XR) as tr:
        tr.stream_configure(arena_bytes=4 << 30, max_batch_events=8, max_inflight=1,
                            max_batch_clusters=limit, no_copy=True)
        tickets = [tr.submit(c, e.row_counts, 1) for c, e in zip(pinned, evs)]
        assert all(t is not None for t in tickets)
        got = _drain(tr, tickets)
        st = tr.stream_stats()
    for t, r in zip(tickets, ref):
        _same(got[t], r)
    if cap:
        assert st["batches"] == 4 and st["max_batch_events"] == 1
    else:  # the three queued behind the first run together (unless it ended first)
        assert st["batches"] < 4 and st["max_batch_events"] >= 2
    # the longest single launch and submit are kept beside the sums
    assert 0 < st["max_launch_ms"] <= st["host_launch_ms"]
    assert st["max_submit_ms"] > 0


def test_cluster_limit_is_validated():
    with Tracker(XR) as tr:
        with pytest.raises(TrackerError):
            tr.stream_configure(max_batch_clusters=-1)


def test_batching_policy_holds_small_requests_while_a_batch_runs(pool):
    """With the batching policy, requests that arrive while a batch runs wait
    and go together once it ends, instead of forming a second small batch at
    once (two slots are free); results are unchanged."""
    big = S.central_event(seed=71)
    small = pool[:3]
    with Tracker(XR) as alone:
        ref_big = alone.track(big.clusters, big.row_counts, 1)
        ref = [alone.track(e.clusters, e.row_counts, 1) for e in small]
    pinned = [torch.from_numpy(e.clusters).pin_memory() for e in [big] + small]
    with Tracker(XR) as tr:
        tr.stream_configure(arena_bytes=8 << 30, max_batch_events=8, max_inflight=2, no_copy=True)
        tr.stream_set_batching(min_batch_clusters=1 << 30, max_wait_us=2_000_000)
        t_big = tr.submit(pinned[0], big.row_counts, 1)   # nothing runs: goes at once
        tickets = [tr.submit(c, e.row_counts, 1) for c, e in zip(pinned[1:], small)]
        got = _drain(tr, [t_big] + tickets)
        st = tr.stream_stats()
    _same(got[t_big], ref_big)
    for t, r in zip(tickets, ref):
        _same(got[t], r)
    assert st["batches"] == 2 and st["max_batch_events"] == 3
    with Tracker(XR) as tr:
        with pytest.raises(TrackerError):
            tr.stream_set_batching(min_batch_clusters=-1)
        with pytest.raises(TrackerError):
            tr.stream_set_batching(max_wait_us=-5)
