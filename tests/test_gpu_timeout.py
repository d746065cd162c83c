"""A device-side wait that runs out (failure detection without a GPU fault).

Every wait on a bulk copy in the grid and neighbour kernels is bounded; when
the bound is reached the CTA records TPC_ERR_TIMEOUT, waits (again bounded)
for its copies in flight, and returns, and every later stage of the call
does nothing (the buffers it would index were never written).  The test
field debug_wait_polls makes the first wait give up after a single
non-blocking poll, so the time-out path runs on purpose: the call must
report TPC_ERR_TIMEOUT, and the next call on the same tracker, with the
normal bound, must give results identical to a fresh tracker's.  Nothing
here faults, traps or hangs the GPU: the copies complete as usual, only the
first wait stops looking early.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import XR  # noqa: E402
from paper_1712_09430_gb300 import capi, synth as S  # noqa: E402
from paper_1712_09430_gb300.tracker import Tracker, TrackerError  # noqa: E402


@pytest.fixture(scope="module")
def event():
    return S.central_event(seed=3, scale=0.1)


def _same(a, b):
    np.testing.assert_array_equal(a.tracks.view(np.uint8), b.tracks.view(np.uint8))
    np.testing.assert_array_equal(a.hit_ids, b.hit_ids)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_wait_time_out_is_reported_and_the_tracker_stays_usable(event, use_graph):
    ev = event
    with Tracker(XR, exact_fp32=1) as fresh:
        want = fresh.track(ev.clusters, ev.row_counts, 1)
    with Tracker(XR, exact_fp32=1, use_graph=use_graph, debug_wait_polls=1) as tr:
        for _ in range(2):   # twice: the failed call leaves nothing behind
            with pytest.raises(TrackerError) as e:
                tr.track(ev.clusters, ev.row_counts, 1)
            assert e.value.code == capi.TPC_ERR_TIMEOUT
        tr.set_params(debug_wait_polls=0)
        got = tr.track(ev.clusters, ev.row_counts, 1)
        got2 = tr.track(ev.clusters, ev.row_counts, 1)
    _same(got, want)
    _same(got2, want)


def test_wait_time_out_in_the_request_loop(event):
    ev = event
    with Tracker(XR, exact_fp32=1) as fresh:
        want = fresh.track(ev.clusters, ev.row_counts, 1)
    with Tracker(XR, exact_fp32=1, debug_wait_polls=1) as tr:
        tr.stream_configure(arena_bytes=1 << 30)
        t = tr.submit(ev.clusters, ev.row_counts, 1)
        t_end = time.time() + 60
        with pytest.raises(TrackerError) as e:
            while tr.poll(t, timeout_us=1000) is None:
                assert time.time() < t_end
        assert e.value.code == capi.TPC_ERR_TIMEOUT
        tr.set_params(debug_wait_polls=0)
        t = tr.submit(ev.clusters, ev.row_counts, 1)
        r = None
        while r is None:
            r = tr.poll(t, timeout_us=1000)
            assert time.time() < t_end
    _same(r, want)
