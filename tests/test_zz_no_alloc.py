"""The allocation-free entry point tpc_links_noalloc, through the C ABI.

It serves callers that cannot allocate device memory while they run (trigger
components with device memory fixed at start-up, latency-critical loops where
cudaMalloc/cudaFree would synchronize the device).  Its links must equal the
cleaned links of the FP32_EXACT oracle (exact build) and of the allocating
path (tpc_track_sectors, TPC_DUMP_LINKS), exactly -- they are integers -- on
consecutive calls that share its scratch; a warm call must not change the
device's free memory; errors (scratch too small for the bin tables, invalid
input, a capturing stream) are reported and the next call starts afresh.
"""
import ctypes as C
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1712_09430_gb300 import capi, synth as S  # noqa: E402
from paper_1712_09430_gb300.tracker import Tracker, default_params  # noqa: E402

XR = S.row_x().astype(np.float32)


def _geometry():
    g = capi.tpc_geometry()
    g.n_rows = len(XR)
    g.n_sectors = 36
    g.row_x = XR.ctypes.data_as(C.POINTER(C.c_float))
    g.tan_half_open = math.tan(math.radians(10.0))
    g.z_max = 250.0
    return g


def _call(clusters, row_counts, params, stream=None, d_cl=None, d_links=None):
    L = capi.lib()
    n = len(clusters)
    if d_cl is None:
        d_cl = torch.from_numpy(np.ascontiguousarray(clusters, np.float32)).cuda()
    if d_links is None:
        d_links = torch.full((2 * max(n, 1),), -7, dtype=torch.int32, device="cuda")
    rc = np.ascontiguousarray(row_counts, np.int32)
    g = _geometry()
    torch.cuda.synchronize()
    r = L.tpc_links_noalloc(C.byref(g), C.byref(params), C.c_void_p(d_cl.data_ptr()),
                            rc.ctypes.data_as(C.c_void_p), C.c_void_p(d_links.data_ptr()), stream)
    return r, d_links


def _links_noalloc(ev, params):
    r, d_links = _call(ev.clusters, ev.row_counts, params)
    assert r == capi.TPC_OK, capi.STATUS_NAMES.get(r, r)
    return d_links.cpu().numpy()[:2 * ev.n].reshape(2, ev.n)


def _links_tracker(ev, params):
    with Tracker(S.row_x(), bz=ev.bz, params=params) as tr:
        tr.track(ev.clusters, ev.row_counts, 1)
        return tr.dump(capi.TPC_DUMP_LINKS)


def test_links_noalloc_empty_event_is_a_warm_up():
    L = capi.lib()
    g = _geometry()
    rc = np.zeros(36 * 159, np.int32)
    r = L.tpc_links_noalloc(C.byref(g), None, None, rc.ctypes.data_as(C.c_void_p), None, None)
    assert r == capi.TPC_OK


@pytest.mark.parametrize("exact", [1, 0])
def test_links_noalloc_equal_oracle_and_allocating_path_on_consecutive_calls(exact):
    p = default_params(exact_fp32=exact, bin_target=0.5)
    big = S.pp_event(seed=2, scale=4.0)     # ~40 k clusters
    small = S.pp_event(seed=9)              # ~10 k: runs after the big one in the same scratch
    assert big.n <= capi.TPC_NOALLOC_MAX_CLUSTERS
    for ev in (big, small, big):
        want = _links_tracker(ev, p)
        got = _links_noalloc(ev, p)
        assert (want[0] >= 0).sum() > 1000
        np.testing.assert_array_equal(got, want)
        if exact:
            o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR, mode="f32")
            np.testing.assert_array_equal(got[0], o["up"], err_msg="up links vs oracle")
            np.testing.assert_array_equal(got[1], o["dn"], err_msg="down links vs oracle")


def test_links_noalloc_warm_call_allocates_no_device_memory():
    p = default_params(exact_fp32=1)
    ev = S.pp_event(seed=5, scale=3.0)
    d_cl = torch.from_numpy(ev.clusters).cuda()
    d_links = torch.empty((2 * ev.n,), dtype=torch.int32, device="cuda")
    r, _ = _call(ev.clusters, ev.row_counts, p, d_cl=d_cl, d_links=d_links)   # warm
    assert r == capi.TPC_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        r, _ = _call(ev.clusters, ev.row_counts, p, d_cl=d_cl, d_links=d_links)
        assert r == capi.TPC_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_links_noalloc_rejects_oversize_event():
    ev = S.central_event(seed=3, scale=0.05)   # ~100 k clusters > the fixed maximum
    assert ev.n > capi.TPC_NOALLOC_MAX_CLUSTERS
    r, _ = _call(ev.clusters, ev.row_counts, default_params())
    assert r == capi.TPC_ERR_INVALID


def test_links_noalloc_bin_tables_beyond_the_scratch_are_nomem():
    ev = S.pp_event(seed=2, scale=4.0)
    # a bin per 1/1000 of a cluster: every row with clusters takes about
    # 2000 table entries, far beyond the 8 MiB scratch
    assert (ev.row_counts > 0).sum() * 2000 * 4 > capi.TPC_NOALLOC_SCRATCH_BYTES
    r, _ = _call(ev.clusters, ev.row_counts, default_params(bin_target=0.001))
    assert r == capi.TPC_ERR_NOMEM


def test_links_noalloc_invalid_input_then_recovers():
    p = default_params(exact_fp32=1)
    ev = S.pp_event(seed=3)
    bad = ev.clusters.copy()
    bad[17, 1] = np.nan
    r, _ = _call(bad, ev.row_counts, p)
    assert r == capi.TPC_ERR_INVALID
    got = _links_noalloc(ev, p)    # the shared scratch holds no trace of the failed call
    o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR, mode="f32")
    np.testing.assert_array_equal(got[0], o["up"])
    np.testing.assert_array_equal(got[1], o["dn"])


def test_links_noalloc_refuses_a_capturing_stream():
    p = default_params()
    ev = S.pp_event(seed=4)
    d_cl = torch.from_numpy(ev.clusters).cuda()
    d_links = torch.zeros((2 * ev.n,), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    L = capi.lib()
    rc = np.ascontiguousarray(ev.row_counts, np.int32)
    g = _geometry()
    with torch.cuda.graph(graph, stream=s):
        r = L.tpc_links_noalloc(C.byref(g), C.byref(p), C.c_void_p(d_cl.data_ptr()),
                                rc.ctypes.data_as(C.c_void_p), C.c_void_p(d_links.data_ptr()),
                                C.c_void_p(s.cuda_stream))
        d_links.add_(0)   # the capture records something of its own
    assert r == capi.TPC_ERR_INVALID
    got = _links_noalloc(ev, p)   # and the next call outside the capture works
    assert (got[0] >= 0).sum() > 100
