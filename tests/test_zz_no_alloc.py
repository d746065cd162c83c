"""The allocation-free entry point tpc_links_noalloc, through the C ABI.

It serves callers that cannot allocate device memory while they run (trigger
components with device memory fixed at start-up, latency-critical loops where
cudaMalloc/cudaFree would synchronize the device).  Its links must equal the
cleaned links of the allocating path (tpc_track_sectors, TPC_DUMP_LINKS),
exactly -- they are integers -- on consecutive calls that share its scratch.
"""
import ctypes as C
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

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


def _links_noalloc(ev, params):
    L = capi.lib()
    d_cl = torch.from_numpy(ev.clusters).cuda()
    d_links = torch.full((2 * ev.n,), -7, dtype=torch.int32, device="cuda")
    rc = np.ascontiguousarray(ev.row_counts, np.int32)
    g = _geometry()
    torch.cuda.synchronize()
    r = L.tpc_links_noalloc(C.byref(g), C.byref(params), C.c_void_p(d_cl.data_ptr()),
                            rc.ctypes.data_as(C.c_void_p), C.c_void_p(d_links.data_ptr()), None)
    assert r == capi.TPC_OK, capi.STATUS_NAMES.get(r, r)
    return d_links.cpu().numpy().reshape(2, ev.n)


def _links_tracker(ev, params):
    with Tracker(S.row_x(), bz=ev.bz, params=params) as tr:
        tr.track(ev.clusters, ev.row_counts, 1)
        return tr.dump(capi.TPC_DUMP_LINKS)


@pytest.mark.parametrize("exact", [1, 0])
def test_links_noalloc_equal_allocating_path_on_consecutive_calls(exact):
    p = default_params(exact_fp32=exact, bin_target=0.5)
    big = S.pp_event(seed=2, scale=4.0)     # ~40 k clusters
    small = S.pp_event(seed=9)              # ~10 k: runs after the big one in the same scratch
    assert big.n <= capi.TPC_NOALLOC_MAX_CLUSTERS
    for ev in (big, small, big):
        want = _links_tracker(ev, p)
        got = _links_noalloc(ev, p)
        assert (want[0] >= 0).sum() > 1000
        np.testing.assert_array_equal(got, want)


def test_links_noalloc_rejects_oversize_event():
    ev = S.central_event(seed=3, scale=0.05)   # ~100 k clusters > the fixed maximum
    assert ev.n > capi.TPC_NOALLOC_MAX_CLUSTERS
    L = capi.lib()
    p = default_params()
    d_cl = torch.from_numpy(ev.clusters).cuda()
    d_links = torch.empty((2 * ev.n,), dtype=torch.int32, device="cuda")
    rc = np.ascontiguousarray(ev.row_counts, np.int32)
    g = _geometry()
    r = L.tpc_links_noalloc(C.byref(g), C.byref(p), C.c_void_p(d_cl.data_ptr()),
                            rc.ctypes.data_as(C.c_void_p), C.c_void_p(d_links.data_ptr()), None)
    assert r == capi.TPC_ERR_INVALID
