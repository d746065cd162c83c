"""CPU-only checks of the C ABI library: it builds, loads and exports every
function the header declares; parameter defaults match the oracle's."""
import ctypes as C

import numpy as np

import oracle
from paper_1712_09430_gb300 import capi, default_params


def test_library_exports_every_header_function():
    L = capi.lib()
    names = capi.exported_symbols()
    assert "tpc_track_sectors" in names and "tpc_stream_submit" in names
    for n in names:
        assert hasattr(L, n), n


def test_param_defaults_match_oracle_readings():
    p = default_params()
    o = oracle.default_params()
    for f in ("k_win", "d_max2", "sigma_y", "sigma_z", "var_s", "var_q", "var_t", "n_sigma",
              "w_min", "w_max", "s_max", "y_margin"):
        assert np.float32(getattr(p, f)) == np.float32(getattr(o, f)), f
    for f in ("l_seed", "g_max", "n_min_tracklet", "n_min_track", "own_num", "own_den"):
        assert getattr(p, f) == getattr(o, f), f


def test_struct_sizes():
    assert C.sizeof(capi.tpc_track) == 4 * 22


_C_PROGRAM = r"""
#include <stddef.h>
#include <stdio.h>
#include "tpc_tracker.h"

int main(void)
{
    /* every entry point the header declares, from plain C */
    void* fns[] = {(void*)tpc_params_default, (void*)tpc_tracker_create, (void*)tpc_tracker_destroy,
                   (void*)tpc_tracker_set_params, (void*)tpc_track_sectors, (void*)tpc_fetch_output,
                   (void*)tpc_autotune, (void*)tpc_stream_configure, (void*)tpc_stream_submit,
                   (void*)tpc_stream_poll, (void*)tpc_stream_poll_view, (void*)tpc_stream_release,
                   (void*)tpc_stream_get_stats, (void*)tpc_debug_dump, (void*)tpc_stage_times,
                   (void*)tpc_last_error, (void*)tpc_links_noalloc, (void*)tpc_stream_poll_any,
                   (void*)tpc_stream_set_batching};
    tpc_params p;
    tpc_params_default(&p);  /* host only: no device needed */
    printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(tpc_cluster), sizeof(tpc_geometry),
           sizeof(tpc_params), sizeof(tpc_track), sizeof(tpc_fit), sizeof(tpc_merge), sizeof(tpc_t0),
           sizeof(tpc_output), sizeof(tpc_stream_view), sizeof(tpc_stream_stats), sizeof(fns) / sizeof(fns[0]));
    printf("%d %d %d %g %g %d\n", p.n_min_tracklet, p.tracklets_per_warp, p.schedule, (double)p.bin_target,
           (double)p.k_win, p.count_work);
    printf("%d %u %d %d\n", TPC_NOALLOC_MAX_CLUSTERS, (unsigned)TPC_NOALLOC_SCRATCH_BYTES,
           (int)TPC_STREAM_BATCH_CLUSTERS, p.debug_wait_polls);
    return 0;
}
"""


def test_header_is_plain_c_and_matches_the_binding(tmp_path):
    """A C99 program compiles against the header with warnings as errors,
    links the library, and sees the same struct sizes and parameter defaults
    as the Python binding (no device is used)."""
    import os
    import shutil
    import subprocess
    import pytest
    from paper_1712_09430_gb300 import build_ext

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    capi.lib()  # builds the library if needed
    lib = build_ext.LIB
    src = tmp_path / "abi.c"
    src.write_text(_C_PROGRAM)
    exe = tmp_path / "abi"
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", build_ext.INCLUDE, str(src), "-o", str(exe),
           lib, "-Wl,-rpath," + os.path.dirname(lib)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    sizes, defaults, consts = r.stdout.split("\n")[:3]
    got = [int(v) for v in sizes.split()]
    want = [16, C.sizeof(capi.tpc_geometry), C.sizeof(capi.tpc_params), C.sizeof(capi.tpc_track),
            C.sizeof(capi.tpc_fit), C.sizeof(capi.tpc_merge), C.sizeof(capi.tpc_t0),
            C.sizeof(capi.tpc_output), C.sizeof(capi.tpc_stream_view), C.sizeof(capi.tpc_stream_stats)]
    assert got[:10] == want and got[10] == len(capi.exported_symbols())
    p = default_params()
    d = defaults.split()
    assert [int(d[0]), int(d[1]), int(d[2]), int(d[5])] == [p.n_min_tracklet, p.tracklets_per_warp,
                                                             p.schedule, p.count_work]
    assert float(d[3]) == p.bin_target and abs(float(d[4]) - p.k_win) < 1e-6
    assert [int(v) for v in consts.split()] == [capi.TPC_NOALLOC_MAX_CLUSTERS, capi.TPC_NOALLOC_SCRATCH_BYTES,
                                                 capi.TPC_STREAM_BATCH_CLUSTERS, 0]
