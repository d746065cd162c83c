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
