"""CPU oracle of the per-sector TPC tracker and of the final track fit
(test infrastructure only).

Only tests/, the package smoke check and the CPU-baseline leg of the
benchmark load this module.  The CUDA path never imports it, and it imports
nothing from the CUDA path.  See tpc_oracle.c for what each function follows
and what pins it; tpc_refit.c holds the full Kalman filter refit.

Two builds of the same C source:
  mode="f64"  FP64 accuracy reference
  mode="f32"  FP32_EXACT: the same expressions in binary32, no FMA contraction
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "tpc_oracle.c"), os.path.join(_HERE, "tpc_refit.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIBS = {}

N_TL_F = 16  # x y z s t q cy[6] cz[3] chi2
N_FIT = 24   # x p[5] cov[15] chi2 ndf status


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("k_win", "d_max2", "n_sigma", "w_min", "w_max",
                                          "s_max", "y_margin", "sigma_y", "sigma_z", "var_s",
                                          "var_q", "var_t")] + \
               [(n, C.c_int) for n in ("g_max", "l_seed", "n_min_tracklet", "n_min_track",
                                       "own_num", "own_den")]


class FitParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("sigma_y", "sigma_z", "var_s", "var_t", "var_q", "s_max",
                                          "bz")] + [("b", C.c_double * 5)]


class MergeParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("chi2_max", "gap", "overlap", "window", "cos_t", "sin_t")]


class T0Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("y_cut", "bin", "z_max", "radius")] + \
               [("window", C.c_int), ("n_min", C.c_int)]


class Geom(C.Structure):
    _fields_ = [("n_rows", C.c_int), ("n_sectors", C.c_int), ("row_x", C.POINTER(C.c_float)),
                ("tan_half_open", C.c_float), ("z_max", C.c_float)]


def _lib_path(mode):
    return os.path.join(_BUILD, f"liboracle_{mode}.so")


def build(force=False):
    """Compile both oracle modes with gcc (-ffp-contract=off, no fast math)."""
    os.makedirs(_BUILD, exist_ok=True)
    for mode, real in (("f64", "double"), ("f32", "float")):
        out = _lib_path(mode)
        if not force and os.path.exists(out) and \
                os.path.getmtime(out) >= max(os.path.getmtime(f) for f in _SRCS):
            continue
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                "-shared", f"-DORACLE_REAL={real}", *_SRCS, "-o", out + ".tmp", "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True)
        os.replace(out + ".tmp", out)


def lib(mode="f64"):
    if mode not in _LIBS:
        build()
        L = C.CDLL(_lib_path(mode))
        P, V = C.POINTER, C.c_void_p
        L.orc_params_default.argtypes = [P(Params)]
        L.orc_run.restype = V
        L.orc_run.argtypes = [P(Params), P(Geom), C.c_double, C.c_int, V, V, C.c_int]
        L.orc_sizes.argtypes = [V, P(C.c_int64), P(C.c_double)]
        L.orc_copy_links.argtypes = [V, V, V, V, V]
        L.orc_copy_tracklets.argtypes = [V, V, V, V, V, V, V, V]
        L.orc_copy_tracks.argtypes = [V, V, V, V, V]
        L.orc_free.argtypes = [V]
        L.orc_propagate.argtypes = [P(Params), C.c_double, V, C.c_double]
        L.orc_update_state.argtypes = [P(Params), V, C.c_double, C.c_double, P(C.c_double)]
        L.orc_fit_hits.argtypes = [P(Params), C.c_double, V, C.c_int, V, V, V, P(C.c_double)]
        L.orc_refit_tracks.argtypes = [P(FitParams), C.c_int, V, V, V, V, V, C.c_int]
        L.orc_refit_propagate.argtypes = [P(FitParams), V, C.c_double]
        L.orc_refit_update.argtypes = [P(FitParams), V, C.c_double, C.c_double, P(C.c_double)]
        L.orc_merge_tracks.argtypes = [P(FitParams), P(MergeParams), C.c_int, C.c_int, V, V, V, V, V,
                                       C.c_int]
        L.orc_merge_rotate.argtypes = [P(FitParams), V, C.c_double, C.c_double]
        L.orc_merge_propagate.argtypes = [P(FitParams), V, C.c_double]
        L.orc_merge_chi2.argtypes = [V, V, P(C.c_double)]
        L.orc_t0_tracks.argtypes = [P(FitParams), P(T0Params), C.c_int, C.c_int, V, V, V]
        L.orc_max_threads.restype = C.c_int
        L.orc_real_size.restype = C.c_int
        _LIBS[mode] = L
    return _LIBS[mode]


def _set_field(st, k, v):
    """Set field k of a ctypes structure; a name that is not a field raises
    (setattr alone would keep it as a plain attribute and change nothing)."""
    if k not in {f for f, _ in type(st)._fields_}:
        raise TypeError(f"unknown oracle parameter {k!r}")
    setattr(st, k, v)


def default_params(**over) -> Params:
    p = Params()
    lib("f64").orc_params_default(C.byref(p))
    for k, v in over.items():
        _set_field(p, k, v)
    return p


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def geometry(row_x, n_sectors=36, tan_half_open=None, z_max=250.0):
    import math
    xr = np.ascontiguousarray(row_x, dtype=np.float32)
    g = Geom()
    g.n_rows = len(xr)
    g.n_sectors = n_sectors
    g.row_x = xr.ctypes.data_as(C.POINTER(C.c_float))
    g.tan_half_open = math.tan(math.radians(10.0)) if tan_half_open is None else tan_half_open
    g.z_max = z_max
    g._keep = xr
    return g


def run(clusters, row_counts, n_events, bz, row_x, params=None, mode="f64", threads=0,
        n_sectors=36):
    """Track a batch of events; returns a dict of numpy arrays.

    clusters   float32 [N, 4] (x, y, z, id bits), grouped by (event, sector, row)
    row_counts int32 [n_events * n_sectors * n_rows]
    Output indices are global cluster indices (positions in `clusters`);
    tracklets and tracks are in canonical order (event, sector, row, id)."""
    L = lib(mode)
    p = params if params is not None else default_params()
    g = geometry(row_x, n_sectors=n_sectors)
    cl = np.ascontiguousarray(clusters, dtype=np.float32)
    rc = np.ascontiguousarray(row_counts, dtype=np.int32)
    assert cl.ndim == 2 and cl.shape[1] == 4
    assert rc.size == n_events * n_sectors * g.n_rows and int(rc.sum()) == len(cl)
    res = L.orc_run(C.byref(p), C.byref(g), float(bz), int(n_events), _ptr(cl), _ptr(rc), int(threads))
    try:
        sz = (C.c_int64 * 5)()
        secs = C.c_double()
        L.orc_sizes(res, sz, C.byref(secs))
        N, T, TH, M, MH = [int(v) for v in sz]
        out = dict(seconds=secs.value)
        for k in ("up_raw", "dn_raw", "up", "dn"):
            out[k] = np.empty(N, np.int32)
        L.orc_copy_links(res, _ptr(out["up_raw"]), _ptr(out["dn_raw"]), _ptr(out["up"]),
                         _ptr(out["dn"]))
        out["start"] = np.empty(T, np.int32)
        out["tl_unit"] = np.empty(T, np.int32)
        out["tl_f"] = np.empty((T, N_TL_F), np.float64)
        out["tl_n"] = np.empty(T, np.int32)
        out["tl_alive"] = np.empty(T, np.int32)
        out["tl_hit_off"] = np.empty(T + 1, np.int64)
        out["tl_hits"] = np.empty(TH, np.int32)
        L.orc_copy_tracklets(res, _ptr(out["start"]), _ptr(out["tl_unit"]), _ptr(out["tl_f"]),
                             _ptr(out["tl_n"]), _ptr(out["tl_alive"]), _ptr(out["tl_hit_off"]),
                             _ptr(out["tl_hits"]))
        out["trk_t"] = np.empty(M, np.int32)
        out["trk_n"] = np.empty(M, np.int32)
        out["trk_hit_off"] = np.empty(M + 1, np.int64)
        out["trk_hits"] = np.empty(MH, np.int32)
        L.orc_copy_tracks(res, _ptr(out["trk_t"]), _ptr(out["trk_n"]), _ptr(out["trk_hit_off"]),
                          _ptr(out["trk_hits"]))
        return out
    finally:
        L.orc_free(res)


# single-function access for the pin tests ---------------------------------

def state_vec(x, y, z, s, t, q, cy=(0, 0, 0, 0, 0, 0), cz=(0, 0, 0)):
    return np.array([x, y, z, s, t, q, *cy, *cz], dtype=np.float64)


def propagate(v, x1, bz, params=None, mode="f64"):
    v = np.array(v, dtype=np.float64)
    p = params if params is not None else default_params()
    ok = lib(mode).orc_propagate(C.byref(p), float(bz), _ptr(v), float(x1))
    return bool(ok), v


def update(v, my, mz, params=None, mode="f64", chi2=0.0):
    v = np.array(v, dtype=np.float64)
    p = params if params is not None else default_params()
    c = C.c_double(chi2)
    lib(mode).orc_update_state(C.byref(p), _ptr(v), float(my), float(mz), C.byref(c))
    return v, c.value


def fit_hits(v, x, y, z, bz, params=None, mode="f64"):
    v = np.array(v, dtype=np.float64)
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    p = params if params is not None else default_params()
    c = C.c_double(0.0)
    n = lib(mode).orc_fit_hits(C.byref(p), float(bz), _ptr(v), len(x), _ptr(x), _ptr(y), _ptr(z),
                               C.byref(c))
    return n, v, c.value


def max_threads():
    return int(lib("f64").orc_max_threads())


# final track fit (tpc_refit.c) ---------------------------------------------

def fit_params(bz, field=None, params=None, **over) -> FitParams:
    """Constants of the refit: cluster errors, reset variances and s_max from
    the tracker params, the constant field bz and the polynomial terms
    field = (b1..b5) of Bz = bz + z (b1 + z b2) + rho^2 (b3 + z (b4 + z b5))."""
    p = params if params is not None else default_params()
    f = FitParams()
    for k in ("sigma_y", "sigma_z", "var_s", "var_t", "var_q", "s_max"):
        setattr(f, k, getattr(p, k))
    f.bz = bz
    for j, v in enumerate(field if field is not None else (0.0,) * 5):
        f.b[j] = v
    for k, v in over.items():
        _set_field(f, k, v)
    return f


def refit_tracks(o, clusters, bz, field=None, params=None, mode="f64", threads=0, fp=None):
    """Refit the selected tracks of an oracle result `o` (run()): start state
    from each track's tracklet (tl_f x..q), clusters from `clusters` by the
    track's hit positions.  Returns float64 [M, N_FIT]."""
    f = fp if fp is not None else fit_params(bz, field, params)
    st6 = np.ascontiguousarray(o["tl_f"][o["trk_t"], :6], np.float64)
    return refit_lists(st6, o["trk_hit_off"], o["trk_hits"], clusters, f, mode, threads)


def refit_lists(st6, hit_off, hits, clusters, fp, mode="f64", threads=0):
    st6 = np.ascontiguousarray(st6, np.float64).reshape(-1, 6)
    M = len(st6)
    off = np.ascontiguousarray(hit_off, np.int64)
    h = np.ascontiguousarray(hits, np.int32)
    cl = np.ascontiguousarray(clusters, np.float32)
    out = np.zeros((M, N_FIT), np.float64)
    lib(mode).orc_refit_tracks(C.byref(fp), M, _ptr(st6), _ptr(off), _ptr(h), _ptr(cl), _ptr(out),
                               int(threads))
    return out


def fit_vec(x, p, S5=None):
    """31-vector of the single-step refit entries: x, p[5], the covariance
    factor S (C = S S^T) row-major."""
    v = np.zeros(31)
    v[0] = x
    v[1:6] = p
    if S5 is not None:
        v[6:] = np.asarray(S5, dtype=np.float64).reshape(25)
    return v


def factor_of(v):
    return v[6:31].reshape(5, 5)


def cov_of(v):
    """C = S S^T of a 31-vector."""
    S5 = factor_of(v)
    return S5 @ S5.T


def unpack_cov(v, at=6):
    """Symmetric 5x5 from 15 packed lower entries (a refit output row)."""
    C5 = np.zeros((5, 5))
    k = at
    for i in range(5):
        for j in range(i + 1):
            C5[i, j] = C5[j, i] = v[k]
            k += 1
    return C5


def refit_propagate(v, x1, fp, mode="f64"):
    v = np.array(v, dtype=np.float64)
    ok = lib(mode).orc_refit_propagate(C.byref(fp), _ptr(v), float(x1))
    return bool(ok), v


def refit_update(v, my, mz, fp, mode="f64", chi2=0.0):
    v = np.array(v, dtype=np.float64)
    c = C.c_double(chi2)
    lib(mode).orc_refit_update(C.byref(fp), _ptr(v), float(my), float(mz), C.byref(c))
    return v, c.value


# track merging (tpc_refit.c, Phase II) -------------------------------------

def merge_params(chi2_max=30.0, gap=50.0, overlap=5.0, window=5.0, angle_deg=20.0) -> MergeParams:
    import math
    m = MergeParams()
    m.chi2_max, m.gap, m.overlap, m.window = chi2_max, gap, overlap, window
    m.cos_t = float(np.float32(math.cos(math.radians(angle_deg))))
    m.sin_t = float(np.float32(math.sin(math.radians(angle_deg))))
    return m


def merge_tracks(unit, fits, x_last, fp, mp=None, n_sectors=36, mode="f64"):
    """Merge links of refitted tracks (canonical order).  unit[M] = event *
    n_sectors + sector; fits [M, N_FIT] (refit outputs); x_last[M].  Returns
    (next[M] int32, chi2[M])."""
    mp = mp if mp is not None else merge_params()
    u = np.ascontiguousarray(unit, np.int32)
    f = np.ascontiguousarray(fits, np.float64)
    xl = np.ascontiguousarray(x_last, np.float64)
    M = len(u)
    nxt = np.full(M, -1, np.int32)
    chi = np.zeros(M, np.float64)
    lib(mode).orc_merge_tracks(C.byref(fp), C.byref(mp), M, n_sectors, _ptr(u), _ptr(f), _ptr(xl),
                               _ptr(nxt), _ptr(chi), 0)
    return nxt, chi


def merge_vec(x, p, C5=None):
    """31-vector of the merge entries: x, p[5], C[5][5] row-major."""
    v = np.zeros(31)
    v[0] = x
    v[1:6] = p
    if C5 is not None:
        v[6:] = np.asarray(C5, np.float64).reshape(25)
    return v


def merge_rotate(v, cos_t, sin_t, fp, mode="f64"):
    v = np.array(v, dtype=np.float64)
    ok = lib(mode).orc_merge_rotate(C.byref(fp), _ptr(v), float(cos_t), float(sin_t))
    return bool(ok), v


def merge_propagate(v, x1, fp, mode="f64"):
    v = np.array(v, dtype=np.float64)
    ok = lib(mode).orc_merge_propagate(C.byref(fp), _ptr(v), float(x1))
    return bool(ok), v


def merge_chi2(va, vb, mode="f64"):
    va = np.ascontiguousarray(va, np.float64)
    vb = np.ascontiguousarray(vb, np.float64)
    c = C.c_double()
    ok = lib(mode).orc_merge_chi2(_ptr(va), _ptr(vb), C.byref(c))
    return bool(ok), c.value


# continuous readout: collision offsets (tpc_refit.c) ------------------------

def t0_params(y_cut=1.0, bin=0.25, z_max=250.0, radius=1.0, window=8, n_min=8) -> T0Params:
    t = T0Params()
    t.y_cut, t.bin, t.z_max, t.radius, t.window, t.n_min = y_cut, bin, z_max, radius, window, n_min
    return t


def t0_tracks(unit, fits, fp, tp=None, n_sectors=36, mode="f64"):
    """Per refitted track: (collision, u, D) of the continuous-readout
    readings; returns float64 [M, 3]."""
    tp = tp if tp is not None else t0_params()
    u = np.ascontiguousarray(unit, np.int32)
    f = np.ascontiguousarray(fits, np.float64)
    out = np.zeros((len(u), 3))
    lib(mode).orc_t0_tracks(C.byref(fp), C.byref(tp), len(u), n_sectors, _ptr(u), _ptr(f), _ptr(out))
    return out
