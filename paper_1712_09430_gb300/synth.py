"""Seeded synthetic TPC events (FP64 physics, FP32 clusters).

This module only draws inputs: helix tracks, their crossings with the pad-row
planes of the 36 sectors, Gaussian smearing, per-row cluster loss and uniform
noise clusters.  It holds none of the tracker's arithmetic (no neighbour
search, no Kalman filter, no selection) and serves both the CUDA path and the
CPU oracle.

Geometry (the TPC of Sec. 2, Fig. 1 a,b): two halves of 18 trapezoidal sectors
with a 10 degree half-opening; 159 pad rows that are planes x = X_r in the
sector frame (63 rows at 0.75 cm pitch from 85 cm, 64 at 1.0 cm from 135 cm,
32 at 1.5 cm from 199.5 cm).  Sector s < 18 is side A (z >= 0), s >= 18 is
side C (z < 0); its centre azimuth is 20 deg * (s mod 18) + 10 deg.

Track model: a helix in a constant field Bz along the beam.  The signed
curvature is k = -KAPPA * Bz * q / pT, so a positive charge in +Bz turns
clockwise (towards -y when moving along +x), as the Lorentz force F = q v x B
gives.  Position along the transverse path length s:
    X(s) = vx + (sin(phi0 + k s) - sin(phi0)) / k
    Y(s) = vy - (cos(phi0 + k s) - cos(phi0)) / k
    Z(s) = vz + tan(lambda) * s
Only the first outgoing branch in each sector frame is kept (cos(phi_local) > 0
from the vertex on), so a looper contributes one half-turn.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KAPPA = 0.00299792458  # curvature [1/cm] per (T * c/GeV)
N_ROWS = 159
N_SECTORS = 36
TAN_HALF_OPEN = math.tan(math.radians(10.0))
Z_MAX = 250.0
SIGMA = 0.1  # cm, cluster smearing in y and z


def row_x() -> np.ndarray:
    """Pad-row radii X_r (cm), float64, exactly representable in float32."""
    r = np.arange(N_ROWS, dtype=np.float64)
    x = np.where(r < 63, 85.0 + 0.75 * r,
                 np.where(r < 127, 135.0 + 1.0 * (r - 63), 199.5 + 1.5 * (r - 127)))
    return x


def sector_alpha(s) -> np.ndarray:
    return np.radians(20.0 * (np.asarray(s) % 18) + 10.0)


@dataclasses.dataclass
class Tracks:
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    phi0: np.ndarray   # lab-frame azimuth of the momentum at the vertex
    pt: np.ndarray     # GeV/c
    tanl: np.ndarray   # dz/ds
    q: np.ndarray      # +-1

    def __len__(self):
        return len(self.pt)

    @staticmethod
    def concat(parts):
        return Tracks(*[np.concatenate([getattr(p, f.name) for p in parts])
                        for f in dataclasses.fields(Tracks)])


@dataclasses.dataclass
class Event:
    """One event (or one time-frame slice): clusters grouped by (sector, row).

    clusters   float32 [N, 4]: x, y, z, id (uint32 bit pattern in column 3)
    row_counts int32 [36 * 159], CSR counts in (sector, row) order
    label      int32 [N]: generating track index, -1 for noise
    true_y, true_z, true_s  float64 [N]: noise-free crossing (NaN for noise)
    tracks     the generated tracks
    bz         field in T
    """
    clusters: np.ndarray
    row_counts: np.ndarray
    label: np.ndarray
    true_y: np.ndarray
    true_z: np.ndarray
    true_s: np.ndarray
    tracks: Tracks
    bz: float

    @property
    def n(self):
        return len(self.clusters)

    @property
    def ids(self):
        return self.clusters.view(np.uint32)[:, 3]


def _draw_pt(rng, n, mean, lo=0.1, hi=10.0):
    """Exponential pT by inverse CDF, redrawn outside [lo, hi]."""
    pt = np.empty(n)
    todo = np.arange(n)
    while len(todo):
        u = rng.random(len(todo))
        v = -mean * np.log1p(-u)
        ok = (v >= lo) & (v <= hi)
        pt[todo[ok]] = v[ok]
        todo = todo[~ok]
    return pt


def gen_tracks(rng, n_prim, n_sec, pt_mean=0.6, eta_max=0.9, phi_lo=0.0,
               phi_hi=2 * math.pi, sec_dmax=50.0, vz=0.0) -> Tracks:
    """Primaries from (0, 0, vz) plus secondaries from vertices d * u_hat,
    d ~ U[0, sec_dmax] cm, u_hat isotropic; shared pT/eta/phi/charge laws."""
    n = n_prim + n_sec
    pt = _draw_pt(rng, n, pt_mean)
    eta = rng.uniform(-eta_max, eta_max, n)
    phi = rng.uniform(phi_lo, phi_hi, n)
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    vx = np.zeros(n)
    vy = np.zeros(n)
    vzz = np.full(n, float(vz))
    if n_sec:
        d = rng.uniform(0.0, sec_dmax, n_sec)
        cth = rng.uniform(-1.0, 1.0, n_sec)
        ph = rng.uniform(0.0, 2 * math.pi, n_sec)
        sth = np.sqrt(1.0 - cth * cth)
        vx[n_prim:] = d * sth * np.cos(ph)
        vy[n_prim:] = d * sth * np.sin(ph)
        vzz[n_prim:] += d * cth
    return Tracks(vx, vy, vzz, phi, pt, np.sinh(eta), q)


def curvature(tracks: Tracks, bz: float) -> np.ndarray:
    return -KAPPA * bz * tracks.q / tracks.pt


def helix_lab(tracks: Tracks, bz: float, idx, s):
    """Lab-frame helix point at transverse path length s (closed form)."""
    k = curvature(tracks, bz)[idx]
    p0 = tracks.phi0[idx]
    s = np.asarray(s, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        X = tracks.vx[idx] + np.where(k != 0, (np.sin(p0 + k * s) - np.sin(p0)) / k, s * np.cos(p0))
        Y = tracks.vy[idx] - np.where(k != 0, (np.cos(p0 + k * s) - np.cos(p0)) / k, -s * np.sin(p0))
    Z = tracks.vz[idx] + tracks.tanl[idx] * s
    return X, Y, Z


def _candidate_sectors(tracks: Tracks, bz: float):
    """(track, azimuthal sector 0..17) pairs the outgoing branch may cross.

    The branch is sampled at 64 points between the vertex and min(half a turn,
    the path to leave radius 260 cm); every sector whose wedge holds a sample
    at radius >= 80 cm is taken, together with both neighbours."""
    n = len(tracks)
    k = curvature(tracks, bz)
    with np.errstate(divide="ignore"):
        half_turn = np.where(k != 0, math.pi / np.abs(k), np.inf)
    s_end = np.minimum(half_turn, 330.0)
    frac = np.linspace(0.0, 1.0, 64)
    s = s_end[:, None] * frac[None, :]
    X, Y, _ = helix_lab(tracks, bz, np.arange(n)[:, None], s)
    rho = np.hypot(X, Y)
    az = np.mod(np.arctan2(Y, X), 2 * math.pi)
    sec = np.floor(az / math.radians(20.0)).astype(np.int64) % 18
    inside = rho >= 80.0
    mask = np.zeros((n, 18), dtype=bool)
    ti = np.broadcast_to(np.arange(n)[:, None], sec.shape)
    for dsec in (-1, 0, 1):
        mask[ti[inside], (sec[inside] + dsec) % 18] = True
    return np.nonzero(mask)


def crossings(tracks: Tracks, bz: float, xr=None):
    """Noise-free crossings of the outgoing branch with every pad-row plane.

    Returns dict of equal-length arrays: track, sector (0..35), row, y, z,
    sphi (sin of the local direction angle at the crossing) and path (the
    transverse path length from the vertex)."""
    if xr is None:
        xr = row_x()
    tr_idx, az_sec = _candidate_sectors(tracks, bz)
    if len(tr_idx) == 0:
        z = np.zeros(0)
        return dict(track=z.astype(np.int64), sector=z.astype(np.int64), row=z.astype(np.int64),
                    y=z, z=z, sphi=z, path=z)
    k = curvature(tracks, bz)[tr_idx]
    alpha = sector_alpha(az_sec)
    ca, sa = np.cos(alpha), np.sin(alpha)
    vx, vy = tracks.vx[tr_idx], tracks.vy[tr_idx]
    x0 = vx * ca + vy * sa
    y0 = -vx * sa + vy * ca
    phl0 = np.angle(np.exp(1j * (tracks.phi0[tr_idx] - alpha)))  # wrapped to (-pi, pi]
    outgoing = np.cos(phl0) > 0.0
    X = xr[None, :]
    w = np.sin(phl0)[:, None] + k[:, None] * (X - x0[:, None])
    ok = outgoing[:, None] & (np.abs(w) < 1.0) & (X > x0[:, None])
    wc = np.clip(w, -1.0, 1.0)
    phl = np.arcsin(wc)
    dphi = phl - phl0[:, None]
    kk = k[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        path = np.where(kk != 0, dphi / kk, (X - x0[:, None]) / np.cos(phl0)[:, None])
        # y = y0 - (cos(phl) - cos(phl0)) / k, written without cancellation
        y = y0[:, None] + np.where(kk != 0,
                                   2.0 * np.sin(0.5 * (phl + phl0[:, None])) * np.sin(0.5 * dphi) / kk,
                                   path * np.sin(phl0)[:, None])
    z = tracks.vz[tr_idx][:, None] + tracks.tanl[tr_idx][:, None] * path
    ok &= path >= 0.0
    ok &= np.abs(y) <= X * TAN_HALF_OPEN
    ok &= np.abs(z) <= Z_MAX
    it, ir = np.nonzero(ok)
    zz = z[it, ir]
    sector = az_sec[it] + np.where(zz >= 0.0, 0, 18)
    return dict(track=tr_idx[it], sector=sector, row=ir, y=y[it, ir], z=zz,
                sphi=w[it, ir], path=path[it, ir])


def _assemble(rng, tracks, bz, cr, eff, sigma, noise_frac=0.0, noise_sector=None):
    """Cluster loss, smearing and noise, then one (sector, row) grouping."""
    keep = rng.random(len(cr["row"])) < eff
    sec = cr["sector"][keep]
    row = cr["row"][keep]
    ty = cr["y"][keep]
    tz = cr["z"][keep]
    ts = cr["sphi"][keep]
    lab = cr["track"][keep].astype(np.int64)
    yy = ty + rng.normal(0.0, sigma, len(ty)) if sigma > 0 else ty.copy()
    zz = tz + rng.normal(0.0, sigma, len(tz)) if sigma > 0 else tz.copy()
    n_noise = int(round(noise_frac * len(ty)))
    if n_noise:
        ns = (rng.integers(0, N_SECTORS, n_noise) if noise_sector is None
              else np.full(n_noise, noise_sector))
        ns, nr, ny, nz = _noise(rng, n_noise, ns)
        nan = np.full(n_noise, np.nan)
        sec = np.concatenate([sec, ns]); row = np.concatenate([row, nr])
        yy = np.concatenate([yy, ny]); zz = np.concatenate([zz, nz])
        ty = np.concatenate([ty, nan]); tz = np.concatenate([tz, nan]); ts = np.concatenate([ts, nan])
        lab = np.concatenate([lab, np.full(n_noise, -1)])
    base = Event(np.zeros((0, 4), np.float32), np.zeros(N_SECTORS * N_ROWS, np.int32),
                 np.zeros(0, np.int32), np.zeros(0), np.zeros(0), np.zeros(0), tracks, float(bz))
    return _rebuild(rng, base, sec, row, yy, zz, lab, ty, tz, ts)


def make_event(seed, n_prim, n_sec=0, pt_mean=0.6, noise_frac=0.05, eff=0.95, sigma=SIGMA,
               bz=0.5, phi_lo=0.0, phi_hi=2 * math.pi, only_sector=None, vz=0.0) -> Event:
    rng = np.random.default_rng(seed)
    tracks = gen_tracks(rng, n_prim, n_sec, pt_mean=pt_mean, phi_lo=phi_lo, phi_hi=phi_hi, vz=vz)
    cr = crossings(tracks, bz)
    if only_sector is not None:
        m = cr["sector"] == only_sector
        cr = {key: v[m] for key, v in cr.items()}
    return _assemble(rng, tracks, bz, cr, eff, sigma, noise_frac, only_sector)


def _rebuild(rng, ev: Event, sec, row, y, z, lab, ty, tz, ts):
    """Group clusters by (sector, row) in a random order inside each row,
    cast to float32 clusters and give them a random permutation of ids."""
    n = len(y)
    key = ((np.asarray(sec, np.int64) * N_ROWS + np.asarray(row, np.int64)) << 32) | \
        rng.integers(0, 1 << 32, n, dtype=np.int64)
    order = np.argsort(key, kind="stable")
    sec, row = sec[order], row[order]
    xr = row_x()
    cl = np.empty((n, 4), dtype=np.float32)
    cl[:, 0] = xr[row].astype(np.float32)
    cl[:, 1] = y[order].astype(np.float32)
    cl[:, 2] = z[order].astype(np.float32)
    cl.view(np.uint32)[:, 3] = rng.permutation(n).astype(np.uint32)
    counts = np.bincount(sec * N_ROWS + row, minlength=N_SECTORS * N_ROWS).astype(np.int32)
    return Event(cl, counts, lab[order].astype(np.int32), ty[order], tz[order], ts[order],
                 ev.tracks, ev.bz)


def _unpack(ev: Event):
    sec_row = np.repeat(np.arange(N_SECTORS * N_ROWS), ev.row_counts)
    return (sec_row // N_ROWS, sec_row % N_ROWS, ev.clusters[:, 1].astype(np.float64),
            ev.clusters[:, 2].astype(np.float64), ev.label.astype(np.int64), ev.true_y, ev.true_z,
            ev.true_s)


def _noise(rng, n_noise, sectors):
    """Uniform noise: row uniform, y uniform over the row's width, z uniform
    over the sector's drift half."""
    xr = row_x()
    ns = sectors
    nr = rng.integers(0, N_ROWS, n_noise)
    half = xr[nr] * TAN_HALF_OPEN
    ny = rng.uniform(-1.0, 1.0, n_noise) * half
    nz = rng.uniform(0.0, Z_MAX, n_noise) * np.where(ns < 18, 1.0, -1.0)
    return ns, nr, ny, nz


def _add_noise(rng, ev: Event, n_noise):
    ns = rng.integers(0, N_SECTORS, n_noise)
    if n_noise == 0:
        return ev
    sec, row, y, z, lab, ty, tz, ts = _unpack(ev)
    ns, nr, ny, nz = _noise(rng, n_noise, ns)
    nan = np.full(n_noise, np.nan)
    return _rebuild(rng, ev, np.concatenate([sec, ns]), np.concatenate([row, nr]),
                    np.concatenate([y, ny]), np.concatenate([z, nz]),
                    np.concatenate([lab, np.full(n_noise, -1)]), np.concatenate([ty, nan]),
                    np.concatenate([tz, nan]), np.concatenate([ts, nan]))


def min_bias_tracks(rng) -> int:
    """Multiplicity from the impact parameter b ~ U[0, 15] fm:
    N = 10 + 9990 * (1 - b / 15) ** 8.5 (10 tracks peripheral, 10,000 central)."""
    b = rng.uniform(0.0, 15.0)
    return int(round(10 + 9990 * (1.0 - b / 15.0) ** 8.5))


# ---------------------------------------------------------------------------
# The five workloads.  Sizes follow the single-sector, pp, central Pb-Pb,
# continuous-readout time-frame and streaming configurations.
# ---------------------------------------------------------------------------

def single_sector(seed=1, n_prim=200, scale=1.0) -> Event:
    """One sector (sector 0), 200 primaries over its 20 degree wedge, 5 % noise."""
    a = math.radians(10.0)
    return make_event(seed, int(round(n_prim * scale)), 0, pt_mean=0.6, noise_frac=0.05,
                      phi_lo=a - math.radians(10.0), phi_hi=a + math.radians(10.0), only_sector=0)


def pp_event(seed=2, scale=1.0) -> Event:
    """36 sectors, 60 primaries + 6 secondaries (10 %), 5 % noise (~10 k clusters)."""
    n = max(1, int(round(60 * scale)))
    return make_event(seed, n, max(0, int(round(0.1 * n))), pt_mean=0.6, noise_frac=0.05)


def central_event(seed=3, scale=1.0) -> Event:
    """36 sectors, 10,000 primaries (pT mean 0.5) + 3,000 secondaries, 10 % noise."""
    return make_event(seed, int(round(10000 * scale)), int(round(3000 * scale)), pt_mean=0.5,
                      noise_frac=0.10)


def min_bias_event(seed, scale=1.0) -> Event:
    """One min-bias collision: N(b) primaries, 30 % secondaries, 10 % noise."""
    rng = np.random.default_rng(seed)
    n = max(1, int(round(min_bias_tracks(rng) * scale)))
    return make_event(int(rng.integers(1 << 62)), n, int(round(0.3 * n)), pt_mean=0.5,
                      noise_frac=0.10)


def time_frame(seed=4, n_coll=50, scale=1.0) -> Event:
    """Continuous-readout time-frame: n_coll min-bias collisions overlaid, each
    shifted by a drift-time offset dz ~ U[-250, 250] cm applied as
    z' = z + sign(z) * dz; clusters whose |z'| > 250 or whose sign flips are
    dropped.  10 % noise on top."""
    rng = np.random.default_rng(seed)
    secs, rows, ys, zs, labs, tys, tzs, tss, trks = [], [], [], [], [], [], [], [], []
    lab_off = 0
    coll_dz, track_coll = [], []
    for c in range(n_coll):
        n = max(1, int(round(min_bias_tracks(rng) * scale)))
        ev = make_event(int(rng.integers(1 << 62)), n, int(round(0.3 * n)), pt_mean=0.5,
                        noise_frac=0.0)
        dz = rng.uniform(-Z_MAX, Z_MAX)
        sec, row, y, z, lab, ty, tz, ts = _unpack(ev)
        sgn = np.where(sec < 18, 1.0, -1.0)
        z2 = z + sgn * dz
        tz2 = tz + sgn * dz
        keep = (np.abs(z2) <= Z_MAX) & (z2 * sgn >= 0.0)
        secs.append(sec[keep]); rows.append(row[keep]); ys.append(y[keep]); zs.append(z2[keep])
        labs.append(np.where(lab[keep] >= 0, lab[keep] + lab_off, -1))
        tys.append(ty[keep]); tzs.append(tz2[keep]); tss.append(ts[keep])
        trks.append(ev.tracks)
        coll_dz.append(dz)
        track_coll.append(np.full(len(ev.tracks), c, np.int32))
        lab_off += len(ev.tracks)
    tracks = Tracks.concat(trks)
    base = Event(np.zeros((0, 4), np.float32), np.zeros(N_SECTORS * N_ROWS, np.int32),
                 np.zeros(0, np.int32), np.zeros(0), np.zeros(0), np.zeros(0), tracks, 0.5)
    ev = _rebuild(rng, base, np.concatenate(secs), np.concatenate(rows), np.concatenate(ys),
                  np.concatenate(zs), np.concatenate(labs), np.concatenate(tys),
                  np.concatenate(tzs), np.concatenate(tss))
    ev = _add_noise(rng, ev, int(round(0.10 * ev.n)))
    # truth of the overlay: each collision's drift offset, each track's collision
    ev.coll_dz = np.array(coll_dz)
    ev.track_coll = np.concatenate(track_coll) if track_coll else np.zeros(0, np.int32)
    return ev


def concat_events(events):
    """Batch layout: clusters concatenated in event order, row_counts [E * 36 * 159]."""
    cl = np.concatenate([e.clusters for e in events]) if events else np.zeros((0, 4), np.float32)
    rc = np.concatenate([e.row_counts for e in events]) if events else np.zeros(0, np.int32)
    return np.ascontiguousarray(cl), np.ascontiguousarray(rc)


def tiny_lattice_events(n_events, seed):
    """Many tiny events for exhaustive parity: in each, one random sector gets
    a patch of 3-30 consecutive pad rows with up to 50 clusters a row whose y
    and z lie on a 0.05 cm lattice (|y| <= 1.5 cm, |z| in [10, 13] cm), so
    that clusters at identical positions and exact distance ties are common,
    plus up to three lines of one cluster per row (so that chains and
    tracklets form).  Cluster ids are a random permutation.  Returns the batch
    layout (clusters, row_counts [n_events * 36 * 159])."""
    rng = np.random.default_rng(seed)
    xr = row_x()
    rcs, cls = [], []
    for _ in range(n_events):
        rc = np.zeros(N_SECTORS * N_ROWS, np.int32)
        sec = int(rng.integers(0, N_SECTORS))
        nr = int(rng.integers(3, 31))
        r0 = int(rng.integers(0, N_ROWS - nr + 1))
        n_lines = int(rng.integers(0, 4))
        ly = rng.integers(-20, 21, n_lines) * 0.05
        lsl = rng.integers(-2, 3, n_lines) * 0.05
        lz = rng.integers(200, 261, n_lines) * 0.05
        side = 1.0 if sec < N_SECTORS // 2 else -1.0
        for j in range(nr):
            r = r0 + j
            k = int(rng.integers(0, 51 - 2 * n_lines)) if j % 7 else int(rng.integers(0, 6))
            y = np.concatenate([rng.integers(-30, 31, k) * 0.05, ly + lsl * j])
            z = np.concatenate([rng.integers(200, 261, k) * 0.05, lz])
            rc[sec * N_ROWS + r] = len(y)
            c = np.zeros((len(y), 4), np.float32)
            c[:, 0] = xr[r]
            c[:, 1] = y
            c[:, 2] = side * z
            cls.append(c)
        rcs.append(rc)
    cl = np.concatenate(cls) if cls else np.zeros((0, 4), np.float32)
    cl.view(np.uint32)[:, 3] = rng.permutation(len(cl)).astype(np.uint32)
    return np.ascontiguousarray(cl), np.concatenate(rcs)
