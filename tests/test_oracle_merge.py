"""Pins of the track-merging oracle (Phase II step 3 of Sec. 2, Table 1 row
3: matching by covariance) against things other than itself: the
generator's exact crossings in two sector frames, finite differences, a
linear-algebra chi2, chi2 statistics of true split pairs (in a sector and
across a border), and hand-built cases of the pairing rule."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_09430_gb300 import synth as S

XR = S.row_x()
BZ = 0.5
C20 = math.cos(math.radians(20.0))
S20 = math.sin(math.radians(20.0))


def _tracks(rng, n, pt_lo=0.3, pt_hi=3.0, phi_lo=0.0, phi_hi=2 * math.pi):
    pt = np.exp(rng.uniform(math.log(pt_lo), math.log(pt_hi), n))
    phi = rng.uniform(phi_lo, phi_hi, n)
    tanl = rng.uniform(-0.9, 0.9, n)
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    z0 = np.zeros(n)
    return S.Tracks(z0, z0.copy(), z0.copy(), phi, pt, tanl, q)


def _by_sector(cr, m):
    sel = cr["track"] == m
    out = {}
    for s in np.unique(cr["sector"][sel]):
        ss = sel & (cr["sector"] == s)
        o = np.argsort(cr["row"][ss])
        out[int(s)] = {k: v[ss][o] for k, v in cr.items()}
    return out


def _theta(sa, sb):
    """Rotation from sector sa's frame to sector sb's (adjacent, one side)."""
    la, lb = sa % 18, sb % 18
    return 1 if lb == (la + 1) % 18 else (-1 if lb == (la + 17) % 18 else 0)


def _border_pairs(rng, n, min_rows=12):
    tr = _tracks(rng, n)
    cr = S.crossings(tr, BZ)
    pairs = []
    for m in range(len(tr)):
        secs = _by_sector(cr, m)
        ks = sorted(secs, key=lambda s: secs[s]["row"][0])
        for sa, sb in zip(ks, ks[1:]):
            if sa // 18 != sb // 18 or _theta(sa, sb) == 0:
                continue
            a, b = secs[sa], secs[sb]
            if len(a["row"]) < min_rows or len(b["row"]) < min_rows:
                continue
            if np.any(np.diff(a["row"]) != 1) or np.any(np.diff(b["row"]) != 1):
                continue
            pairs.append((m, sa, sb, a, b))
    return tr, pairs


# ----------------------------------------------------------------- rotation

def test_rotation_lands_on_the_next_sector_crossing():
    """A state at a track's last crossing in one sector, rotated into the
    adjacent sector's frame and propagated to the track's first crossing
    there, equals the generator's crossing (y, sin phi exact; z within the
    arc-series bound)."""
    rng = np.random.default_rng(31)
    tr, pairs = _border_pairs(rng, 3000, min_rows=3)
    fp = oracle.fit_params(BZ)
    n = 0
    for m, sa, sb, a, b in pairs:
        th = _theta(sa, sb)
        qpt = tr.q[m] / tr.pt[m]
        v = oracle.merge_vec(XR[a["row"][-1]], [a["y"][-1], a["z"][-1], a["sphi"][-1], tr.tanl[m], qpt])
        ok, w = oracle.merge_rotate(v, C20, th * S20, fp)
        if not ok:
            continue
        ok, w = oracle.merge_propagate(w, XR[b["row"][0]], fp)
        if not ok:
            continue
        assert abs(w[1] - b["y"][0]) < 1e-9, (w[1], b["y"][0])
        assert abs(w[3] - b["sphi"][0]) < 1e-11
        assert abs(w[2] - b["z"][0]) < 1e-7
        n += 1
    assert n > 200


@pytest.mark.parametrize("sign", [1, -1])
def test_rotation_jacobian_matches_finite_differences(sign):
    """Every column of the rotation's Jacobian: with C = e_k e_k^T the
    rotated covariance is J[:, k] J[:, k]^T; compare with central
    differences of (rotate, then step back to the unperturbed plane)."""
    rng = np.random.default_rng(32)
    fp = oracle.fit_params(BZ)
    for _ in range(100):
        x = rng.uniform(90, 240)
        p0 = np.array([rng.uniform(-0.15, 0.15) * x, rng.uniform(-100, 100), rng.uniform(-0.6, 0.6),
                       rng.uniform(-1, 1), rng.uniform(-3, 3)])
        ok, w0 = oracle.merge_rotate(oracle.merge_vec(x, p0), C20, sign * S20, fp)
        if not ok:
            continue
        for k in range(5):
            C5 = np.zeros((5, 5))
            C5[k, k] = 1.0
            _, w = oracle.merge_rotate(oracle.merge_vec(x, p0, C5), C20, sign * S20, fp)
            Cr = w[6:].reshape(5, 5)
            jk = Cr[:, k] / math.sqrt(Cr[k, k])
            h = 1e-6 * max(1.0, abs(p0[k]))
            outs = []
            for sgn in (1, -1):
                pp = p0.copy()
                pp[k] += sgn * h
                _, wr = oracle.merge_rotate(oracle.merge_vec(x, pp), C20, sign * S20, fp)
                _, wr = oracle.merge_propagate(wr, w0[0], fp)
                outs.append(wr[1:6])
            fd = (outs[0] - outs[1]) / (2 * h)
            assert np.allclose(jk, fd, rtol=1e-5, atol=1e-7), (k, jk, fd)


# --------------------------------------------------------------------- chi2

def test_chi2_equals_linear_algebra():
    rng = np.random.default_rng(33)
    for _ in range(200):
        A = rng.normal(size=(5, 5))
        B = rng.normal(size=(5, 5))
        Ca, Cb = A @ A.T + 0.01 * np.eye(5), B @ B.T + 0.01 * np.eye(5)
        pa, pb = rng.normal(size=5), rng.normal(size=5)
        ok, c2 = oracle.merge_chi2(oracle.merge_vec(100, pa, Ca), oracle.merge_vec(100, pb, Cb))
        d = pa - pb
        assert ok and abs(c2 - d @ np.linalg.solve(Ca + Cb, d)) < 1e-9 * max(1.0, c2)
    # not positive definite: refused
    ok, _ = oracle.merge_chi2(oracle.merge_vec(100, np.zeros(5), -np.eye(5)),
                              oracle.merge_vec(100, np.zeros(5), np.zeros((5, 5))))
    assert not ok


# ------------------------------------------------ statistics of true pairs

def _refit_segment(c, tr, m, rng, fp):
    xs = XR[c["row"]]
    y = c["y"] + S.SIGMA * rng.normal(size=len(xs))
    z = c["z"] + S.SIGMA * rng.normal(size=len(xs))
    cl = np.stack([xs, y, z, np.zeros_like(xs)], axis=1).astype(np.float32)
    st6 = np.array([np.float32(xs[0]), c["y"][0], c["z"][0], c["sphi"][0], tr.tanl[m], tr.q[m] / tr.pt[m]])
    f = oracle.refit_lists(st6[None], np.array([0, len(xs)]), np.arange(len(xs)), cl, fp)[0]
    return f, float(np.float32(xs[-1]))


def test_split_pairs_chi2_in_sector():
    """Tracks split by a 20-row gap in one sector: every pair is merged, and
    the link chi2 follows chi2 with 5 degrees of freedom (mean 5)."""
    rng = np.random.default_rng(34)
    tr = _tracks(rng, 1500, pt_lo=0.4, pt_hi=5.0)
    cr = S.crossings(tr, BZ)
    fp = oracle.fit_params(BZ)
    units, fits, xl = [], [], []
    for m in range(len(tr)):
        for s, c in _by_sector(cr, m).items():
            if len(c["row"]) < 100 or np.any(np.diff(c["row"]) != 1):
                continue
            ev = len(units) // 2
            for sl in (slice(0, 40), slice(60, None)):
                cc = {k: v[sl] for k, v in c.items()}
                f, x_last = _refit_segment(cc, tr, m, rng, fp)
                units.append(ev * 36 + s)
                fits.append(f)
                xl.append(x_last)
            break
    fits = np.array(fits)
    nxt, chi = oracle.merge_tracks(np.array(units), fits, np.array(xl), fp)
    a = np.arange(0, len(units), 2)
    assert len(a) > 300
    assert np.mean(nxt[a] == a + 1) > 0.99
    c2 = chi[a][nxt[a] == a + 1]
    assert 4.5 < c2.mean() < 5.5, c2.mean()
    assert np.all(nxt[a + 1] == -1)


def test_split_pairs_chi2_across_sector_border():
    """The two segments of a track in adjacent sectors: merged, with the
    link chi2 of mean 5 (rotation, its Jacobian and the propagated
    covariance consistent)."""
    rng = np.random.default_rng(35)
    tr, pairs = _border_pairs(rng, 6000, min_rows=15)
    fp = oracle.fit_params(BZ)
    units, fits, xl = [], [], []
    for i, (m, sa, sb, a, b) in enumerate(pairs):
        for s, c in ((sa, a), (sb, b)):
            f, x_last = _refit_segment(c, tr, m, rng, fp)
            units.append(i * 36 + s)
            fits.append(f)
            xl.append(x_last)
    units = np.array(units)
    # canonical order: by unit (the pair's two sectors may come in either order)
    o = np.argsort(units, kind="stable")
    inv = np.empty_like(o)
    inv[o] = np.arange(len(o))
    nxt, chi = oracle.merge_tracks(units[o], np.array(fits)[o], np.array(xl)[o], fp)
    ia, ib = inv[0::2], inv[1::2]
    assert len(ia) > 200
    linked = nxt[ia] == ib
    assert linked.mean() > 0.97, linked.mean()
    c2 = chi[ia][linked]
    assert 4.5 < c2.mean() < 5.6, c2.mean()


# ----------------------------------------------------------- pairing rule

def _fit_row(x, p, var=1e-4):
    f = np.zeros(oracle.N_FIT)
    f[0] = x
    f[1:6] = p
    C5 = np.eye(5) * var
    f[6:21] = [C5[i][j] for i in range(5) for j in range(i + 1)]
    return f


def _outer_of(p_in, x_in, x_out, fp):
    ok, w = oracle.merge_propagate(oracle.merge_vec(x_in, p_in), x_out, fp)
    assert ok
    return w[1:6]


def test_pairing_mutual_best_and_ties():
    fp = oracle.fit_params(BZ)
    pa = np.array([1.0, 20.0, 0.05, 0.2, 0.5])
    xb = 170.0
    pb = _outer_of(pa, 100.0, xb, fp)
    # A (inner) and two outer candidates: B1 exact, B2 off by 2 sigma in y
    off = pb.copy()
    off[0] += 0.02
    fits = np.array([_fit_row(100.0, pa), _fit_row(xb, pb), _fit_row(xb, off)])
    units = np.zeros(3, np.int32)
    xl = np.array([120.0, 190.0, 190.0])
    nxt, chi = oracle.merge_tracks(units, fits, xl, fp)
    assert list(nxt) == [1, -1, -1] and chi[0] < 1e-6
    # identical candidates: the smaller index wins
    fits2 = np.array([_fit_row(100.0, pa), _fit_row(xb, off), _fit_row(xb, off)])
    nxt, _ = oracle.merge_tracks(units, fits2, xl, fp)
    assert list(nxt) == [1, -1, -1]
    # two inner tracks prefer the same outer one: only the mutual best links,
    # even though the other inner track has a compatible second choice
    pa2 = pa.copy()
    pa2[0] += 0.01
    pc = _outer_of(pa2, 100.0, xb, fp)
    pc[0] += 0.03
    fits3 = np.array([_fit_row(100.0, pa), _fit_row(100.0, pa2), _fit_row(xb, pb), _fit_row(xb, pc)])
    nxt, _ = oracle.merge_tracks(np.zeros(4, np.int32), fits3, np.array([120.0, 120.0, 190, 190]), fp)
    assert nxt[0] == 2 and nxt[1] == -1


def test_candidate_geometry():
    fp = oracle.fit_params(BZ)
    pa = np.array([1.0, 20.0, 0.05, 0.2, 0.5])
    xb = 170.0
    pb = _outer_of(pa, 100.0, xb, fp)
    fits = np.array([_fit_row(100.0, pa), _fit_row(xb, pb)])
    for xl_a, expect in ((120.0, 1), (169.9, 1), (170.0, -1), (119.0, -1), (100.0, -1)):
        nxt, _ = oracle.merge_tracks(np.zeros(2, np.int32), fits, np.array([xl_a, 190.0]), fp)
        assert nxt[0] == expect, (xl_a, nxt)
    # other event, other side, non-adjacent sector: never
    for ub in (36, 18, 2):
        nxt, _ = oracle.merge_tracks(np.array([0, ub]), fits, np.array([120.0, 190.0]), fp)
        assert nxt[0] == -1
    # outside the y window (5 cm) after propagation: never, whatever the chi2
    far = pb.copy()
    far[0] += 5.5
    fw = np.array([_fit_row(100.0, pa), _fit_row(xb, far, var=100.0)])
    nxt, _ = oracle.merge_tracks(np.zeros(2, np.int32), fw, np.array([120.0, 190.0]), fp)
    assert nxt[0] == -1
    nxt, _ = oracle.merge_tracks(np.zeros(2, np.int32), fw, np.array([120.0, 190.0]), fp,
                                 mp=oracle.merge_params(window=6.0))
    assert nxt[0] == 1
    # the same in z
    far_z = pb.copy()
    far_z[1] += 5.5
    fz = np.array([_fit_row(100.0, pa), _fit_row(xb, far_z, var=100.0)])
    nxt, _ = oracle.merge_tracks(np.zeros(2, np.int32), fz, np.array([120.0, 190.0]), fp)
    assert nxt[0] == -1
    nxt, _ = oracle.merge_tracks(np.zeros(2, np.int32), fz, np.array([120.0, 190.0]), fp,
                                 mp=oracle.merge_params(window=6.0))
    assert nxt[0] == 1
    # a failed fit never merges
    f2 = fits.copy()
    f2[1, 23] = 1
    nxt, _ = oracle.merge_tracks(np.zeros(2, np.int32), f2, np.array([120.0, 190.0]), fp)
    assert nxt[0] == -1


def test_border_candidates_side_and_rotation_point():
    """Across a border: B is A's continuation rotated into the adjacent
    sector.  Linked when B's sector is adjacent on the same side, never on
    the other side.  A curling track is rotated at its outermost cluster:
    at its innermost one the direction in B's frame would exceed s_max."""
    fp = oracle.fit_params(BZ)
    # phi falls from ~64 deg at x = 100 to ~15 deg at x = 140 (k ~ 0.0198/cm)
    pa = np.array([10.0, 20.0, 0.9, 0.3, 13.2])
    ok, w = oracle.merge_propagate(oracle.merge_vec(100.0, pa), 140.0, fp)
    assert ok and 0.1 < w[3] < 0.4
    ok, w = oracle.merge_rotate(w, C20, -S20, fp)   # into the previous sector
    assert ok
    ok, wb = oracle.merge_propagate(w, 146.0, fp)
    assert ok
    # rotating at the innermost cluster instead fails the s_max check
    assert not oracle.merge_rotate(oracle.merge_vec(100.0, pa), C20, -S20, fp)[0]
    fits = np.array([_fit_row(100.0, pa), _fit_row(146.0, wb[1:6])])
    xl = np.array([140.0, 190.0])
    # A in sector 1, B in sector 0 (theta = -20 deg): linked
    nxt, _ = oracle.merge_tracks(np.array([0, 1]), fits[::-1], xl[::-1], fp)
    assert nxt[1] == 0
    # B in sector 18 (side C, next to sector 1 in the azimuth): never
    nxt, _ = oracle.merge_tracks(np.array([1, 18]), fits, xl, fp)
    assert nxt[0] == -1
