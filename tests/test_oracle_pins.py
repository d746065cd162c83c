"""Pins of the CPU oracle against things other than itself.

Each test names the function of oracle/tpc_oracle.c it pins and the
external fact it uses: the generator's closed-form helix, finite differences,
the Bayesian posterior in information form, weighted least squares, exact
fixed points, hand-built neighbour cases and invariants the method states
(at most one track hypothesis per hit, Sec. 2; seeds of at least 3 clusters,
Sec. 2 step 1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1712_09430_gb300 import synth as S

XR = S.row_x()
BZ = 0.5


def _tracks(rng, n, pt_lo=0.1, pt_hi=5.0, vtx=0.0):
    pt = np.exp(rng.uniform(math.log(pt_lo), math.log(pt_hi), n))
    phi = rng.uniform(math.radians(2), math.radians(18), n)
    tanl = rng.uniform(-1.0, 1.0, n)
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    vx = rng.uniform(-vtx, vtx, n)
    vy = rng.uniform(-vtx, vtx, n)
    vz = rng.uniform(-vtx, vtx, n)
    return S.Tracks(vx, vy, vz, phi, pt, tanl, q)


def _rows_of_track(cr, m, sector):
    sel = (cr["track"] == m) & (cr["sector"] == sector)
    o = np.argsort(cr["row"][sel])
    return {k: v[sel][o] for k, v in cr.items()}


# ---------------------------------------------------------------- generator

def test_generator_crossings_lie_on_lab_helix():
    """Every noise-free crossing is the lab helix point at the returned path
    length, rotated into the sector frame, on the pad-row plane."""
    rng = np.random.default_rng(11)
    tr = S.gen_tracks(rng, 300, 100, pt_mean=0.5)
    cr = S.crossings(tr, BZ)
    X, Y, Z = S.helix_lab(tr, BZ, cr["track"], cr["path"])
    a = S.sector_alpha(cr["sector"])
    xl = X * np.cos(a) + Y * np.sin(a)
    yl = -X * np.sin(a) + Y * np.cos(a)
    assert np.max(np.abs(xl - XR[cr["row"]])) < 1e-9
    assert np.max(np.abs(yl - cr["y"])) < 1e-9
    assert np.max(np.abs(Z - cr["z"])) < 1e-9
    # direction: numerical derivative of the lab helix, local frame
    h = 1e-5
    X1, Y1, _ = S.helix_lab(tr, BZ, cr["track"], cr["path"] + h)
    X0, Y0, _ = S.helix_lab(tr, BZ, cr["track"], cr["path"] - h)
    dyl = (-(X1 - X0) * np.sin(a) + (Y1 - Y0) * np.cos(a)) / (2 * h)
    assert np.max(np.abs(dyl - cr["sphi"])) < 1e-7
    assert np.all(np.abs(cr["y"]) <= XR[cr["row"]] * S.TAN_HALF_OPEN)
    # side A sectors hold z >= 0, side C z < 0
    assert np.all((cr["z"] >= 0) == (cr["sector"] < 18))


def test_generator_lorentz_sign():
    """A positive charge in +Bz moving along +x bends towards -y (F = q v x B)."""
    tr = S.Tracks(np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(1), np.array([0.3]),
                  np.zeros(1), np.array([1.0]))
    X, Y, _ = S.helix_lab(tr, BZ, np.array([0]), np.array([10.0]))
    assert X[0] > 0 and Y[0] < 0


def test_generator_sizes():
    e = S.pp_event()
    assert abs(e.n - 10000) < 1000
    assert e.row_counts.sum() == e.n and len(e.row_counts) == 36 * 159
    ids = e.ids
    assert len(np.unique(ids)) == e.n
    # x of each cluster is its row plane
    rows = np.repeat(np.arange(36 * 159), e.row_counts) % 159
    assert np.all(e.clusters[:, 0] == XR[rows].astype(np.float32))


def test_tiny_lattice_events_carry_ties():
    """The exhaustive parity inputs: valid layout, and rows with clusters at
    identical positions (so that the tie rules decide links) in most events."""
    cl, rc = S.tiny_lattice_events(200, seed=12)
    assert rc.size == 200 * 36 * 159 and int(rc.sum()) == len(cl)
    rows = np.repeat(np.arange(rc.size), rc)
    assert np.all(cl[:, 0] == XR[rows % 159].astype(np.float32))
    sec = (rows // 159) % 36
    assert np.all((cl[:, 2] > 0) == (sec < 18))
    assert len(np.unique(cl.view(np.uint32)[:, 3])) == len(cl)
    dup_events = set()
    off = np.concatenate([[0], np.cumsum(rc)])
    for rr in np.nonzero(rc > 1)[0]:
        yz = cl[off[rr]:off[rr + 1], 1:3]
        if len(np.unique(yz, axis=0)) < len(yz):
            dup_events.add(rr // (36 * 159))
    assert len(dup_events) > 100


# -------------------------------------------------------------- propagation

@pytest.mark.parametrize("inward,bz", [(False, BZ), (True, BZ), (False, -BZ), (True, -BZ)])
def test_propagate_follows_exact_helix(inward, bz):
    """orc_prop: one pad-row step from the exact state at row r lands on the
    exact crossing at the next row, outward and inward, in either field
    direction.  y and sin(phi) are exact; z is exact up to the first
    neglected term of the arc series, |t L| (5/112) u^6.  A dropped u^2 or
    u^4 term, an unsigned chord or a wrong curvature sign exceeds that
    bound."""
    rng = np.random.default_rng(5)
    tr = _tracks(rng, 200, vtx=20.0)
    cr = S.crossings(tr, bz)
    n_steps = 0
    u4_power = 0
    for m in range(len(tr)):
        k = -0.00299792458 * bz * tr.q[m] / tr.pt[m]
        for sec in np.unique(cr["sector"][cr["track"] == m]):
            c = _rows_of_track(cr, m, sec)
            for j in range(len(c["row"]) - 1):
                a, b = (j + 1, j) if inward else (j, j + 1)
                if abs(c["row"][a] - c["row"][b]) != 1:
                    continue
                qpt = tr.q[m] / tr.pt[m]
                v = oracle.state_vec(XR[c["row"][a]], c["y"][a], c["z"][a], c["sphi"][a],
                                     tr.tanl[m], qpt)
                ok, w = oracle.propagate(v, XR[c["row"][b]], bz)
                if not ok:
                    continue
                d = XR[c["row"][b]] - XR[c["row"][a]]
                chord = math.hypot(d, c["y"][b] - c["y"][a])
                u = k * chord / 2
                bound = abs(tr.tanl[m]) * chord * (5 / 112) * u ** 6 * 1.5 + 1e-12
                assert abs(w[1] - c["y"][b]) < 1e-11
                assert abs(w[3] - c["sphi"][b]) < 1e-12
                assert abs(w[2] - c["z"][b]) < bound, (abs(w[2] - c["z"][b]), bound)
                # the u^4 term is resolvable on this step
                if abs(tr.tanl[m]) * chord * 3 / 40 * u ** 4 > 100 * bound:
                    u4_power += 1
                n_steps += 1
    assert n_steps > 5000
    assert u4_power > 500


@pytest.mark.parametrize("inward", [False, True])
def test_propagate_straight_line_at_zero_field(inward):
    """Bz = 0 (the degenerate field of the method): a track is a straight
    line, so one pad-row step from the exact crossing keeps sin(phi) and q/pT,
    moves y by d tan(phi) and z by t times the chord, all exactly (up to
    rounding) on the generator's straight-line crossings."""
    rng = np.random.default_rng(8)
    tr = _tracks(rng, 100, vtx=20.0)
    cr = S.crossings(tr, 0.0)
    n_steps = 0
    for m in range(len(tr)):
        for sec in np.unique(cr["sector"][cr["track"] == m]):
            c = _rows_of_track(cr, m, sec)
            for j in range(len(c["row"]) - 1):
                a, b = (j + 1, j) if inward else (j, j + 1)
                if abs(c["row"][a] - c["row"][b]) != 1:
                    continue
                v = oracle.state_vec(XR[c["row"][a]], c["y"][a], c["z"][a], c["sphi"][a],
                                     tr.tanl[m], tr.q[m] / tr.pt[m])
                ok, w = oracle.propagate(v, XR[c["row"][b]], 0.0)
                if not ok:
                    continue
                assert c["sphi"][a] == c["sphi"][b] and w[3] == v[3] and w[5] == v[5]
                assert abs(w[1] - c["y"][b]) < 1e-10
                assert abs(w[2] - c["z"][b]) < 1e-10
                n_steps += 1
    assert n_steps > 2000


def test_propagate_multi_row_and_stop():
    rng = np.random.default_rng(6)
    tr = _tracks(rng, 50, pt_lo=0.5, pt_hi=5.0)
    cr = S.crossings(tr, BZ)
    for m in range(len(tr)):
        c = _rows_of_track(cr, m, cr["sector"][cr["track"] == m][0])
        if len(c["row"]) < 20:
            continue
        v = oracle.state_vec(XR[c["row"][0]], c["y"][0], c["z"][0], c["sphi"][0], tr.tanl[m],
                             tr.q[m] / tr.pt[m])
        for j in range(1, len(c["row"])):
            ok, v = oracle.propagate(v, XR[c["row"][j]], BZ)
            assert ok
        assert abs(v[1] - c["y"][-1]) < 1e-7 and abs(v[2] - c["z"][-1]) < 1e-7
    # |sin phi| beyond s_max fails and leaves the state untouched
    v = oracle.state_vec(100.0, 0.0, 0.0, 0.949, 0.0, 0.0)
    ok, w = oracle.propagate(v, 101.0, BZ)
    assert ok
    v = oracle.state_vec(100.0, 0.0, 0.0, 0.94, 0.0, -2.0)  # k = +0.003 per cm
    ok, w = oracle.propagate(v, 105.0, BZ)
    assert not ok and np.array_equal(w, v)


def _jac_from_transport(v0, x1, bz):
    """Columns of F read off the transported covariance of unit variances."""
    out = {}
    v = v0.copy(); v[6:15] = 0.0; v[8] = 1.0    # c11 (s) = 1
    _, w = oracle.propagate(v, x1, bz); out["a"] = w[7]          # c10' = dy/ds
    v = v0.copy(); v[6:15] = 0.0; v[11] = 1.0   # c22 (q) = 1
    _, w = oracle.propagate(v, x1, bz); out["b"] = w[9]; out["e"] = w[10]  # c20', c21'
    v = v0.copy(); v[6:15] = 0.0; v[14] = 1.0   # cz11 (t) = 1
    _, w = oracle.propagate(v, x1, bz); out["g"] = w[13]         # cz10' = dz/dt
    return out


@pytest.mark.parametrize("bz", [0.0, 0.5])
def test_transport_matches_finite_differences(bz):
    """Covariance transport uses the Jacobian of orc_prop: exact at Bz = 0 for
    dy/ds, exact always for ds/dq and dz/dt, and to the stated
    approximation order for dy/ds and dy/dq in a field."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        x = rng.uniform(85, 240)
        d = rng.choice([-1, 1]) * rng.uniform(0.5, 3.5)
        s = rng.uniform(-0.8, 0.8)
        t = rng.uniform(-1, 1)
        q = rng.uniform(-5, 5) if bz else 0.0
        v0 = oracle.state_vec(x, rng.uniform(-10, 10), rng.uniform(-100, 100), s, t, q)
        J = _jac_from_transport(v0, x + d, bz)

        def prop(dv):
            ok, w = oracle.propagate(v0 + dv, x + d, bz)
            assert ok
            return w
        hs, hq, ht = 1e-6, 1e-5, 1e-6
        e = np.zeros(15)
        e[3] = hs; fd_a = (prop(e)[1] - prop(-e)[1]) / (2 * hs)
        e[:] = 0; e[5] = hq
        fd_b = (prop(e)[1] - prop(-e)[1]) / (2 * hq)
        fd_e = (prop(e)[3] - prop(-e)[3]) / (2 * hq)
        e[:] = 0; e[4] = ht; fd_g = (prop(e)[2] - prop(-e)[2]) / (2 * ht)
        kB = -0.00299792458 * bz
        assert abs(J["e"] - kB * d) < 1e-15
        assert abs(J["e"] - fd_e) < 1e-9
        assert abs(J["g"] - fd_g) < 1e-7 * max(1.0, abs(fd_g))
        if bz == 0.0:
            assert abs(J["a"] - fd_a) < 1e-6 * max(1.0, abs(fd_a))
            assert J["b"] == 0.0
        else:
            assert abs(J["a"] - fd_a) < 2e-3 * abs(fd_a)
            assert np.sign(J["b"]) == np.sign(fd_b) and abs(J["b"] - fd_b) < 0.05 * abs(fd_b)


# ------------------------------------------------------------------- update

def test_update_equals_bayesian_posterior():
    """orc_update: posterior of the Gaussian prior (p, C) and one measurement
    of y (resp. z) with variance sigma^2, in information form; the chi2
    increment equals the minimised objective (prior term + residual term)."""
    rng = np.random.default_rng(8)
    P = oracle.default_params()
    sy2 = P.sigma_y ** 2
    sz2 = P.sigma_z ** 2
    for _ in range(200):
        A = rng.normal(size=(3, 3)); Cy = A @ A.T + 0.1 * np.eye(3)
        B = rng.normal(size=(2, 2)); Cz = B @ B.T + 0.1 * np.eye(2)
        py = rng.normal(size=3); pz = rng.normal(size=2)
        my, mz = rng.normal(), rng.normal()
        v = oracle.state_vec(100.0, py[0], pz[0], py[1], pz[1], py[2],
                             cy=(Cy[0, 0], Cy[1, 0], Cy[1, 1], Cy[2, 0], Cy[2, 1], Cy[2, 2]),
                             cz=(Cz[0, 0], Cz[1, 0], Cz[1, 1]))
        w, chi2 = oracle.update(v, my, mz)
        for C0, p0, m, s2, got_p, got_c in (
                (Cy, py, my, sy2, w[[1, 3, 5]], w[6:12]),
                (Cz, pz, mz, sz2, w[[2, 4]], w[12:15])):
            n = len(p0)
            H = np.zeros((1, n)); H[0, 0] = 1.0
            Ci = np.linalg.inv(C0)
            Cp = np.linalg.inv(Ci + H.T @ H / s2)
            pp = Cp @ (Ci @ p0 + H.T[:, 0] * m / s2)
            assert np.allclose(got_p, pp, rtol=1e-10, atol=1e-12)
            tri = [Cp[i, j] for i in range(n) for j in range(i + 1)]
            assert np.allclose(got_c, tri, rtol=1e-9, atol=1e-12)
        obj = 0.0
        for C0, p0, m, s2, pp in ((Cy, py, my, sy2, w[[1, 3, 5]]), (Cz, pz, mz, sz2, w[[2, 4]])):
            dp = pp - p0
            obj += dp @ np.linalg.inv(C0) @ dp + (m - pp[0]) ** 2 / s2
        assert abs(chi2 - obj) < 1e-9 * max(1.0, obj)


# ---------------------------------------------------------------------- fit

def test_fit_noise_free_helix_fixed_point():
    """Phase-2 fit on unsmeared helix hits, iterated from the previous result:
    converges to the generated parameters within 1e-9 relative (scale floor
    1 cm, 1 cm, 1, 1, 1 c/GeV)."""
    rng = np.random.default_rng(9)
    tr = _tracks(rng, 60, pt_lo=0.2, pt_hi=10.0, vtx=10.0)
    cr = S.crossings(tr, BZ)
    n_done = 0
    for m in range(len(tr)):
        secs = cr["sector"][cr["track"] == m]
        if len(secs) == 0:
            continue
        c = _rows_of_track(cr, m, np.bincount(secs).argmax())
        if len(c["row"]) < 30 or np.any(np.diff(c["row"]) != 1):
            continue
        rows = c["row"][::-1]
        y, z = c["y"][::-1], c["z"][::-1]
        qpt = tr.q[m] / tr.pt[m]
        # start: truth at the outermost hit, perturbed
        v = oracle.state_vec(XR[rows[0]], y[0] + 0.05, z[0] - 0.05, c["sphi"][-1] + 0.01,
                             tr.tanl[m] * 1.01, 0.8 * qpt)
        for it in range(30):
            n, w, chi2 = oracle.fit_hits(v, XR[rows], y, z, BZ)
            assert n == len(rows)
            # back to the outermost hit, row by row, for the next pass
            v = w
            for r in rows[::-1][1:]:
                ok, v = oracle.propagate(v, XR[r], BZ)
                assert ok
            truth = np.array([y[-1], z[-1], c["sphi"][0], tr.tanl[m], qpt])
            got = w[[1, 2, 3, 4, 5]]
            if np.all(np.abs(got - truth) <= 1e-9 * np.maximum(np.abs(truth), 1.0)):
                break
        else:
            pytest.fail(f"no convergence for track {m}: {got - truth}")
        assert abs(w[0] - XR[rows[-1]]) == 0.0
        n_done += 1
    assert n_done >= 20


def test_fit_z_block_bz0_is_weighted_least_squares():
    """Bz = 0 with exact y (so the arc lengths are exact): the (z, t) block is
    a linear filter, and its result at the last hit equals weighted least
    squares of z on the signed path length.  The reset prior on z (variance
    sigma_z^2 at the start point, centred on the first measurement) counts as
    a second measurement there; a large prior on t (var_t = 1e4) is
    negligible."""
    rng = np.random.default_rng(10)
    P = oracle.default_params(var_t=1e4)
    for _ in range(50):
        s = rng.uniform(-0.5, 0.5)
        tau = s / math.sqrt(1 - s * s)
        t = rng.uniform(-1, 1)
        rows = np.arange(158, 10, -1)
        x = XR[rows]
        y0, z0 = rng.uniform(-5, 5), rng.uniform(20, 100)
        y = y0 + tau * (x - x[0])
        path = (x - x[0]) / math.sqrt(1 - s * s)
        z = z0 + t * path + rng.normal(0, 0.1, len(x))
        v = oracle.state_vec(x[0], y[0], z[0], s, rng.uniform(-1, 1), 0.0)
        n, w, _ = oracle.fit_hits(v, x, y, z, 0.0, params=P)
        assert n == len(x)
        wts = np.ones(len(x)); wts[0] = 2.0
        b, a = np.polyfit(path, z, 1, w=np.sqrt(wts))
        assert abs(w[2] - (a + b * path[-1])) < 1e-9 * max(1.0, abs(w[2]))
        # t is dz per unit path; the path runs backwards (x decreasing)
        assert abs(w[4] - b) < 1e-9
        assert abs(w[1] - y[-1]) < 1e-9 and abs(w[3] - s) < 1e-12


def test_fit_y_block_bz0_fixed_point_is_least_squares_line():
    """Bz = 0 with smeared y: the (y, sin phi) block, iterated from its own
    result, settles on the weighted least-squares line y = a + b x (the reset
    prior on y, centred on the first measurement, counts as a second
    measurement there): y at the last hit = a + b x, sin phi = b / sqrt(1 + b^2).
    The block is nonlinear in sin phi (y' = y + d s / sqrt(1 - s^2)), so the
    filter meets the line only to second order in how far its running slope
    strays from the final one; a tight prior on s (variance 1e-6, centred on
    the previous pass) keeps that below 1e-3 and the gap below 1e-4 cm (a
    hundredth of the line's statistical error)."""
    rng = np.random.default_rng(11)
    P = oracle.default_params(var_s=1e-6)
    for _ in range(30):
        s = rng.uniform(-0.5, 0.5)
        tau = s / math.sqrt(1 - s * s)
        rows = np.arange(158, 10, -1)
        x = XR[rows]
        y = rng.uniform(-5, 5) + tau * (x - x[0]) + rng.normal(0, 0.1, len(x))
        z = 50.0 + 0.3 * (x - x[0])
        sv = s + 0.02
        for _ in range(40):
            v = oracle.state_vec(x[0], y[0], z[0], sv, 0.3, 0.0)
            n, w, _ = oracle.fit_hits(v, x, y, z, 0.0, params=P)
            assert n == len(x)
            done = abs(w[3] - sv) < 1e-14
            sv = w[3]
            if done:
                break
        else:
            pytest.fail("no fixed point")
        wts = np.ones(len(x)); wts[0] = 2.0
        b, a = np.polyfit(x, y, 1, w=np.sqrt(wts))
        assert abs(w[1] - (a + b * x[-1])) < 1e-4
        assert abs(w[3] - b / math.sqrt(1 + b * b)) < 1e-5


def test_chi2_per_ndf_is_one_on_smeared_isolated_tracks():
    """The full oracle on isolated smeared tracks without noise: mean
    chi2/ndf of the Phase-2 fits is 1 within 5 %."""
    vals = []
    for seed in range(40):
        ev = S.make_event(1000 + seed, 30, 0, pt_mean=1.0, noise_frac=0.0, eff=1.0)
        o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR)
        for k, t in enumerate(o["trk_t"]):
            n = o["tl_n"][t]
            if n >= 30:
                vals.append(o["tl_f"][t, 15] / (2 * n - 5))
    vals = np.array(vals)
    assert len(vals) > 1000
    assert 0.95 <= vals.mean() <= 1.05, vals.mean()


# --------------------------------------------------------------- neighbours

def _hand_event(clusters_by_row, sector=0):
    """clusters_by_row: list of (row, y, z, id) in one sector."""
    rc = np.zeros(36 * 159, np.int32)
    cl = sorted(clusters_by_row, key=lambda c: c[0])
    arr = np.zeros((len(cl), 4), np.float32)
    for i, (r, y, z, cid) in enumerate(cl):
        arr[i, 0] = np.float32(XR[r]); arr[i, 1] = y; arr[i, 2] = z
        arr.view(np.uint32)[i, 3] = cid
        rc[sector * 159 + r] += 1
    return arr, rc


def test_neighbours_collinear_triple_and_row_limits():
    # straight radial line y = 0, z = 10 on rows 0, 1, 2 and 156, 157, 158
    cl, rc = _hand_event([(0, 0.0, 10.0, 1), (1, 0.0, 10.0, 2), (2, 0.0, 10.0, 3),
                          (156, 0.0, 10.0, 4), (157, 0.0, 10.0, 5), (158, 0.0, 10.0, 6)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert list(o["up_raw"]) == [-1, 2, -1, -1, 5, -1]
    assert list(o["dn_raw"]) == [-1, 0, -1, -1, 3, -1]
    # rows 0 and 158 have no links of their own, so the cleaner drops all
    assert list(o["up"]) == [-1] * 6


def test_neighbours_exact_tie_goes_to_smaller_ids():
    # i on row 1 at y = 0; d on row 0 at y = 0; two up candidates at +-0.1,
    # tt = 0.5 so both give D = 0.05^2 exactly: the smaller up id wins.
    for id_a, id_b, want in ((7, 3, "b"), (3, 7, "a")):
        cl, rc = _hand_event([(0, 0.0, 10.0, 1), (1, 0.0, 10.0, 2),
                              (2, 0.1, 10.0, id_a), (2, -0.1, 10.0, id_b)])
        o = oracle.run(cl, rc, 1, BZ, XR)
        ys = cl[:, 1]
        u = o["up_raw"][1]
        assert u >= 0 and (ys[u] > 0) == (want == "a")
    # equal up, two equal-D down candidates: the smaller down id wins
    for id_a, id_b, want in ((9, 4, "b"), (4, 9, "a")):
        cl, rc = _hand_event([(0, 0.1, 10.0, id_a), (0, -0.1, 10.0, id_b), (1, 0.0, 10.0, 2),
                              (2, 0.0, 10.0, 3)])
        o = oracle.run(cl, rc, 1, BZ, XR)
        d = o["dn_raw"][2]
        assert d >= 0 and (cl[d, 1] > 0) == (want == "a")


def test_neighbours_cuts():
    # D cut: middle hit off the line by 0.6 cm in z -> D = 0.36 > 0.25: no link
    cl, rc = _hand_event([(0, 0.0, 10.0, 1), (1, 0.0, 10.6, 2), (2, 0.0, 10.0, 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == -1 and o["dn_raw"][1] == -1
    # just inside: 0.45 cm -> D = 0.2025 passes (windows are 1.125 cm)
    cl, rc = _hand_event([(0, 0.0, 10.0, 1), (1, 0.0, 10.45, 2), (2, 0.0, 10.0, 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == 2 and o["dn_raw"][1] == 0
    # window: the up candidate 1.2 cm away in y (W = 1.5 * 0.75 = 1.125) is no candidate
    cl, rc = _hand_event([(0, 0.0, 10.0, 1), (1, 0.0, 10.0, 2), (2, 1.2, 10.0, 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == -1
    # the window is centred on y_i * X_u / X_r (a line through the origin)
    yi = 20.0
    yu = np.float32(np.float32(yi) * (np.float32(XR[2]) / np.float32(XR[1])))
    yd = np.float32(np.float32(yi) * (np.float32(XR[0]) / np.float32(XR[1])))
    cl, rc = _hand_event([(0, yd, 10.0, 1), (1, yi, 10.0, 2), (2, yu, 10.0, 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == 2 and o["dn_raw"][1] == 0
    # a straight line whose slope differs from the radial one (y_i / X_r =
    # 0.117) by 1.45 < k_win: inside the windows centred on y_i * X/X_r
    # (offset 1.0875 cm < W = 1.125 cm), outside windows centred on y_i
    # (offset 1.175 cm)
    sl = 10.0 / XR[1] + 1.45
    cl, rc = _hand_event([(0, 10.0 - sl * 0.75, 10.0, 1), (1, 10.0, 10.0, 2),
                          (2, 10.0 + sl * 0.75, 10.0, 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == 2 and o["dn_raw"][1] == 0


def test_neighbours_where_the_row_pitch_changes():
    """N2/N3 across the pitch change at rows 62/63/64 (X = 131.5, 135, 136):
    the collinearity residual interpolates at tt = (X_r - X_d) / (X_u - X_d)
    = 7/9, and each window scales with its own row distance (W_d = 5.25,
    W_u = 1.5 cm)."""
    # a straight line in z (dz/dx = 0.5) links with D = 0; the midpoint
    # (tt = 1/2) would be 0.625 cm off the middle cluster
    z = lambda x: 10.0 + 0.5 * (x - XR[62])
    cl, rc = _hand_event([(62, 0.0, z(XR[62]), 1), (63, 0.0, z(XR[63]), 2), (64, 0.0, z(XR[64]), 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == 2 and o["dn_raw"][1] == 0
    # an up cluster 1.6 cm away in z is outside W_u = 1.5 although the pair
    # (D = 0.127 with a down cluster 4 cm away, inside W_d) would pass the cut
    cl, rc = _hand_event([(62, 0.0, 6.0, 1), (63, 0.0, 10.0, 2), (64, 0.0, 11.6, 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == -1 and o["dn_raw"][1] == -1
    cl, rc = _hand_event([(62, 0.0, 6.0, 1), (63, 0.0, 10.0, 2), (64, 0.0, 11.4, 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == 2 and o["dn_raw"][1] == 0


def test_neighbour_window_scales_with_row_distance():
    """N2: at the 1.5 cm pitch of the outer rows the window is 1.5 * 1.5 =
    2.25 cm: a collinear triple with 1.8 cm steps in y links."""
    cl, rc = _hand_event([(130, -1.8, 10.0, 1), (131, 0.0, 10.0, 2), (132, 1.8, 10.0, 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == 2 and o["dn_raw"][1] == 0


def test_neighbour_cut_is_inclusive():
    """N3: a pair with D exactly equal to D_max^2 = 0.25 (the middle cluster
    0.5 cm off the line in z) is kept."""
    cl, rc = _hand_event([(0, 0.0, 10.0, 1), (1, 0.0, 10.5, 2), (2, 0.0, 10.0, 3)])
    o = oracle.run(cl, rc, 1, BZ, XR)
    assert o["up_raw"][1] == 2 and o["dn_raw"][1] == 0


def test_cleaner_asymmetric_case():
    # A (row 2, y = 0) links up to B (row 3, y = 0.3) with D = 0.15^2, but B's
    # best pair is (E above, C below) on the line y = 0.3 with D = 0, so B
    # links down to C and the cleaner drops A -> B while keeping C <-> B.
    cl, rc = _hand_event([
        (1, 0.0, 10.0, 1),            # 0
        (2, 0.0, 10.0, 2),            # 1  A
        (2, 0.3, 10.0, 3),            # 2  C
        (3, 0.3, 10.0, 4),            # 3  B
        (4, 0.3, 10.0, 5),            # 4  E
    ])
    o = oracle.run(cl, rc, 1, BZ, XR)
    up, dn, up2, dn2 = o["up_raw"], o["dn_raw"], o["up"], o["dn"]
    assert up[1] == 3                       # A -> B
    assert dn[3] == 2                       # B -> C, not back to A
    assert up2[1] == -1                     # so the cleaner drops A -> B
    assert up2[2] == 3 and dn2[3] == 2      # C <-> B survives
    for i in range(len(cl)):
        if up2[i] >= 0:
            assert dn2[up2[i]] == i
        if dn2[i] >= 0:
            assert up2[dn2[i]] == i


# ------------------------------------------------------ event-level invariants

@pytest.fixture(scope="module")
def central_small():
    ev = S.central_event(seed=3, scale=0.05)
    return ev, oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR)


def test_links_symmetric_after_cleaning(central_small):
    ev, o = central_small
    up, dn = o["up"], o["dn"]
    i = np.nonzero(up >= 0)[0]
    assert np.all(dn[up[i]] == i)
    j = np.nonzero(dn >= 0)[0]
    assert np.all(up[dn[j]] == j)
    # links join adjacent rows only
    rows = np.repeat(np.arange(36 * 159), ev.row_counts) % 159
    assert np.all(rows[up[i]] == rows[i] + 1)


def test_start_hits_one_per_chain(central_small):
    ev, o = central_small
    up, dn = o["up"], o["dn"]
    seen = np.zeros(ev.n, bool)
    for s in o["start"]:
        assert up[s] >= 0 and dn[s] < 0
        n, j = 1, s
        assert not seen[j]
        seen[j] = True
        while up[j] >= 0:
            j = up[j]
            assert not seen[j]
            seen[j] = True
            n += 1
        assert n >= 3
    # every chain of length >= 3 has its start in the list
    starts = set(o["start"].tolist())
    for s in np.nonzero((up >= 0) & (dn < 0))[0]:
        n, j = 1, s
        while up[j] >= 0:
            j = up[j]; n += 1
        assert (n >= 3) == (s in starts)
    # canonical order: (unit, row, id) ascending
    rows = np.repeat(np.arange(36 * 159), ev.row_counts)
    key = rows[o["start"]].astype(np.int64) * (1 << 32) + ev.ids[o["start"]]
    assert np.all(np.diff(key) > 0)


def test_selection_single_owner_and_best_instance(central_small):
    _check_selection(*central_small)


def test_selection_rules_on_a_denser_event():
    """The same invariants where overlaps are common enough that some live
    tracklets own between half and 70 % of their clusters."""
    ev = S.central_event(seed=3, scale=0.5)
    _check_selection(ev, oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR))


def _check_selection(ev, o):
    """Sel1/Sel2 (readings): each cluster in at most one track; a track keeps
    only clusters its tracklet owns, owns >= 10 and >= 70 % of them; every
    cluster of a live tracklet is owned by the live tracklet with the largest
    key (more clusters, then smaller id); every rejected live tracklet fails
    a rule."""
    hits = o["trk_hits"]
    assert len(np.unique(hits)) == len(hits)      # each cluster in <= 1 track
    key = lambda t: (int(o["tl_n"][t]) << 32) | (0xFFFFFFFF - int(t))
    owner_of = {}
    for m, t in enumerate(o["trk_t"]):
        h = hits[o["trk_hit_off"][m]:o["trk_hit_off"][m + 1]]
        n = o["tl_n"][t]
        assert o["tl_alive"][t] and len(h) >= 10 and 10 * len(h) >= 7 * n
        th = o["tl_hits"][o["tl_hit_off"][t]:o["tl_hit_off"][t + 1]]
        assert set(h.tolist()) <= set(th.tolist())
        for x in h:
            owner_of[int(x)] = t
    # a hit of a live tracklet that it does not keep belongs to a live
    # tracklet with a larger key (more hits, or as many and a smaller id)
    by_hit = {}
    for t in np.nonzero(o["tl_alive"])[0]:
        for x in o["tl_hits"][o["tl_hit_off"][t]:o["tl_hit_off"][t + 1]]:
            by_hit.setdefault(int(x), []).append(int(t))
    for x, ts in by_hit.items():
        best = max(ts, key=key)
        if x in owner_of:
            assert owner_of[x] == best
    # every live tracklet that is not a track fails an acceptance rule
    acc = set(o["trk_t"].tolist())
    for t in np.nonzero(o["tl_alive"])[0]:
        if t in acc:
            continue
        th = o["tl_hits"][o["tl_hit_off"][t]:o["tl_hit_off"][t + 1]]
        owned = sum(1 for x in th if max(by_hit[int(x)], key=key) == t)
        assert owned < 10 or 10 * owned < 7 * o["tl_n"][t]


# ------------------------------------------- hand-built straight tracks

def _line_clusters(rows, sector=3, y0=2.0, b=0.05, z0=40.0, t=0.3):
    """Exact clusters of one straight track (zero field) on the given pad
    rows of one sector: y = y0 + b (x - X_0), z = z0 + t * path, ids 0.."""
    rows = np.asarray(rows)
    x = XR[rows].astype(np.float64)
    y = y0 + b * (x - XR[0])
    z = z0 + t * (x - XR[0]) * math.sqrt(1 + b * b)
    rc = np.zeros(36 * 159, np.int32)
    rc[sector * 159 + rows] = 1
    cl = np.zeros((len(rows), 4), np.float32)
    cl[:, 0] = x
    cl[:, 1] = y
    cl[:, 2] = z
    cl.view(np.uint32)[:, 3] = np.arange(len(rows))
    return cl, rc


def test_gap_of_g_max_empty_rows_is_bridged():
    """T6/T7: the search stops after more than g_max = 8 consecutive misses.
    A straight track with 8 empty rows in its middle is one track of all its
    clusters (both seed chains' tracklets cross the gap; the one with the
    smaller id wins); with 9 empty rows it is two tracks, split at the gap."""
    g_max = oracle.default_params().g_max
    assert g_max == 8
    for gap in (g_max, g_max + 1):
        inner, outer = np.arange(20, 50), np.arange(50 + gap, 81)
        cl, rc = _line_clusters(np.concatenate([inner, outer]))
        o = oracle.run(cl, rc, 1, 0.0, XR)
        tracks = sorted(sorted(o["trk_hits"][o["trk_hit_off"][m]:o["trk_hit_off"][m + 1]].tolist())
                        for m in range(len(o["trk_t"])))
        if gap == g_max:
            assert tracks == [list(range(len(cl)))]
        else:
            assert tracks == [list(range(len(inner))), list(range(len(inner), len(cl)))]


def test_shortest_kept_track_has_ten_clusters():
    """T8/Sel2: a straight track on exactly 10 rows is kept with all 10
    clusters; on 9 rows it is not."""
    for n, kept in ((10, True), (9, False)):
        cl, rc = _line_clusters(np.arange(30, 30 + n))
        o = oracle.run(cl, rc, 1, 0.0, XR)
        assert len(o["trk_t"]) == (1 if kept else 0)
        if kept:
            assert sorted(o["trk_hits"].tolist()) == list(range(n))


def test_phase2_covariance_is_a_fresh_fit_of_its_clusters():
    """T7: Phase 2 restarts from the reset covariance.  At Bz = 0 the (z, t)
    block is linear, so its covariance at the innermost cluster is the
    inverse information of the Phase-2 clusters alone (each sigma_z^2, the
    reset prior on z counting as one more measurement at the outermost
    cluster, and var_t on t); carrying Phase 1's information over would make
    it smaller."""
    p = oracle.default_params()
    b = 0.05
    rows = np.concatenate([np.arange(20, 50), np.arange(58, 81)])
    cl, rc = _line_clusters(rows, b=b)
    o = oracle.run(cl, rc, 1, 0.0, XR)
    assert len(o["trk_t"]) == 1 and o["trk_n"][0] == len(rows)
    x = XR[rows].astype(np.float64)
    path = (x - x[0]) * math.sqrt(1 + b * b)      # signed, from the innermost cluster
    H = np.stack([np.ones_like(path), path], axis=1)
    info = H.T @ H / p.sigma_z ** 2
    info += np.outer(H[-1], H[-1]) / p.sigma_z ** 2
    info[1, 1] += 1.0 / p.var_t
    C = np.linalg.inv(info)
    f = o["tl_f"][o["trk_t"][0]]
    assert f[0] == np.float32(XR[20])
    got = np.array([f[12], f[13], f[14]])
    want = np.array([C[0, 0], C[1, 0], C[1, 1]])
    assert np.allclose(got, want, rtol=1e-9, atol=0), (got, want)


def _tracklet_hits(o):
    return [o["tl_hits"][o["tl_hit_off"][t]:o["tl_hit_off"][t + 1]].tolist() for t in range(len(o["tl_n"]))]


@pytest.mark.parametrize("coord", [1, 2])
def test_search_window_floor(coord):
    """T5: the window half-width is at least w_min = 0.3 cm.  With n_sigma = 2
    the sigma window of Phase 2 after many clusters is ~0.21 cm, so a cluster
    0.25 cm off the line (in y, or in z) is taken only through the floor."""
    P = oracle.default_params(n_sigma=2.0)
    cl, rc = _line_clusters(np.arange(20, 81))
    k = 5                                            # row 25
    cl[k, coord] += np.float32(0.25)
    o = oracle.run(cl, rc, 1, 0.0, XR, params=P)
    assert len(o["trk_t"]) == 1 and k in o["trk_hits"].tolist()


@pytest.mark.parametrize("coord", [1, 2])
def test_search_window_ceiling(coord):
    """T5: the window half-width is at most w_max = 3 cm.  Phase 2 restarts
    from the reset covariance at the outermost cluster (row 80); three empty
    rows later its sigma window is ~7 cm in y and ~14 cm in z, so a lone
    cluster 3.5 cm off the line on row 76 is skipped only through the
    ceiling."""
    rows = np.concatenate([np.arange(20, 77), [80]])
    cl, rc = _line_clusters(rows)
    k = int(np.nonzero(rows == 76)[0][0])
    cl[k, coord] += np.float32(3.5)
    o = oracle.run(cl, rc, 1, 0.0, XR)
    assert len(o["trk_t"]) == 1
    assert sorted(o["trk_hits"].tolist()) == [i for i in range(len(rows)) if i != k]
    assert all(k not in h for h in _tracklet_hits(o))


def test_search_tie_goes_to_the_smaller_id():
    """T5: of two clusters at the same distance (the same position) the one
    with the smaller id is taken."""
    rows = np.arange(20, 81)
    cl, rc = _line_clusters(rows)
    k = int(np.nonzero(rows == 50)[0][0])
    dup = cl[k].copy()
    dup.view(np.uint32)[3] = len(cl)                 # a larger id than every other cluster
    cl = np.insert(cl, k + 1, dup, axis=0)
    rc[3 * 159 + 50] += 1
    o = oracle.run(cl, rc, 1, 0.0, XR)
    assert len(o["trk_t"]) == 1
    h = o["trk_hits"].tolist()
    assert k in h and k + 1 not in h


def test_search_distance_is_normalised_per_coordinate():
    """T5: candidates are ranked by dy^2 / S_y + dz^2 / S_z.  After Phase 2's
    reset and three empty rows S_z is ~4 S_y (var_t = 1, var_s = 0.25), so of
    two lone candidates on row 76, 0.4 cm off in y and 0.5 cm off in z, the
    z one is nearer (0.25 / 16 < 0.16 / 4); in cm it is the other way round."""
    rows = np.concatenate([np.arange(20, 76), [76, 76], [80]])
    cl, rc = _line_clusters(rows)
    rc[3 * 159 + 76] = 2
    a, b = int(np.nonzero(rows == 76)[0][0]), int(np.nonzero(rows == 76)[0][1])
    cl[a, 1] += np.float32(0.4)
    cl[b, 2] += np.float32(0.5)
    o = oracle.run(cl, rc, 1, 0.0, XR)
    took = [h for h in _tracklet_hits(o) if a in h or b in h]
    assert took and all(b in h and a not in h for h in took)


@pytest.mark.parametrize("beyond,kept", [(1.0, True), (3.0, False)])
def test_sector_edge_margin(beyond, kept):
    """T6: a prediction may lie up to y_margin = 2 cm beyond the sector edge
    |y| = X tan 10 deg before the search stops: a straight track running 1 cm
    beyond the edge is kept, one running 3 cm beyond it is not."""
    rows = np.arange(20, 81)
    cl, rc = _line_clusters(rows)
    cl[:, 1] = (XR[rows].astype(np.float64) * math.tan(math.radians(10.0)) + beyond).astype(np.float32)
    o = oracle.run(cl, rc, 1, 0.0, XR)
    assert len(o["trk_t"]) == (1 if kept else 0)


def test_phase1_misses_count_consecutive_rows():
    """T6: the miss count restarts at every cluster found.  A straight track
    with two gaps of 5 empty rows: the tracklet seeded on its inner part
    (the first in canonical order) crosses both in Phase 1 (10 misses in all,
    never more than 8 in a row) and keeps every cluster."""
    rows = np.concatenate([np.arange(20, 51), np.arange(56, 61), np.arange(66, 81)])
    cl, rc = _line_clusters(rows)
    o = oracle.run(cl, rc, 1, 0.0, XR)
    assert o["start"][0] == 1                        # the inner chain starts at row 21
    assert o["tl_n"][0] == len(rows)


def test_tracklet_clusters_ascend_by_row(central_small):
    """T7: a tracklet's clusters are stored in ascending row order, one per
    row."""
    ev, o = central_small
    rows = np.repeat(np.arange(36 * 159), ev.row_counts) % 159
    for t in range(len(o["tl_n"])):
        h = o["tl_hits"][o["tl_hit_off"][t]:o["tl_hit_off"][t + 1]]
        assert np.all(np.diff(rows[h]) > 0)


def test_isolated_tracks_links_follow_truth():
    """Sparse stiff tracks without noise: every cleaned link joins consecutive
    clusters of the same generated track."""
    ev = S.make_event(77, 20, 0, pt_mean=2.0, noise_frac=0.0, eff=1.0)
    o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR)
    i = np.nonzero(o["up"] >= 0)[0]
    assert len(i) > 1000
    assert np.all(ev.label[o["up"][i]] == ev.label[i])


def test_isolated_tracks_efficiency():
    import qa
    effs = []
    for seed in range(10):
        ev = S.make_event(500 + seed, 40, 0, pt_mean=1.0, noise_frac=0.0)
        o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR)
        q = qa.qa(ev.label, ev.row_counts, o["trk_hit_off"], o["trk_hits"])
        effs.append(q["eff"])
        assert q["fake"] == 0.0
    assert np.mean(effs) > 0.97


def test_fp32_exact_mode_is_float():
    assert oracle.lib("f32").orc_real_size() == 4
    assert oracle.lib("f64").orc_real_size() == 8
