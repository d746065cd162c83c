"""Pins of the refit oracle (oracle/tpc_refit.c) against things other than
itself: the generator's closed-form helix, finite differences, the Bayesian
posterior in information form, a Gauss-Newton least-squares step on the
closed-form helix (small-noise limit), exact fixed points, pull and chi2
statistics, and tracks integrated numerically (Runge-Kutta) through a
non-uniform field.

The refit is the final full Kalman filter fit of Sec. 2 ("Track fit",
Table 1 row 4) with a polynomial field (same passage)."""
import math

import numpy as np
import pytest

import oracle
from paper_1712_09430_gb300 import synth as S

XR = S.row_x()
BZ = 0.5
KAPPA = 0.00299792458


def _tracks(rng, n, pt_lo=0.2, pt_hi=5.0, vtx=0.0):
    pt = np.exp(rng.uniform(math.log(pt_lo), math.log(pt_hi), n))
    phi = rng.uniform(math.radians(2), math.radians(18), n)
    tanl = rng.uniform(-1.0, 1.0, n)
    q = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    vx = rng.uniform(-vtx, vtx, n)
    vy = rng.uniform(-vtx, vtx, n)
    vz = rng.uniform(-vtx, vtx, n)
    return S.Tracks(vx, vy, vz, phi, pt, tanl, q)


def _long_segments(tr, bz, min_rows=40):
    """Per track: the crossings in its dominant sector, rows consecutive."""
    cr = S.crossings(tr, bz)
    out = []
    for m in range(len(tr)):
        sel = cr["track"] == m
        if not np.any(sel):
            continue
        sec = np.bincount(cr["sector"][sel]).argmax()
        sel &= cr["sector"] == sec
        o = np.argsort(cr["row"][sel])
        c = {k: v[sel][o] for k, v in cr.items()}
        if len(c["row"]) < min_rows or np.any(np.diff(c["row"]) != 1):
            continue
        out.append((m, c))
    return out


def _truth_in(tr, m, c):
    """Truth state (x, y, z, s, t, q) at the innermost crossing."""
    return np.array([XR[c["row"][0]], c["y"][0], c["z"][0], c["sphi"][0], tr.tanl[m],
                     tr.q[m] / tr.pt[m]])


def refit_double(st6, x, y, z, fp, mode="f64"):
    """The two passes of the refit (outward from st6, then inward from the
    outermost hit), driven through orc_refit_propagate / orc_refit_update in
    double precision so the pins are not limited by float32 cluster input.
    The per-track routine orc_refit_tracks runs the same sequence (checked
    below in test_refit_tracks_equals_step_sequence)."""
    n = len(x)
    v = oracle.fit_vec(st6[0], st6[1:6])

    def init(v, k):
        v = v.copy()
        v[1], v[2] = y[k], z[k]
        v[6:] = np.diag(np.sqrt([fp.sigma_y ** 2, fp.sigma_z ** 2, fp.var_s, fp.var_t,
                                 fp.var_q])).reshape(25)
        return v

    chi2 = 0.0
    for k in range(n):
        ok, v = oracle.refit_propagate(v, x[k], fp, mode)
        assert ok
        if k == 0:
            v, chi2 = init(v, k), 0.0
        else:
            v, chi2 = oracle.refit_update(v, y[k], z[k], fp, mode, chi2)
    for j in range(n):
        k = n - 1 - j
        ok, v = oracle.refit_propagate(v, x[k], fp, mode)
        assert ok
        if j == 0:
            v, chi2 = init(v, k), 0.0
        else:
            v, chi2 = oracle.refit_update(v, y[k], z[k], fp, mode, chi2)
    return v, chi2


# ------------------------------------------------------------- propagation

@pytest.mark.parametrize("inward,bz", [(False, BZ), (True, BZ), (False, -BZ), (True, -BZ)])
def test_refit_propagate_follows_exact_helix(inward, bz):
    """orc_refit_propagate (uniform field, either direction): one pad-row step
    from the exact state at row r lands on the generator's closed-form
    crossing at the next row; z within the first neglected term of the arc
    series."""
    rng = np.random.default_rng(21)
    tr = _tracks(rng, 150, pt_lo=0.1, vtx=20.0)
    fp = oracle.fit_params(bz)
    n_steps = 0
    for m, c in _long_segments(tr, bz, min_rows=5):
        k = -KAPPA * bz * tr.q[m] / tr.pt[m]
        for j in range(len(c["row"]) - 1):
            a, b = (j + 1, j) if inward else (j, j + 1)
            v = oracle.fit_vec(XR[c["row"][a]], [c["y"][a], c["z"][a], c["sphi"][a], tr.tanl[m],
                                                 tr.q[m] / tr.pt[m]])
            ok, w = oracle.refit_propagate(v, XR[c["row"][b]], fp)
            if not ok:
                continue
            d = XR[c["row"][b]] - XR[c["row"][a]]
            chord = math.hypot(d, c["y"][b] - c["y"][a])
            u = k * chord / 2
            bound = abs(tr.tanl[m]) * chord * (5 / 112) * u ** 6 * 1.5 + 1e-12
            assert abs(w[0] - XR[c["row"][b]]) == 0.0
            assert abs(w[1] - c["y"][b]) < 1e-11
            assert abs(w[3] - c["sphi"][b]) < 1e-12
            assert abs(w[2] - c["z"][b]) < bound
            assert w[4] == tr.tanl[m] and w[5] == tr.q[m] / tr.pt[m]
            n_steps += 1
    assert n_steps > 3000


@pytest.mark.parametrize("bz", [0.0, 0.5, -0.5])
def test_refit_jacobian_matches_finite_differences(bz):
    """Every entry of the transport Jacobian: with the factor S = e_k e_k^T
    (C = e_k e_k^T) the transported covariance's column k is J[:, k]; compare
    with central differences of the propagated state (uniform field)."""
    rng = np.random.default_rng(22)
    fp = oracle.fit_params(bz)
    names = ["y", "z", "s", "t", "q"]
    for _ in range(150):
        x = rng.uniform(85, 240)
        d = rng.choice([-1, 1]) * rng.uniform(0.3, 6.0)
        p0 = np.array([rng.uniform(-10, 10), rng.uniform(-100, 100), rng.uniform(-0.8, 0.8),
                       rng.uniform(-1, 1), rng.uniform(-8, 8) if bz else rng.uniform(-1, 1)])
        for kcol in range(5):
            C5 = np.zeros((5, 5))
            C5[kcol, kcol] = 1.0
            ok, w = oracle.refit_propagate(oracle.fit_vec(x, p0, C5), x + d, fp)
            assert ok
            Jk = oracle.cov_of(w)[:, kcol]
            h = 1e-6 * max(1.0, abs(p0[kcol]))
            pp, pm = p0.copy(), p0.copy()
            pp[kcol] += h
            pm[kcol] -= h
            _, wp = oracle.refit_propagate(oracle.fit_vec(x, pp), x + d, fp)
            _, wm = oracle.refit_propagate(oracle.fit_vec(x, pm), x + d, fp)
            fd = (wp[1:6] - wm[1:6]) / (2 * h)
            for i in range(5):
                assert abs(Jk[i] - fd[i]) < 2e-7 * max(1.0, abs(fd[i])), \
                    (names[i], names[kcol], Jk[i], fd[i])


def test_refit_field_polynomial_terms():
    """The polynomial field enters the curvature at the straight-line
    midpoint of the step: over one step ds = -kappa Bz(rho_m, z_m) q d.
    Each term checked on its own against its closed form."""
    x, d = 150.0, 2.0
    p0 = np.array([3.0, 80.0, 0.2, 0.7, 2.0])
    c0 = math.sqrt(1 - p0[2] ** 2)
    xm, ym, zm = x + d / 2, p0[0] + d / 2 * p0[2] / c0, p0[1] + d / 2 * p0[3] / c0
    r2 = xm * xm + ym * ym
    terms = [zm, zm * zm, r2, r2 * zm, r2 * zm * zm]
    for j, tj in enumerate(terms):
        b = [0.0] * 5
        b[j] = 1e-3 / tj  # 1 mT from this term alone
        fp = oracle.fit_params(BZ, field=b)
        ok, w = oracle.refit_propagate(oracle.fit_vec(x, p0), x + d, fp)
        assert ok
        ds = w[3] - p0[2]
        expect = -KAPPA * (BZ + 1e-3) * p0[4] * d
        assert abs(ds - expect) < 1e-15, (j, ds, expect)


# ------------------------------------------------------------------ update

def test_refit_update_equals_bayesian_posterior():
    """orc_refit_update: posterior of the Gaussian prior (p, C) and the 2-D
    measurement (y, z) with variance diag(sy^2, sz^2), in information form;
    the chi2 increment equals the minimised objective."""
    rng = np.random.default_rng(23)
    fp = oracle.fit_params(BZ)
    V = np.diag([fp.sigma_y ** 2, fp.sigma_z ** 2])
    H = np.zeros((2, 5))
    H[0, 0] = H[1, 1] = 1.0
    for _ in range(200):
        A = rng.normal(size=(5, 5))
        C0 = A @ A.T + 0.05 * np.eye(5)
        p0 = rng.normal(size=5)
        m = rng.normal(size=2)
        w, chi2 = oracle.refit_update(oracle.fit_vec(100.0, p0, np.linalg.cholesky(C0)), m[0], m[1], fp)
        Ci = np.linalg.inv(C0)
        Cp = np.linalg.inv(Ci + H.T @ np.linalg.inv(V) @ H)
        pp = Cp @ (Ci @ p0 + H.T @ np.linalg.inv(V) @ m)
        assert np.allclose(w[1:6], pp, rtol=1e-9, atol=1e-11)
        assert np.allclose(oracle.cov_of(w), Cp, rtol=1e-8, atol=1e-11)
        dp = pp - p0
        r = m - H @ pp
        obj = dp @ Ci @ dp + r @ np.linalg.inv(V) @ r
        assert abs(chi2 - obj) < 1e-8 * max(1.0, obj)


# ------------------------------------------------------------------- refit

def _helix_model(theta, x0, xs, bz):
    """Closed-form helix from the state theta = (y, z, s, t, q) at x0 to the
    planes xs, uniform field: s(x) = s0 + k (x - x0),
    y = y0 + (x - x0) (s0 + s) / (c0 + c), z = z0 + t (asin s - asin s0) / k."""
    y0, z0, s0, t, q = theta
    k = -KAPPA * bz * q
    d = xs - x0
    s = s0 + k * d
    c0, c = math.sqrt(1 - s0 * s0), np.sqrt(1 - s * s)
    y = y0 + d * (s0 + s) / (c0 + c)
    if k == 0.0:
        arc = d / c0
    else:
        arc = (np.arcsin(s) - math.asin(s0)) / k
    return y, z0 + t * arc


@pytest.mark.parametrize("bz", [0.0, 0.5])
def test_refit_small_noise_is_gauss_newton(bz):
    """Small-noise limit: the refit's deviation from the truth equals one
    Gauss-Newton step of weighted least squares on the closed-form helix
    (Jacobian by finite differences, weights 1/sigma^2), and its covariance
    equals (A^T W A)^-1; priors on s, t, q made negligible."""
    rng = np.random.default_rng(24)
    tr = _tracks(rng, 60, pt_lo=0.3, pt_hi=5.0, vtx=5.0)
    fp = oracle.fit_params(bz, var_s=100.0, var_t=100.0, var_q=1e4)
    eps = 1e-6
    n_done = 0
    for m, c in _long_segments(tr, bz, min_rows=40):
        truth = _truth_in(tr, m, c)
        xs = XR[c["row"]]
        y = c["y"] + eps * rng.normal(size=len(xs))
        z = c["z"] + eps * rng.normal(size=len(xs))
        start = truth.copy()
        start[3] += 1e-4
        start[5] *= 1.001
        v, _ = refit_double(start, xs, y, z, fp)
        th0 = truth[1:6]
        py, pz = _helix_model(th0, xs[0], xs, bz)
        r = np.concatenate([y - py, z - pz])
        A = np.zeros((2 * len(xs), 5))
        for j in range(5):
            h = 1e-6 * max(1.0, abs(th0[j]))
            tp, tm = th0.copy(), th0.copy()
            tp[j] += h
            tm[j] -= h
            yp, zp = _helix_model(tp, xs[0], xs, bz)
            ym, zm = _helix_model(tm, xs[0], xs, bz)
            A[:, j] = np.concatenate([yp - ym, zp - zm]) / (2 * h)
        W = np.concatenate([np.full(len(xs), 1 / fp.sigma_y ** 2), np.full(len(xs), 1 / fp.sigma_z ** 2)])
        if bz == 0.0:
            A = A[:, :4]  # q is not observable without a field
        info = A.T @ (W[:, None] * A)
        cov = np.linalg.inv(info)
        step = cov @ (A.T @ (W * r))
        got = v[1:6] - th0
        C5 = oracle.cov_of(v)
        nk = A.shape[1]
        scale = np.sqrt(np.diag(cov))
        # the estimate: deviations agree to 1e-3 of their own size (sigma-scaled)
        dev = np.abs(got[:nk] - step) / (eps * scale / 0.1)
        assert np.all(dev < 1e-3), (m, got[:nk], step)
        # the covariance, correlation-scaled
        rel = np.abs(C5[:nk, :nk] - cov) / np.outer(scale, scale)
        assert np.all(rel < 1e-5), rel.max()
        assert v[0] == xs[0]
        n_done += 1
    assert n_done >= 20


def test_refit_noise_free_fixed_point():
    """Unsmeared helix hits: the refit, iterated from its previous output,
    converges to the generated parameters at the innermost cluster within
    1e-9 (scale floor 1 cm, 1 cm, 1, 1, 1 c/GeV)."""
    rng = np.random.default_rng(25)
    tr = _tracks(rng, 60, pt_lo=0.2, pt_hi=10.0, vtx=10.0)
    fp = oracle.fit_params(BZ)
    n_done = 0
    for m, c in _long_segments(tr, BZ, min_rows=30):
        truth = _truth_in(tr, m, c)
        xs = XR[c["row"]]
        st = truth + np.array([0.0, 0.05, -0.05, 0.01, 0.01, 0.2 * truth[5]])
        for it in range(30):
            v, _ = refit_double(st, xs, c["y"], c["z"], fp)
            st = v[:6]
            if np.all(np.abs(st[1:] - truth[1:]) <= 1e-9 * np.maximum(np.abs(truth[1:]), 1.0)):
                break
        else:
            pytest.fail(f"no convergence for track {m}: {st[1:] - truth[1:]}")
        n_done += 1
    assert n_done >= 20


def test_refit_pulls_and_chi2_on_smeared_tracks():
    """Gaussian-smeared isolated tracks (sigma 0.1 cm): pulls of all five
    parameters at the innermost cluster have mean 0 and width 1, and chi2/ndf
    has mean 1 (within the statistical tolerance of ~1000 tracks).  A dropped
    cross term of the transport shows up as a wrong width."""
    rng = np.random.default_rng(26)
    tr = _tracks(rng, 1800, pt_lo=0.2, pt_hi=5.0, vtx=5.0)
    fp = oracle.fit_params(BZ)
    pulls, chi = [], []
    for m, c in _long_segments(tr, BZ, min_rows=30):
        truth = _truth_in(tr, m, c)
        xs = XR[c["row"]]
        y = c["y"] + S.SIGMA * rng.normal(size=len(xs))
        z = c["z"] + S.SIGMA * rng.normal(size=len(xs))
        v, chi2 = refit_double(truth, xs, y, z, fp)
        C5 = oracle.cov_of(v)
        pulls.append((v[1:6] - truth[1:]) / np.sqrt(np.diag(C5)))
        chi.append(chi2 / (2 * len(xs) - 5))
    pulls = np.array(pulls)
    assert len(pulls) > 800
    mu, sd = pulls.mean(axis=0), pulls.std(axis=0)
    assert np.all(np.abs(mu) < 0.12), mu
    assert np.all(np.abs(sd - 1.0) < 0.08), sd
    assert 0.97 <= np.mean(chi) <= 1.03, np.mean(chi)


FIELD = (2e-5, -4e-8, -8e-8, 1e-10, 1e-13)  # b1..b5: about 1 % non-uniformity


def _bz_poly(x, y, z, bz, b):
    r2 = x * x + y * y
    return bz + z * (b[0] + z * b[1]) + r2 * (b[2] + z * (b[3] + z * b[4]))


def _rk4_track(st6, xs, bz, b, dx=0.01):
    """Integrate dy/dx = s / c, ds/dx = -kappa Bz(x, y, z) q, dz/dx = t / c
    (transverse curvature of a charge in an axial field, pT and tan(lambda)
    constant) with classical Runge-Kutta from st6 to every plane in xs."""
    x, y, z, s, t, q = st6

    def f(x, u):
        y, z, s = u
        c = math.sqrt(1 - s * s)
        return np.array([s / c, t / c, -KAPPA * _bz_poly(x, y, z, bz, b) * q])

    u = np.array([y, z, s])
    out = []
    for xt in xs:
        while x < xt:
            h = min(dx, xt - x)
            k1 = f(x, u)
            k2 = f(x + h / 2, u + h / 2 * k1)
            k3 = f(x + h / 2, u + h / 2 * k2)
            k4 = f(x + h, u + h * k3)
            u = u + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            x = x + h
        out.append(u.copy())
    return np.array(out)


def test_refit_polynomial_field_recovers_truth():
    """Tracks integrated numerically (RK4, 0.01 cm steps) through the
    polynomial field: the iterated refit with the same polynomial recovers
    the starting parameters (field held at the step midpoint, so to a small
    bound), while the uniform-field refit of the same hits is biased by far
    more."""
    rng = np.random.default_rng(27)
    n_done = 0
    for _ in range(12):
        s0 = rng.uniform(-0.3, 0.3)
        st6 = np.array([XR[0], rng.uniform(-5, 5), rng.uniform(10, 60), s0, rng.uniform(0.1, 0.8),
                        rng.choice([-1, 1]) / rng.uniform(0.3, 3.0)])
        rows = np.arange(0, 159)
        xs = XR[rows]
        u = _rk4_track(st6, xs, BZ, FIELD)
        if np.any(np.abs(u[:, 2]) > 0.9):
            continue
        y, z = u[:, 0], u[:, 1]
        errs = {}
        for name, field in (("poly", FIELD), ("uniform", None)):
            fp = oracle.fit_params(BZ, field=field)
            st = st6 + np.array([0.0, 0.02, 0.02, 0.005, 0.01, 0.05 * st6[5]])
            for it in range(20):
                v, _ = refit_double(st, xs, y, z, fp)
                st = v[:6]
            errs[name] = np.abs(st[1:] - st6[1:])
        assert errs["poly"][0] < 2e-5 and errs["poly"][1] < 2e-5, errs["poly"]
        assert errs["poly"][2] < 2e-7 and errs["poly"][3] < 2e-7, errs["poly"]
        assert errs["poly"][4] < 1e-4 * abs(st6[5]), errs["poly"]
        assert errs["uniform"][4] > 30 * errs["poly"][4] + 1e-6, (errs["uniform"], errs["poly"])
        n_done += 1
    assert n_done >= 8


def test_refit_tracks_equals_step_sequence():
    """orc_refit_tracks (float32 clusters, per-track loop) runs exactly the two
    passes of the single-step entries, including ndf and status."""
    rng = np.random.default_rng(28)
    tr = _tracks(rng, 40, vtx=5.0)
    fp = oracle.fit_params(BZ)
    segs = _long_segments(tr, BZ, min_rows=20)
    cl, off, st6, ref = [], [0], [], []
    for m, c in segs:
        xs = XR[c["row"]].astype(np.float32)
        y = (c["y"] + S.SIGMA * rng.normal(size=len(xs))).astype(np.float32)
        z = (c["z"] + S.SIGMA * rng.normal(size=len(xs))).astype(np.float32)
        for k in range(len(xs)):
            cl.append([xs[k], y[k], z[k], 0.0])
        off.append(off[-1] + len(xs))
        s = _truth_in(tr, m, c)
        s[0] = np.float32(s[0])
        st6.append(s)
        v, chi2 = refit_double(s, xs.astype(np.float64), y.astype(np.float64), z.astype(np.float64), fp)
        F = oracle.factor_of(v)
        packed = []
        for i in range(5):
            for j in range(i + 1):
                acc = F[i, 0] * F[j, 0]
                for m_ in range(1, 5):
                    acc = acc + F[i, m_] * F[j, m_]
                packed.append(acc)
        ref.append(np.concatenate([v[:6], packed, [chi2, 2 * len(xs) - 5, 0]]))
    out = oracle.refit_lists(np.array(st6), np.array(off), np.arange(off[-1]), np.array(cl, np.float32), fp)
    np.testing.assert_array_equal(out, np.array(ref))


def test_refit_stops_at_s_max():
    """A track that turns past |sin phi| = s_max fails the fit: status 1, the
    output is the state reached, ndf counts the clusters filtered."""
    fp = oracle.fit_params(BZ)
    q = -20.0  # 0.05 GeV/c, k = 0.03/cm: sin(phi) grows by 0.03 per cm
    s0 = 0.5
    st6 = np.array([XR[0], 0.0, 10.0, s0, 0.1, q])
    xs = XR[:40]
    with np.errstate(invalid="ignore"):
        y, z = _helix_model(st6[1:], XR[0], xs, BZ)  # NaN past the turn: never read
    ok_rows = int(np.sum(np.abs(s0 - KAPPA * BZ * q * (xs - xs[0])) <= 0.95))
    assert 3 < ok_rows < 40
    cl = np.stack([xs, y, z, np.zeros_like(xs)], axis=1).astype(np.float32)
    out = oracle.refit_lists(st6[None], np.array([0, len(xs)]), np.arange(len(xs)), cl, fp)[0]
    assert out[23] == 1
    assert out[22] == 2 * ok_rows - 5
    assert out[0] == np.float32(xs[ok_rows - 1])


def test_refit_fp32_close_to_fp64():
    """The FP32_EXACT build stays close to FP64 on smeared tracks (not a pin:
    the FP32 arithmetic is what the CUDA exact mode reproduces bit for bit)."""
    rng = np.random.default_rng(29)
    tr = _tracks(rng, 200, vtx=5.0)
    fp = oracle.fit_params(BZ)
    cl, off, st6 = [], [0], []
    for m, c in _long_segments(tr, BZ, min_rows=30):
        xs = XR[c["row"]]
        for k in range(len(xs)):
            cl.append([xs[k], c["y"][k] + S.SIGMA * rng.normal(), c["z"][k] + S.SIGMA * rng.normal(), 0])
        off.append(off[-1] + len(xs))
        st6.append(_truth_in(tr, m, c))
    args = (np.array(st6), np.array(off), np.arange(off[-1]), np.array(cl, np.float32), fp)
    a = oracle.refit_lists(*args, mode="f64")
    b = oracle.refit_lists(*args, mode="f32")
    assert np.all(a[:, 23] == 0) and np.all(b[:, 23] == 0)
    err = np.abs(a[:, 1:6] - b[:, 1:6])
    sig = np.sqrt(np.stack([oracle.unpack_cov(r)[i, i] for r in a for i in range(5)]).reshape(-1, 5))
    assert np.all(err < 0.01 * sig), (err / sig).max()
