"""Pin of the oracle tracker's y-mirror symmetry.

The sector frame is symmetric about y = 0: the sector spans |y| <= X tan(10
deg) + margin, the neighbour windows are |y_j - y_i R| <= W, a helix with the
opposite charge and sin(phi) is the mirror image of the original, and every
rule of Sec. 2 (links, cleaning, start hits, the filter, selection) treats
+y and -y alike.  Negating y is exact in floating point, so tracking the
mirrored event must give the same links and tracks and filter outputs with
y, sin(phi) and q/pT negated and everything else (z, tan(lambda), the
covariances and chi2) unchanged, bit for bit, in both oracle modes.  A
term that is not odd in (y, sin(phi), q/pT) -- a one-sided bound, a dropped
sign, an offset -- breaks it."""
import numpy as np
import pytest

import oracle
from paper_1712_09430_gb300 import synth as S

XR = S.row_x()
ODD = (1, 3, 5)  # y, sin(phi), q/pT among the 16 filter outputs


@pytest.mark.parametrize("mode", ["f64", "f32"])
@pytest.mark.parametrize("make", [lambda: S.pp_event(seed=7), lambda: S.central_event(seed=5, scale=0.2)],
                         ids=["pp", "central0.2"])
def test_mirrored_event_gives_mirrored_tracks(make, mode):
    ev = make()
    o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR, mode=mode)
    cl = ev.clusters.copy()
    cl[:, 1] = -cl[:, 1]
    o2 = oracle.run(cl, ev.row_counts, 1, ev.bz, XR, mode=mode)
    assert len(o["trk_t"]) > 50
    for k in ("up_raw", "dn_raw", "up", "dn", "start", "tl_n", "tl_alive", "tl_hits", "trk_t", "trk_hits"):
        np.testing.assert_array_equal(o2[k], o[k], err_msg=k)
    want = o["tl_f"].copy()
    want[:, ODD] = -want[:, ODD]
    np.testing.assert_array_equal(o2["tl_f"], want)


@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_refit_of_the_mirrored_event_is_mirrored(mode):
    """The final refit (full 5x5 covariance, a field polynomial in z and
    rho^2, both even in y) of the mirrored event's tracks: x, z, tan(lambda),
    chi2, ndf and status unchanged, y, sin(phi) and q/pT negated, and each
    covariance entry negated exactly when it pairs one of those three with z
    or tan(lambda), bit for bit."""
    ev = S.central_event(seed=5, scale=0.2)
    field = (1e-5, -2e-8, 3e-7, 1e-9, -1e-11)
    o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR, mode=mode)
    cl = ev.clusters.copy()
    cl[:, 1] = -cl[:, 1]
    o2 = oracle.run(cl, ev.row_counts, 1, ev.bz, XR, mode=mode)
    f1 = oracle.refit_tracks(o, ev.clusters, ev.bz, field=field, mode=mode)
    f2 = oracle.refit_tracks(o2, cl, ev.bz, field=field, mode=mode)
    assert len(f1) > 1000 and np.all(f1[:, 23] == f2[:, 23])
    odd = np.array([True, False, True, False, True])  # y z sin(phi) tan(lambda) q/pT
    sign = np.ones(oracle.N_FIT)
    sign[1:6] = np.where(odd, -1.0, 1.0)
    for i in range(5):
        for j in range(i + 1):
            sign[6 + i * (i + 1) // 2 + j] = -1.0 if odd[i] != odd[j] else 1.0
    np.testing.assert_array_equal(f2, f1 * sign)
