"""Phase II end to end in the production build against the FP64 oracle chain.

The other Phase-II tests give the oracle the GPU's own tracks, which
isolates each stage.  Here each side runs its whole chain on its own:

* GPU, production build: Phase I, the final refit, track merging and the
  collision offsets, in one call;
* oracle, FP64: its own Phase-I tracks (tpc_oracle.c), the refit of those
  (tpc_refit.c), the merging of those refits and their collision offsets.

The two chains see slightly different Phase-I tracks (FP32 production vs
FP64), so they are compared through what the chain is for, each side
against generator truth, within a stated tolerance:

* merging: of the "true split pairs" -- consecutive segments, by the radius
  of their innermost cluster, of one generated track -- the fraction each
  chain links (either direction) agrees within 3 percentage points, and
  both chains' links join segments of one generated track in > 95 % of
  cases;
* collision offsets: the number of collisions each chain finds within
  0.3 cm of a generated drift offset agrees within 10 % (at least 1).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from gpu_util import XR  # noqa: E402
from paper_1712_09430_gb300 import synth as S  # noqa: E402
from paper_1712_09430_gb300.tracker import Tracker  # noqa: E402


def _majority(labels, hits):
    v, c = np.unique(labels[hits], return_counts=True)
    return int(v[np.argmax(c)])


def _gpu_chain(ev):
    with Tracker(XR, bz=ev.bz, exact_fp32=0, refit=1, merge=1, t0=1) as tr:
        r = tr.track(ev.clusters, ev.row_counts, 1)
    lists = [r.hits_of(m) for m in range(len(r.tracks))]
    return lists, r.merges["next"].astype(np.int64), r.t0s["collision"], r.t0s["dz"].astype(np.float64)


def _oracle_chain(ev):
    o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, XR, mode="f64")
    fp = oracle.fit_params(ev.bz)
    fits = oracle.refit_tracks(o, ev.clusters, ev.bz, mode="f64", fp=fp)
    unit = o["tl_unit"][o["trk_t"]].astype(np.int32)
    off = o["trk_hit_off"]
    lists = [o["trk_hits"][off[m]:off[m + 1]] for m in range(len(off) - 1)]
    x_last = np.array([ev.clusters[h[-1], 0] for h in lists], np.float64)
    nxt, _ = oracle.merge_tracks(unit, fits, x_last, fp, mode="f64")
    t0 = oracle.t0_tracks(unit, fits, fp, mode="f64")
    return lists, nxt.astype(np.int64), t0[:, 0].astype(np.int32), t0[:, 2]


def _merge_quality(ev, lists, nxt):
    lab = ev.label
    major = np.array([_majority(lab, h) for h in lists])
    r_in = np.array([np.hypot(ev.clusters[h[0], 0], ev.clusters[h[0], 1]) for h in lists])
    linked = set()
    for a, b in enumerate(nxt):
        if b >= 0:
            linked.add((a, int(b)))
            linked.add((int(b), a))
    pairs = []
    for m in np.unique(major[major >= 0]):
        seg = np.flatnonzero(major == m)
        if len(seg) < 2:
            continue
        seg = seg[np.argsort(r_in[seg], kind="stable")]
        pairs += list(zip(seg[:-1], seg[1:]))
    eff = np.mean([(int(a), int(b)) in linked for a, b in pairs]) if pairs else float("nan")
    links = [(a, int(b)) for a, b in enumerate(nxt) if b >= 0]
    purity = np.mean([major[a] == major[b] and major[a] >= 0 for a, b in links]) if links else float("nan")
    return eff, purity, len(pairs), len(links)


def _collisions_found(ev, coll, dz):
    found = 0
    for k in np.unique(coll[coll >= 0]):
        d = dz[coll == k][0]
        if np.min(np.abs(np.asarray(ev.coll_dz) - d)) < 0.3:
            found += 1
    return found


@pytest.mark.parametrize("name", ["lowpt", "central"])
def test_merge_chain_production_vs_fp64_oracle_chain(name):
    ev = (S.make_event(22, 400, 0, pt_mean=0.25, noise_frac=0.05) if name == "lowpt"
          else S.central_event(seed=5, scale=0.2))
    g = _merge_quality(ev, *_gpu_chain(ev)[:2])
    o = _merge_quality(ev, *_oracle_chain(ev)[:2])
    assert g[2] > 50 and o[2] > 50, (g, o)          # enough true split pairs
    assert abs(g[0] - o[0]) <= 0.03, (g, o)
    assert g[1] > 0.95 and o[1] > 0.95, (g, o)


def test_collision_offsets_production_vs_fp64_oracle_chain():
    ev = S.time_frame(seed=7, n_coll=12, scale=0.3)
    _, _, gc, gdz = _gpu_chain(ev)
    _, _, oc, odz = _oracle_chain(ev)
    ng = _collisions_found(ev, gc, gdz)
    no = _collisions_found(ev, oc, odz)
    assert no >= 3
    assert abs(ng - no) <= max(1, int(0.1 * no)), (ng, no)
