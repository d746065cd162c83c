"""Write tests/golden/oracle_central_small.json: the oracle's outputs on one
seeded synthetic event, so that any later change to the oracle's arithmetic
(or to the seeded input generator) shows up as a difference.

The paper prints no worked example with numeric outputs of the tracker (Sec. 2
describes the steps; its tables give processing times and rates), so this
fixture is the oracle's own record.  It calls only the oracle and the seeded
input generator; nothing here runs the CUDA path.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1712_09430_gb300 import synth  # noqa: E402  (seeded inputs only)

PATH = os.path.join(HERE, "oracle_central_small.json")
EVENT = dict(generator="central_event", seed=3, scale=0.05)
# the field polynomial of the refit record (Bz = bz + z (b1 + z b2) + rho^2 (b3 + z (b4 + z b5)))
FIELD = (1e-5, -2e-8, 3e-7, 1e-9, -4e-12)


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def event():
    return getattr(synth, EVENT["generator"])(seed=EVENT["seed"], scale=EVENT["scale"])


def record():
    ev = event()
    out = dict(
        about="oracle outputs on a seeded synthetic event (regression record: the paper prints "
              "no worked example of the tracker's outputs); regenerate with make_golden.py only "
              "for a change of the oracle that names the passage of the paper behind it",
        event=dict(EVENT, bz=float(ev.bz), n_clusters=int(len(ev.clusters)),
                   clusters_sha256=sha(ev.clusters), row_counts_sha256=sha(ev.row_counts)),
        modes={},
    )
    xr = synth.row_x()
    for mode in ("f32", "f64"):
        o = oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, xr, mode=mode)
        fits = oracle.refit_tracks(o, ev.clusters, ev.bz, field=FIELD, mode=mode)
        rec = dict(
            links_up=int((o["up"] >= 0).sum()), links_raw_up=int((o["up_raw"] >= 0).sum()),
            tracklets=int(len(o["start"])), tracklets_alive=int(o["tl_alive"].sum()),
            tracks=int(len(o["trk_t"])), track_clusters=int(len(o["trk_hits"])),
            longest_track=int(o["trk_n"].max()) if len(o["trk_n"]) else 0,
            sha256={k: sha(o[k]) for k in ("up_raw", "dn_raw", "up", "dn", "start", "tl_n",
                                          "tl_alive", "tl_hits", "trk_t", "trk_n", "trk_hits")},
        )
        if mode == "f32":
            # binary32 arithmetic without contraction: the values are exact, so their bits are kept
            rec["sha256"]["tl_f"] = sha(o["tl_f"])
            rec["sha256"]["fits"] = sha(fits)
        else:
            # FP64: a few values, to 12 significant digits
            rec["tl_f_first"] = [float(f"{v:.12g}") for v in o["tl_f"][o["trk_t"][0], :6]]
            rec["fit_first"] = [float(f"{v:.12g}") for v in fits[0, :6]]
            rec["chi2_sum"] = float(f"{float(fits[:, 21].sum()):.12g}")
        out["modes"][mode] = rec
    return out


if __name__ == "__main__":
    with open(PATH, "w") as f:
        json.dump(record(), f, indent=1, sort_keys=True)
        f.write("\n")
    print(PATH)
