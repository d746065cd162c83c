"""Track-finding QA against generator truth (efficiency, clone and fake rates).

Definitions (the paper gives none, so these are stated readings):
* a track matches MC track m if at least 90 % of its hits carry label m,
  otherwise it is fake;
* an (MC track, sector) pair is reconstructable if it left >= 30 clusters in
  that sector of that event;
* efficiency = matched reconstructable pairs / reconstructable pairs;
* clone rate = sum over reconstructable pairs of max(0, matches - 1) /
  reconstructable pairs;
* fake rate = fake tracks / all tracks.
"""
import numpy as np

N_ROWS = 159
N_SECTORS = 36


def unit_of_cluster(row_counts):
    n_units = len(row_counts) // N_ROWS
    return np.repeat(np.arange(n_units), row_counts.reshape(n_units, N_ROWS).sum(1))


def qa(labels, row_counts, trk_hit_off, trk_hits, min_clusters=30, match_frac=0.9):
    """labels: int [N] MC label per cluster (-1 noise), globally unique per event
    (combine event index into the label before calling for batches)."""
    labels = np.asarray(labels, dtype=np.int64)
    unit = unit_of_cluster(np.asarray(row_counts))
    key = unit * (1 << 32) + labels
    sig = labels >= 0
    uk, cnt = np.unique(key[sig], return_counts=True)
    reco = set(uk[cnt >= min_clusters].tolist())
    n_match = {}
    fakes = 0
    M = len(trk_hit_off) - 1
    for m in range(M):
        h = trk_hits[trk_hit_off[m]:trk_hit_off[m + 1]]
        lab = labels[h]
        vals, c = np.unique(lab, return_counts=True)
        j = np.argmax(c)
        if vals[j] >= 0 and c[j] >= match_frac * len(h):
            k = int(unit[h[0]]) * (1 << 32) + int(vals[j])
            n_match[k] = n_match.get(k, 0) + 1
        else:
            fakes += 1
    n_reco = len(reco)
    found = sum(1 for k in reco if n_match.get(k, 0) > 0)
    clones = sum(max(0, n_match.get(k, 0) - 1) for k in reco)
    return dict(n_reconstructable=n_reco, n_tracks=M,
                eff=found / n_reco if n_reco else float("nan"),
                clone=clones / n_reco if n_reco else float("nan"),
                fake=fakes / M if M else 0.0)
