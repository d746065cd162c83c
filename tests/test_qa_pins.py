"""Pins of the track-finding QA definitions (tests/qa.py) on hand-built
cases whose rates follow from the definitions by counting:

* a track matches MC track m when at least 90 % of its hits carry m
  (exactly 90 % matches, just below does not);
* an (MC track, sector) pair is reconstructable from 30 clusters in that
  sector (29 is not), counted per event and sector;
* clones: every match of a reconstructable pair beyond the first;
* fakes: tracks that match nothing, over all tracks.
"""
import numpy as np
import pytest

import qa

NR, NS = qa.N_ROWS, qa.N_SECTORS


def layout(per_unit_labels, n_events=1):
    """Clusters of hand-chosen labels placed unit by unit (row 0 holds them
    all: the QA only reads units).  per_unit_labels: {unit: [labels]}.
    Returns (labels[N], row_counts, first cluster position of each unit)."""
    rc = np.zeros(n_events * NS * NR, np.int32)
    labels, first = [], {}
    pos = 0
    for u in sorted(per_unit_labels):
        lab = per_unit_labels[u]
        rc[u * NR] = len(lab)
        first[u] = pos
        labels.extend(lab)
        pos += len(lab)
    return np.array(labels, np.int64), rc, first


def tracks_of(lists):
    off = np.zeros(len(lists) + 1, np.int64)
    off[1:] = np.cumsum([len(h) for h in lists])
    hits = np.concatenate([np.asarray(h, np.int32) for h in lists]) if lists else np.zeros(0, np.int32)
    return off, hits


def test_ninety_percent_match_threshold():
    # unit 0: MC 1 has 40 clusters, 20 noise clusters after them
    lab, rc, f = layout({0: [1] * 40 + [-1] * 20})
    at = list(range(18)) + [40, 41]            # 18 of 20 hits = 90 %: a match
    below = list(range(17)) + [40, 41, 42]     # 17 of 20 = 85 %: fake
    r = qa.qa(lab, rc, *tracks_of([at]))
    assert r["n_reconstructable"] == 1 and r["eff"] == 1.0 and r["fake"] == 0.0
    r = qa.qa(lab, rc, *tracks_of([below]))
    assert r["eff"] == 0.0 and r["fake"] == 1.0
    # 9 of 10 matches, 8 of 10 does not (the threshold is on the fraction)
    r = qa.qa(lab, rc, *tracks_of([list(range(9)) + [40]]))
    assert r["eff"] == 1.0 and r["fake"] == 0.0
    r = qa.qa(lab, rc, *tracks_of([list(range(8)) + [40, 41]]))
    assert r["eff"] == 0.0 and r["fake"] == 1.0


def test_majority_of_another_track_is_not_a_match_for_the_minority():
    lab, rc, f = layout({0: [1] * 40 + [2] * 40})
    # 19 hits of MC 2 and one of MC 1: matches MC 2 (95 %), not MC 1
    r = qa.qa(lab, rc, *tracks_of([[0] + list(range(40, 59))]))
    assert r["n_reconstructable"] == 2 and r["eff"] == 0.5 and r["fake"] == 0.0
    # and the other way round: 19 of MC 1 (the smaller label) and one of MC 2
    r = qa.qa(lab, rc, *tracks_of([list(range(19)) + [40]]))
    assert r["eff"] == 0.5 and r["fake"] == 0.0


def test_reconstructable_from_thirty_clusters_per_sector():
    # MC 1 leaves 30 clusters in unit 0 and 29 in unit 1; MC 2 leaves 29 in unit 0
    lab, rc, f = layout({0: [1] * 30 + [2] * 29, 1: [1] * 29})
    r = qa.qa(lab, rc, *tracks_of([]))
    assert r["n_reconstructable"] == 1 and r["eff"] == 0.0
    # a track of MC 1 in unit 1 (29 clusters) matches but is not counted in the efficiency
    r = qa.qa(lab, rc, *tracks_of([list(range(f[1], f[1] + 20))]))
    assert r["n_reconstructable"] == 1 and r["eff"] == 0.0 and r["fake"] == 0.0
    # the same MC label in two events is two pairs
    lab2, rc2, f2 = layout({0: [1] * 30, NS: [1] * 30}, n_events=2)
    r = qa.qa(lab2, rc2, *tracks_of([list(range(0, 20))]))
    assert r["n_reconstructable"] == 2 and r["eff"] == 0.5


def test_clone_counts():
    lab, rc, f = layout({0: [1] * 90 + [2] * 40})
    one = list(range(0, 30))
    two = list(range(30, 60))
    three = list(range(60, 90))
    other = list(range(90, 120))
    # two matches of MC 1: one clone; MC 2 found once
    r = qa.qa(lab, rc, *tracks_of([one, two, other]))
    assert r["n_reconstructable"] == 2 and r["eff"] == 1.0
    assert r["clone"] == pytest.approx(1 / 2) and r["fake"] == 0.0
    # three matches: two clones
    r = qa.qa(lab, rc, *tracks_of([one, two, three, other]))
    assert r["clone"] == pytest.approx(2 / 2)
    # one match each: no clone
    r = qa.qa(lab, rc, *tracks_of([one, other]))
    assert r["clone"] == 0.0


def test_clone_counted_per_sector_pair():
    # MC 1 in two units, one match in each: no clone, both found
    lab, rc, f = layout({0: [1] * 30, 1: [1] * 30})
    r = qa.qa(lab, rc, *tracks_of([list(range(0, 20)), list(range(30, 50))]))
    assert r["n_reconstructable"] == 2 and r["eff"] == 1.0 and r["clone"] == 0.0


def test_fake_rate():
    lab, rc, f = layout({0: [1] * 40 + [-1] * 40})
    good = list(range(0, 20))
    noise = list(range(40, 60))                    # all noise: fake
    mixed = list(range(20, 30)) + list(range(40, 50))  # 50 %: fake
    r = qa.qa(lab, rc, *tracks_of([good, noise, mixed]))
    assert r["fake"] == pytest.approx(2 / 3) and r["eff"] == 1.0 and r["n_tracks"] == 3
    r = qa.qa(lab, rc, *tracks_of([]))
    assert r["fake"] == 0.0
