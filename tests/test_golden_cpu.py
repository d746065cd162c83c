"""The oracle against its stored record (tests/golden/oracle_central_small.json,
written by tests/golden/make_golden.py from the oracle alone).

The paper prints no worked example of the tracker's outputs, so the record is
a regression guard: a change of the oracle's arithmetic, or of the seeded
input generator, fails here until the record is regenerated for a reason the
paper gives."""
import json
import math
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402
from paper_1712_09430_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def stored_and_now():
    with open(make_golden.PATH) as f:
        stored = json.load(f)
    return stored, make_golden.record()


def test_seeded_inputs_unchanged(stored_and_now):
    stored, now = stored_and_now
    assert now["event"] == stored["event"], "the seeded input generator changed"


@pytest.mark.parametrize("mode", ["f32", "f64"])
def test_oracle_matches_record(stored_and_now, mode):
    stored, now = stored_and_now
    a, b = now["modes"][mode], stored["modes"][mode]
    assert a.keys() == b.keys()
    for k in a:
        if k in ("tl_f_first", "fit_first"):
            assert all(math.isclose(x, y, rel_tol=1e-10, abs_tol=1e-12) for x, y in zip(a[k], b[k])), k
        elif k == "chi2_sum":
            assert math.isclose(a[k], b[k], rel_tol=1e-10), k
        else:
            assert a[k] == b[k], k


def test_track_length_bound_of_the_detector(stored_and_now):
    # Sec. 1: a trajectory crosses at most 159 pad rows of a sector, so it has
    # at most 159 clusters
    stored, _ = stored_and_now
    assert len(synth.row_x()) == 159
    for mode in ("f32", "f64"):
        assert 0 < stored["modes"][mode]["longest_track"] <= 159
