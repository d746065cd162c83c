"""Host-side rules of bench.py (no GPU): the DRAM traffic of the committed
ncu summary is reported only for the kernel sources it was taken on, and
ranks track disjoint events (weak scaling without a data-path collective)."""
import os
import shutil

import bench

CSRC = os.path.join(bench.ROOT, "paper_1712_09430_gb300", "csrc")
SOURCES = [os.path.join(CSRC, "k_fp.cu"), os.path.join(CSRC, "tpc_dev.cuh")]
SUMMARY = os.path.join(bench.ROOT, "profiles", "k_tracklets_sched_traffic_central8.md")


def test_traffic_only_for_the_sources_it_was_taken_on(tmp_path):
    got = bench.measured_traffic(SOURCES, SUMMARY)
    if got is not None:   # the committed summary matches the committed sources
        assert got > 1e8
    # any change to a source invalidates it
    changed = tmp_path / "k_fp.cu"
    shutil.copy(SOURCES[0], changed)
    with open(changed, "a") as f:
        f.write("\n// edited\n")
    assert bench.measured_traffic([str(changed), SOURCES[1]], SUMMARY) is None
    # and so does a summary without a hash or a missing file
    bare = tmp_path / "summary.md"
    bare.write_text("- traffic_bytes_per_launch: 123\n")
    assert bench.measured_traffic(SOURCES, str(bare)) is None
    assert bench.measured_traffic(SOURCES, str(tmp_path / "missing.md")) is None


def test_ranks_track_disjoint_events():
    seen = set()
    for rank in range(8):
        s = bench.rank_seeds(rank, 8)
        assert len(s) == 8 and not (seen & set(s))
        seen |= set(s)
    assert bench.rank_seeds(0, 8) == list(range(3, 11))   # the single-GPU batch
    assert bench.reduce_step_ms(4.2, None) == 4.2
