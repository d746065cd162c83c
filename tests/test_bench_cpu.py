"""Host-side rules of bench.py (no GPU): the DRAM traffic of the committed
ncu summary is reported only for the kernel sources it was taken on, and
ranks track disjoint events (weak scaling without a data-path collective),
and the reference arm prints the contract's line."""
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


def test_reference_arm_line(capsys, monkeypatch):
    """--impl reference: the oracle on the GPU step's own events, one JSON
    line with the GPU arm's metric and config, its own cpu_baseline and an
    e2e without host-device bytes; ranks other than 0 print nothing."""
    import argparse
    import json
    args = argparse.Namespace(gpus=1, steps=1, warmup=0, batch=1)
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["config"]["workload"] == bench.WORKLOAD
    # the GPU arm's config for the same batch, key for key
    from paper_1712_09430_gb300 import synth
    n = sum(synth.central_event(seed=s).n for s in bench.rank_seeds(0, args.batch))
    assert line["config"] == bench.step_config(args.batch, n, args.gpus)
    assert line["unit"] == "clusters/s" and line["higher_is_better"] is True and line["value"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "clusters/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
