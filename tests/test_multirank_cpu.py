"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank
tracks its own events with no data-path exchange; the only collective is the
max-over-ranks step time.  The CPU oracle stands in for each rank's GPU work
(a rank's result does not depend on the other ranks)."""
import os
import socket
import time

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as tmp

import bench
import oracle
from paper_1712_09430_gb300 import synth as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.rank_seeds(rank, batch=2, base=100)
        evs = [S.pp_event(seed=s) for s in seeds]
        cl, rc = S.concat_events(evs)
        t0 = time.perf_counter()
        o = oracle.run(cl, rc, len(evs), 0.5, S.row_x(), mode="f64", threads=1)
        ms = (time.perf_counter() - t0) * 1e3 + 10.0 * rank   # ranks differ in speed
        ms_all = bench.reduce_step_ms(ms, dist)
        out[rank] = (seeds, int(len(cl)), ms, ms_all, o["trk_hits"].tolist())
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_events_and_take_max_time():
    world = 2
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                        start_method="spawn")
    s0, n0, ms0, all0, h0 = out[0]
    s1, n1, ms1, all1, h1 = out[1]
    assert not set(s0) & set(s1)                      # disjoint events
    assert all0 == all1 == max(ms0, ms1)              # whole-job time = slowest rank
    # each rank's tracks equal a single-process run on its own events
    for seeds, hits in ((s0, h0), (s1, h1)):
        evs = [S.pp_event(seed=s) for s in seeds]
        cl, rc = S.concat_events(evs)
        o = oracle.run(cl, rc, len(evs), 0.5, S.row_x(), mode="f64", threads=1)
        assert o["trk_hits"].tolist() == hits
    value = (n0 + n1) / (all0 * 1e-3)
    assert value > 0
