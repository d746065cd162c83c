"""Benchmark: TPC clusters/s tracked on central Pb-Pb-like events (GB300).

One step = the whole Phase-I hot path (grid build, CA neighbours, cleaning,
start hits, tracklet construction, selection, output) over one batch of
synthetic central Pb-Pb events (10,000 primaries + 3,000 secondaries, 10 %
noise, ~2.05 M clusters each), all 36 sectors of every event in one batched,
graph-replayed launch sequence.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl ours|reference]

value      clusters/s, inputs resident in device memory when the timed region
           starts; the batch (B x 33 MB of clusters) exceeds the 129 MB L2
e2e        the same metric through the C ABI with pinned HOST buffers: H2D of
           the clusters and row counts and D2H of the tracks inside the timed
           region; through the serving API with two batches in flight, so one
           batch's copies overlap the other's kernels (e2e_sync: the
           synchronous call, copies and kernels in turn)
roofline   the dominant kernel (tracklet constructor) against the measured HBM
           copy bandwidth; its algorithmic bytes are counted by the kernel in
           one extra untimed call (params.count_work)
cpu_baseline  the FP64 CPU oracle on the host cores, bounded sample (and the
           FP32_EXACT mode on all cores)
plain_per_sector, multi_queue_per_sector
           the same batch with one launch per (event, sector) per stage, on one
           stream and round-robin over 8 streams (Sec. 3, Sec. 3.1)
batch_sizes  the batched step at 1 and 32 central events per call
stream     min-bias events (Poisson arrivals at 1, 3, 5 kHz) through the
           serving API: p50/p99 latency from arrival to the result in hand
stream_central  central events through the serving API at 250, 500, 1000 Hz
refit      the final refit and the track merging on the same batch (Sec. 2
           Phase II): device time, tracks/s, FP32 ALU roofline of the refit
time_frame a continuous-readout time frame (Sec. 3.3): overlaid shifted
           collisions, the whole chain with the per-collision offsets; and
           five uneven time-frame slices (0.9-8.5 M clusters) in one launch
--impl reference  times the CPU oracle as the reference arm (same metric)

Multi-GPU: events shard across ranks with no collective (weak scaling), one
process per GPU under torchrun.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TPC clusters/s tracked (central Pb-Pb-like); p50/p99 event latency, stream"
WORKLOAD = "central Pb-Pb-like events: 10,000 primaries (pT exp mean 0.5 GeV/c, |eta|<0.9) + " \
           "3,000 secondaries + 10% noise, 36 sectors x 159 pad rows, Bz=0.5 T"


def _gen_event(job):
    kind, seed = job
    from paper_1712_09430_gb300 import synth
    if kind == "timeframe":
        ev = synth.time_frame(seed=seed[0], n_coll=seed[1])
        return ev.clusters, ev.row_counts, ev.label, ev.track_coll, ev.coll_dz
    if kind == "tfslice":
        ev = synth.time_frame(seed=seed[0], n_coll=seed[1])
        return ev.clusters, ev.row_counts
    ev = synth.central_event(seed=seed) if kind == "central" else synth.min_bias_event(seed)
    return ev.clusters, ev.row_counts


def make_inputs(central_seeds, mb_seeds, tf=None, slices=()):
    """Central batch, min-bias pool, (tf = (seed, collisions)) a
    continuous-readout time frame and (slices = [(seed, collisions)]) time-frame
    slices, generated in a spawned process pool (it starts before any CUDA use
    in this process).  The frame and the slices come back only when asked for."""
    jobs = [("timeframe", tf)] if tf else []
    jobs += [("tfslice", sl) for sl in slices]
    jobs += [("central", s) for s in central_seeds] + [("minbias", s) for s in mb_seeds]
    # the longest jobs first, so that they overlap the many short ones
    with mp.get_context("spawn").Pool(min(len(jobs), max(1, os.cpu_count() or 1), 16)) as pool:
        parts = pool.map(_gen_event, jobs, chunksize=1)
    frame = parts.pop(0) if tf else None
    sl = [parts.pop(0) for _ in slices]
    nc = len(central_seeds)
    cl = np.ascontiguousarray(np.concatenate([p[0] for p in parts[:nc]]))
    rc = np.ascontiguousarray(np.concatenate([p[1] for p in parts[:nc]]))
    out = [cl, rc, parts[nc:]]
    if tf:
        out.append(frame)
    if slices:
        out.append(sl)
    return tuple(out)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seconds_target=15.0, ev=None):
    """The FP64 oracle, as it stands, on the host cores: all cores over whole
    central events (OpenMP over (event, sector) units) for ~seconds_target,
    plus 1 and 4 threads (the paper's four CPU cores) on a 6-sector sample."""
    import oracle
    from paper_1712_09430_gb300 import synth
    if ev is None:
        ev = synth.central_event(seed=3)
    cores = os.cpu_count() or 1
    done, t0 = 0, time.perf_counter()
    n_ev = 0
    while True:
        oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, synth.row_x(), mode="f64", threads=cores)
        done += ev.n
        n_ev += 1
        if time.perf_counter() - t0 > seconds_target:
            break
    dt = time.perf_counter() - t0
    # six sectors (one side's first six) of the same event as one unit set
    rc = ev.row_counts.reshape(36, 159)
    sel = np.zeros(36, bool)
    sel[:6] = True
    ncl = int(rc[:6].sum())
    rc6 = np.where(sel[:, None], rc, 0).reshape(-1).astype(np.int32)
    cl6 = ev.clusters[:ncl]
    per_threads = {}
    for th in (1, 4):
        t1 = time.perf_counter()
        oracle.run(cl6, rc6, 1, ev.bz, synth.row_x(), mode="f64", threads=th)
        per_threads[str(th)] = ncl / (time.perf_counter() - t1)
    per_threads[str(cores)] = done / dt
    # the FP32_EXACT mode (binary32 expressions without fused multiply-add)
    # on all cores, one event
    t1 = time.perf_counter()
    oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, synth.row_x(), mode="f32", threads=cores)
    f32 = ev.n / (time.perf_counter() - t1)
    return {"value": done / dt, "unit": "clusters/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_ev} x one central Pb-Pb event ({ev.n} clusters), FP64 oracle, "
                      f"OpenMP over the 36 sectors, {dt:.1f} s wall; 1 and 4 threads on sectors "
                      f"0-5 of the same event ({ncl} clusters); FP32_EXACT mode on one event, all cores",
            "by_threads": per_threads, "f32_exact_all_cores": f32}


def run_reference(args):
    """Reference arm: the CPU oracle, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1712_09430_gb300 import synth
    # the same events as the GPU arm's step (seeds 3.. of its batch), one per
    # step in turn: a bounded sample of that workload
    seeds = rank_seeds(0, args.batch)
    n_ev = max(1, min(len(seeds), args.steps))
    # the whole step's events name the workload (the same config as the GPU
    # arm's); the first n_ev of them are timed
    all_evs = [synth.central_event(seed=s) for s in seeds]
    evs = all_evs[:n_ev]
    cores = os.cpu_count() or 1
    for i in range(max(0, args.warmup)):
        ev = evs[i % n_ev]
        oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, synth.row_x(), mode="f64", threads=cores)
    times, n_cl = [], 0
    for i in range(args.steps):
        ev = evs[i % n_ev]
        t0 = time.perf_counter()
        oracle.run(ev.clusters, ev.row_counts, 1, ev.bz, synth.row_x(), mode="f64", threads=cores)
        times.append(time.perf_counter() - t0)
        n_cl += ev.n
    tot = sum(times)
    value = n_cl / tot
    line = {"metric": METRIC, "value": value, "unit": "clusters/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": step_config(len(seeds), sum(ev.n for ev in all_evs), args.gpus),
            "cpu_baseline": {"value": value, "unit": "clusters/s", "cores": cores, "kind": "oracle",
                             "sample": f"one of the GPU step's {len(seeds)} central events per step "
                                       f"(seeds {seeds[0]}-{seeds[-1]} in turn), {args.steps} steps, "
                                       f"FP64 oracle, OpenMP over the 36 sectors"},
            "e2e": {"value": value, "unit": "clusters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def step_config(batch, n_clusters, world):
    """The workload of one step, as both arms name it: `batch` central
    events per GPU, `n_clusters` of them on rank 0 (every rank's events are
    drawn from the same distribution)."""
    return {"workload": WORKLOAD, "events_per_step": batch * world, "events_per_rank": batch,
            "clusters_per_step": int(n_clusters) * world,
            "l2": f"inputs larger than L2 ({n_clusters * 16 / 1e6:.0f} MB of clusters per step)",
            "parallelism": f"events sharded over {world} GPU(s), no collective"}


def rank_seeds(rank, batch, base=3):
    """Event seeds of one rank: ranks track disjoint events (weak scaling,
    no data-path collective)."""
    return [base + rank * batch + i for i in range(batch)]


def reduce_step_ms(ms, dist, device=None):
    """Whole-job step time = the slowest rank's (max over ranks)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# Launches of our kernels per batched step: plan, grid, neighbours, clean,
# start tiles, start top, start final, start write, seeds, tracklets,
# owner, accept, scan tiles, scan top, emit.
LAUNCHES_PER_STEP = 15


def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    n_central = max([args.batch] + list(args.batch_sizes))
    seeds = rank_seeds(rank, n_central)   # the step's batch is the first args.batch of them
    mb_seeds = [1000 + rank * args.pool + i for i in range(args.pool)] if args.stream_rates else []
    tf_job = (4 + rank, args.tf_collisions) if args.tf_collisions > 0 else None
    sl_jobs = list(args.tf_slices)   # the same slices on every rank
    cl_all, rc_all, mb_pool, *extra = make_inputs(seeds, mb_seeds, tf_job, sl_jobs)   # before any CUDA use
    frame = extra.pop(0) if tf_job else None
    slices = extra.pop(0) if sl_jobs else None
    units_per_event = 36 * 159
    cl_np = np.ascontiguousarray(cl_all[:int(rc_all[:args.batch * units_per_event].sum())])
    rc_np = np.ascontiguousarray(rc_all[:args.batch * units_per_event])
    import torch
    import ctypes as C
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1712_09430_gb300 import capi, synth
    from paper_1712_09430_gb300.tracker import Tracker, TRACK_DTYPE
    L = capi.lib()
    B = args.batch
    N = len(cl_np)
    tr = Tracker(synth.row_x(), bz=0.5, use_graph=1, exact_fp32=1 if args.exact else 0,
                 bin_target=args.bin_target, threads_per_row=args.threads_per_row,
                 tracklets_per_warp=args.tracklets_per_warp, schedule=args.schedule,
                 lanes_per_hit=args.lanes_per_hit)
    stream = torch.cuda.Stream()
    sp = C.c_void_p(stream.cuda_stream)
    dev_cl = torch.from_numpy(cl_np).to(f"cuda:{local}")
    cap_t, cap_h = N // 10 + 1024, N
    out_tr = torch.empty(cap_t * TRACK_DTYPE.itemsize, dtype=torch.uint8, device=dev_cl.device)
    out_h = torch.empty(cap_h, dtype=torch.int32, device=dev_cl.device)
    out = capi.tpc_output(out_tr.data_ptr(), out_h.data_ptr(), cap_t, cap_h, capi.TPC_MEM_DEVICE, 0, 0)
    rc_ptr = rc_np.ctypes.data_as(C.c_void_p)

    def step():
        r = L.tpc_track_sectors(tr.h, C.c_void_p(dev_cl.data_ptr()), rc_ptr, B,
                                capi.TPC_MEM_DEVICE, C.byref(out), sp)
        if r != capi.TPC_OK:
            raise RuntimeError(f"tpc_track_sectors: {capi.STATUS_NAMES.get(r)}: {tr.error()}")

    tuned = None
    if args.autotune:
        from paper_1712_09430_gb300 import autotune
        fields, tuned_ms = autotune.tune(tr, dev_cl, rc_np, B, reps=3)
        tuned = dict(fields, ms=tuned_ms)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage = np.zeros(7)
    t0 = time.perf_counter()
    for i in range(args.steps):
        ev_s[i].record(stream)
        step()
        ev_e[i].record(stream)
        stage += np.array(tr.stage_times())
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    ck = clocks.stop()
    ms = sum(s.elapsed_time(e) for s, e in zip(ev_s, ev_e)) / args.steps
    stage /= args.steps
    ms = reduce_step_ms(ms, dist, dev_cl.device)
    M, MH = out.n_tracks, out.n_hits
    T = len(tr.dump(capi.TPC_DUMP_STARTS)) if rank == 0 else 0
    # the tracklet kernel's own work counts of this batch, from one more call
    # with counting on (untimed; the timed calls do not count), taken before
    # other legs run other batches through the same tracker
    algo_step = None
    if rank == 0:
        tr.set_params(count_work=1)
        step()
        algo_step = algorithmic_bytes(tr, N, T)
        tr.set_params(count_work=0)
    value = N * world / (ms * 1e-3)

    # ---- end to end through the C ABI with pinned host buffers
    e2e = e2e_sync = None
    if not args.no_e2e:
        e2e_sync = run_e2e(L, tr, cl_np, rc_ptr, rc_np, B, N, world, sp, cap_t, cap_h, args)
        e2e_sync["api"] = "tpc_track_sectors with host buffers (synchronous: H2D, kernels, D2H in turn)"
        e2e = run_e2e_stream(tr, cl_np, rc_np, B, N, world, args)
    plain = multi = None
    if args.plain_steps > 0:
        plain = run_plain(L, tr, dev_cl, rc_ptr, B, N, world, sp, out, args, mode=1)
        multi = run_plain(L, tr, dev_cl, rc_ptr, B, N, world, sp, out, args, mode=2)
    stream_res = None
    if args.stream_rates:
        stream_res = [run_stream(tr, mb_pool, args, rate) for rate in args.stream_rates]
    stream_central = None
    if args.stream_central_rates:
        upe = 36 * 159
        offs = np.r_[0, np.cumsum([int(rc_np[e * upe:(e + 1) * upe].sum()) for e in range(B)])]
        central_pool = [(np.ascontiguousarray(cl_np[offs[e]:offs[e + 1]]),
                         np.ascontiguousarray(rc_np[e * upe:(e + 1) * upe])) for e in range(B)]
        stream_central = [run_stream(tr, central_pool, args, rate, batch=args.batch,
                                     workload=f"central Pb-Pb-like events (the step's {B} events, "
                                              "sampled with replacement), Poisson arrivals, one event "
                                              "per request")
                          for rate in args.stream_central_rates]
    batch_sizes = None
    if args.batch_sizes:
        batch_sizes = run_batch_sizes(L, tr, cl_all, rc_all, args, dev_cl.device, sp)
    refit = None
    if args.refit_steps > 0:
        refit = run_refit(L, tr, dev_cl, rc_ptr, B, sp, out, out_tr, out_h, args)
    tframe = None
    if frame is not None:
        tframe = run_time_frame(frame, tr, args, dev_cl.device)
    if slices:
        tframe = tframe or {}
        tframe["uneven_slices"] = run_slices(slices, tr, args, dev_cl.device)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # ---- roofline of the dominant kernel (tracklet construction)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    names = ["grid", "neighbours", "clean+starts", "tracklets", "select+emit"]
    stage_ms = {n: float(v) for n, v in zip(names, stage[:5])}
    dom = max(stage_ms, key=stage_ms.get)
    algo = algo_step if dom == "tracklets" else None
    rl = None
    if algo is not None:
        t_s = stage_ms[dom] * 1e-3
        # the headline: the hot path's per-cluster byte model of the stage
        # (every stage reads its inputs and writes its outputs once: 55 B per
        # input cluster for tracklet construction) x the clusters of a launch
        model_bytes = TRACKLET_MODEL_BYTES_PER_CLUSTER * N
        achieved = model_bytes / t_s / 1e9
        traffic = None
        if B == 8 and not args.exact:
            traffic = measured_traffic(TRACKLET_SOURCES, TRACKLET_TRAFFIC_SUMMARY)
        rl = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
              "frac": achieved / hbm, "traffic": traffic, "kernel": TRACKLET_KERNEL,
              "algorithmic_bytes_per_launch": model_bytes,
              "model": f"{TRACKLET_MODEL_BYTES_PER_CLUSTER} B per input cluster x {N} clusters",
              # the kernel's own count of what it reads and writes (row steps,
              # bin-table rows, candidates), from one untimed counting call
              "frac_counted": algo["bytes"] / t_s / 1e9 / hbm,
              "counted_bytes_per_launch": algo["bytes"], "counted_model": algo["model"],
              # DRAM bytes of one launch (ncu) over the same time
              "frac_dram": (traffic / t_s / 1e9 / hbm) if traffic else None,
              # the whole step against the model's 220 B per cluster
              "frac_step": STEP_MODEL_BYTES_PER_CLUSTER * N / (ms * 1e-3) / 1e9 / hbm,
              "counts": {k: v for k, v in algo.items() if k not in ("bytes", "model")},
              "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy) of measured" if peaks else "fallback"}
    cpu = None if args.no_cpu_baseline else cpu_baseline(args.cpu_seconds)
    line = {"metric": METRIC, "value": value, "unit": "clusters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": step_config(B, int(N), world),
            "execution": {"tracks_per_step": int(M), "tracklets_per_step": int(T),
                          "mode": "exact" if args.exact else "production",
                          "launch": "batched, CUDA graph replay",
                          "autotuned": tuned is not None,
                          "bin_target": float(tr.params.bin_target),
                          "threads_per_row": int(tr.params.threads_per_row),
                          "tracklets_per_warp": int(tr.params.tracklets_per_warp),
                          "lanes_per_hit": int(tr.params.lanes_per_hit),
                          "schedule": int(tr.params.schedule)},
            "events_per_s": B * world / (ms * 1e-3),
            "stage_ms": stage_ms, "wall_s": wall,
            "gpu_launches": LAUNCHES_PER_STEP * args.steps,
            "clocks": ck, "e2e": e2e, "e2e_sync": e2e_sync, "roofline": rl, "cpu_baseline": cpu,
            "plain_per_sector": plain, "multi_queue_per_sector": multi, "stream": stream_res,
            "refit": refit, "time_frame": tframe, "batch_sizes": batch_sizes,
            "stream_central": stream_central}
    if stream_res:
        line["latency_ms"] = {"p50": stream_res[0]["p50_ms"], "p99": stream_res[0]["p99_ms"],
                              "rate_hz": stream_res[0]["rate_hz"]}
    print(json.dumps(line), flush=True)
    tr.close()
    if dist:
        dist.destroy_process_group()


# Algorithmic FP32 operations of one refit step (k_refit.cu; a division or a
# square root counts as one): the helix step with its midpoint field and
# Jacobian (85) plus the square-root transport S <- J S (60), and two scalar
# Potter updates of 129 each.
REFIT_FLOPS_PROPAGATE = 145
REFIT_FLOPS_UPDATE = 258
FP32_LANES_PER_SM = 128  # Blackwell SM: 4 x 32 FP32 lanes, one FMA (2 flops) per lane per clock


def run_refit(L, tr, dev_cl, rc_ptr, B, sp, out, out_tr, out_h, args):
    """The final full Kalman filter refit (Sec. 2 "Track fit") over the same
    batch: the batched step with params.refit = 1, the refit stage timed by
    its own CUDA events (stage 6).  Roofline: FP32 ALU (the refit does ~20
    flops per byte it moves)."""
    import ctypes as C
    import torch
    from paper_1712_09430_gb300 import capi
    from paper_1712_09430_gb300.tracker import TRACK_DTYPE
    tr.set_params(refit=1)

    def step():
        r = L.tpc_track_sectors(tr.h, C.c_void_p(dev_cl.data_ptr()), rc_ptr, B,
                                capi.TPC_MEM_DEVICE, C.byref(out), sp)
        if r != capi.TPC_OK:
            raise RuntimeError(f"tpc_track_sectors: {capi.STATUS_NAMES.get(r)}: {tr.error()}")
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.refit_steps):
        step()
        ms.append(tr.stage_times()[6])
    torch.cuda.synchronize()
    # the same with merging after the refit (Sec. 2 Phase II step 3)
    tr.set_params(merge=1)
    for _ in range(3):
        step()
    ms_merge = []
    for _ in range(args.refit_steps):
        step()
        ms_merge.append(tr.stage_times()[6])
    torch.cuda.synchronize()
    tr.set_params(refit=0, merge=0)
    M = out.n_tracks
    tracks = out_tr[:M * TRACK_DTYPE.itemsize].cpu().numpy().view(TRACK_DTYPE)
    n = tracks["nhits"].astype(np.int64)
    steps = int(np.sum(2 * (n - 1)))
    flops = float(steps) * (REFIT_FLOPS_PROPAGATE + REFIT_FLOPS_UPDATE)
    t = statistics.median(ms) * 1e-3
    props = torch.cuda.get_device_properties(dev_cl.device)
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * 2.07e9 / 1e12
    achieved = flops / t / 1e12
    merge_ms = statistics.median(ms_merge) - t * 1e3
    cpu = None
    if not args.no_cpu_baseline:
        hits = out_h[:out.n_hits].cpu().numpy()
        cpu = oracle_phase2_baseline(tracks, hits, dev_cl.cpu().numpy())
    return {"ms": t * 1e3, "merge_ms": merge_ms, "tracks": int(M), "filter_steps": steps, "cpu_baseline": cpu,
            "tracks_per_s": M / t, "clusters_per_s": float(n.sum()) / t,
            "mode": "exact" if args.exact else "production",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_refit",
                         "algorithmic_flops_per_launch": flops,
                         "model": f"2*(n-1) steps per track x ({REFIT_FLOPS_PROPAGATE} propagate + "
                                  f"{REFIT_FLOPS_UPDATE} update) FP32 ops",
                         "peak_source": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 "
                                        "lanes x 2 flops (FMA) x 2.07 GHz max SM clock (derived)"}}


def oracle_phase2_baseline(tracks, hits, clusters, bz=0.5):
    """The refit and merging oracles (FP64, as they stand, OpenMP for the
    refit) on the host cores, on the tracks of the first event of the batch:
    tracks/s of each.  tracks: host TRACK_DTYPE with hit_off into hits."""
    import oracle
    sel = np.flatnonzero(tracks["event"] == 0)
    if len(sel) == 0:
        return None
    t = tracks[sel]
    off = np.zeros(len(t) + 1, np.int64)
    off[1:] = np.cumsum(t["nhits"])
    h = np.concatenate([hits[a:a + n] for a, n in zip(t["hit_off"], t["nhits"])])
    st6 = np.concatenate([t["x"][:, None], t["p"]], axis=1).astype(np.float64)
    fp = oracle.fit_params(bz)
    t0 = time.perf_counter()
    fits = oracle.refit_lists(st6, off, h, clusters, fp, mode="f64")
    t_refit = time.perf_counter() - t0
    unit = t["event"].astype(np.int32) * 36 + t["sector"]
    x_last = clusters[h[off[1:] - 1], 0].astype(np.float64)
    t0 = time.perf_counter()
    oracle.merge_tracks(unit, fits, x_last, fp, mode="f64")
    t_merge = time.perf_counter() - t0
    return {"kind": "oracle", "cores": oracle.max_threads(), "tracks": int(len(t)),
            "refit_tracks_per_s": len(t) / t_refit, "merge_tracks_per_s": len(t) / t_merge,
            "sample": f"the {len(t)} tracks of one central event; FP64 refit oracle (OpenMP over tracks) "
                      "and merging oracle (one thread)"}


def run_time_frame(frame, tr0, args, device):
    """A continuous-readout time frame (Sec. 3.3, Run 3 conditions): overlaid
    min-bias collisions, each shifted by its unknown drift-time offset, tracked
    as one event with the whole chain: tracking, refit, merging and the
    per-collision offsets.  Inputs resident on the device; clusters/s of the
    whole chain; the collisions found against the generator's offsets."""
    import torch
    from paper_1712_09430_gb300 import synth
    from paper_1712_09430_gb300.tracker import Tracker
    cl, rc, label, track_coll, coll_dz = frame
    p = tr0.params
    dev = torch.from_numpy(cl).to(device)
    res = {}
    for name, over in (("tracking", dict(refit=0, merge=0, t0=0)),
                       ("refit_merge", dict(refit=1, merge=1, t0=0)),
                       ("chain", dict(refit=1, merge=1, t0=1))):
        tr = Tracker(synth.row_x(), bz=0.5, use_graph=1, exact_fp32=p.exact_fp32,
                     bin_target=p.bin_target, threads_per_row=p.threads_per_row,
                     tracklets_per_warp=p.tracklets_per_warp, schedule=p.schedule,
                     lanes_per_hit=p.lanes_per_hit, **over)
        try:
            for _ in range(3):
                r = tr.track(dev, rc, 1)
            torch.cuda.synchronize()
            ms, st = [], np.zeros(7)
            for _ in range(args.tf_steps):
                r = tr.track(dev, rc, 1)
                s7 = np.array(tr.stage_times())
                ms.append(s7[5])
                st += s7
            st /= args.tf_steps
        finally:
            tr.close()
        t = statistics.median(ms)
        res[name] = {"ms": t, "clusters_per_s": len(cl) / (t * 1e-3), "after_selection_ms": float(st[6]),
                     "tracks": int(len(r.tracks))}
    res["collision_offsets_ms"] = res["chain"]["ms"] - res["refit_merge"]["ms"]
    # collisions found by the chain against the generator's offsets
    coll = r.t0s["collision"]
    maj = np.full(len(coll), -1)
    for m in np.flatnonzero(coll >= 0):
        v, c = np.unique(label[r.hits_of(m)], return_counts=True)
        if v[np.argmax(c)] >= 0:
            maj[m] = track_coll[v[np.argmax(c)]]
    found = np.unique(coll[coll >= 0])
    good = 0
    for k in found:
        sel = coll == k
        if np.any(maj[sel] >= 0):
            tc = np.bincount(maj[sel][maj[sel] >= 0]).argmax()
            good += abs(float(r.t0s["dz"][sel][0]) - coll_dz[tc]) < 0.3
    if not args.no_cpu_baseline:
        import oracle
        f = r.fits
        fits = np.concatenate([f["x"][:, None], f["p"], f["cov"], f["chi2"][:, None],
                               f["ndf"][:, None], f["status"][:, None]], axis=1).astype(np.float64)
        unit = r.tracks["event"].astype(np.int32) * 36 + r.tracks["sector"]
        t0 = time.perf_counter()
        oracle.t0_tracks(unit, fits, oracle.fit_params(0.5), mode="f64")
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"kind": "oracle", "cores": 1, "tracks_per_s": len(unit) / dt,
                               "sample": f"the collision offsets of this time frame's {len(unit)} refitted "
                                         "tracks, FP64 oracle, one thread"}
    res.update({"clusters": int(len(cl)), "collisions": int(len(coll_dz)),
                "collisions_found": int(len(found)), "found_within_0.3cm": int(good),
                "tracks_assigned": float((coll >= 0).mean()),
                "workload": f"time frame of {len(coll_dz)} min-bias collisions, each shifted by a drift "
                            "offset ~ U[-250, 250] cm (continuous readout), 10% noise"})
    return res


def run_batch_sizes(L, tr, cl_all, rc_all, args, device, sp):
    """The batched step over other numbers of central events per call (one
    and 32 events beside the eight of the headline step): graph replay,
    inputs resident, CUDA events around each call, median over the steps."""
    import ctypes as C
    import torch
    from paper_1712_09430_gb300 import capi
    from paper_1712_09430_gb300.tracker import TRACK_DTYPE
    upe = 36 * 159
    res = []
    for B in args.batch_sizes:
        rc = np.ascontiguousarray(rc_all[:B * upe])
        n = int(rc.sum())
        dev = torch.from_numpy(np.ascontiguousarray(cl_all[:n])).to(device)
        cap_t, cap_h = n // 10 + 1024, n
        out_tr = torch.empty(cap_t * TRACK_DTYPE.itemsize, dtype=torch.uint8, device=device)
        out_h = torch.empty(cap_h, dtype=torch.int32, device=device)
        out = capi.tpc_output(out_tr.data_ptr(), out_h.data_ptr(), cap_t, cap_h, capi.TPC_MEM_DEVICE, 0, 0)
        rc_ptr = rc.ctypes.data_as(C.c_void_p)
        stream = torch.cuda.Stream(device)

        def step():
            r = L.tpc_track_sectors(tr.h, C.c_void_p(dev.data_ptr()), rc_ptr, B, capi.TPC_MEM_DEVICE,
                                    C.byref(out), C.c_void_p(stream.cuda_stream))
            if r != capi.TPC_OK:
                raise RuntimeError(f"tpc_track_sectors: {capi.STATUS_NAMES.get(r)}: {tr.error()}")
        for _ in range(max(3, args.warmup)):
            step()
        steps = max(5, min(args.steps, int(2000 / max(B, 1))))
        ms = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms)
        res.append({"events": B, "clusters": n, "ms": t, "clusters_per_s": n / (t * 1e-3),
                    "events_per_s": B / (t * 1e-3), "steps": steps, "tracks": int(out.n_tracks)})
        del dev, out_tr, out_h
    return res


def run_slices(slices, tr0, args, device):
    """Continuous-readout time-frame slices of uneven size (about 1, 2, 3, 5
    and 8 M clusters) tracked together in one launch, each slice one event:
    tracking alone and the whole chain (refit, merging, collision offsets).
    Inputs resident on the device; clusters/s of the batch."""
    import torch
    from paper_1712_09430_gb300 import synth
    from paper_1712_09430_gb300.tracker import Tracker
    cl = np.ascontiguousarray(np.concatenate([s[0] for s in slices]))
    rc = np.ascontiguousarray(np.concatenate([s[1] for s in slices]))
    E = len(slices)
    p = tr0.params
    dev = torch.from_numpy(cl).to(device)
    res = {}
    for name, over in (("tracking", dict(refit=0, merge=0, t0=0)), ("chain", dict(refit=1, merge=1, t0=1))):
        tr = Tracker(synth.row_x(), bz=0.5, use_graph=1, exact_fp32=p.exact_fp32,
                     bin_target=p.bin_target, threads_per_row=p.threads_per_row,
                     tracklets_per_warp=p.tracklets_per_warp, schedule=p.schedule,
                     lanes_per_hit=p.lanes_per_hit, **over)
        try:
            for _ in range(3):
                r = tr.track(dev, rc, E)
            ms, st = [], np.zeros(7)
            for _ in range(args.tf_steps):
                r = tr.track(dev, rc, E)
                s7 = np.array(tr.stage_times())
                ms.append(s7[5])
                st += s7
            st /= args.tf_steps
        finally:
            tr.close()
        t = statistics.median(ms)
        names = ["grid", "neighbours", "clean+starts", "tracklets", "select+emit"]
        res[name] = {"ms": t, "clusters_per_s": len(cl) / (t * 1e-3), "tracks": int(len(r.tracks)),
                     "stage_ms": {n: float(v) for n, v in zip(names, st[:5])},
                     "after_selection_ms": float(st[6])}
    res.update({"clusters": int(len(cl)), "slice_clusters": [int(len(s[0])) for s in slices],
                "slice_collisions": [n for _, n in args.tf_slices], "launches": "one batch of all slices",
                "workload": "continuous-readout time-frame slices of uneven size, min-bias collisions "
                            "shifted by drift offsets ~ U[-250, 250] cm, 10% noise, one event each"})
    return res


def run_plain(L, tr, dev_cl, rc_ptr, B, N, world, sp, out, args, mode=1):
    """The same batch with every stage launched once per (event, sector) unit:
    mode 1 on one stream (the Run 1/2 scheduling), mode 2 round-robin over 8
    streams (the multi-queue scheme), for comparison."""
    import ctypes as C
    import torch
    from paper_1712_09430_gb300 import capi
    tr.set_params(plain_per_sector=mode, use_graph=0, n_queues=8)
    try:
        def step():
            r = L.tpc_track_sectors(tr.h, C.c_void_p(dev_cl.data_ptr()), rc_ptr, B,
                                    capi.TPC_MEM_DEVICE, C.byref(out), sp)
            if r != capi.TPC_OK:
                raise RuntimeError(f"plain form: {tr.error()}")
        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.plain_steps):
            step()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.plain_steps
    finally:
        tr.set_params(plain_per_sector=0, use_graph=1)
    units = B * 36
    return {"value": N * world / dt, "unit": "clusters/s", "ms_per_step": dt * 1e3,
            "steps": args.plain_steps, "launches_per_step": units * 9 + 7,
            "note": "every stage launched per (event, sector) unit, " +
                    ("on one stream" if mode == 1 else "round-robin over 8 streams")}


MINBIAS_STREAM = ("min-bias events (b ~ U[0,15] fm, 10-10,000 primaries + 30% secondaries, "
                  "10% noise), Poisson arrivals, one event per request")


def run_stream(tr0, pool, args, rate, batch=None, workload=MINBIAS_STREAM):
    """Serving: Poisson arrivals of events (sampled with replacement from the
    pool) at `rate` Hz for args.stream_seconds, through tpc_stream_submit/poll,
    at most `batch` events and the library's default cluster limit (about 4 M)
    per batch.  Latency = result in hand - arrival (includes queueing, H2D,
    the batched stages and D2H)."""
    batch = batch or args.stream_batch
    from paper_1712_09430_gb300 import synth
    from paper_1712_09430_gb300.tracker import Tracker
    p = tr0.params
    tr = Tracker(synth.row_x(), bz=0.5, exact_fp32=p.exact_fp32, bin_target=p.bin_target,
                 threads_per_row=p.threads_per_row, tracklets_per_warp=p.tracklets_per_warp,
                 schedule=p.schedule, lanes_per_hit=p.lanes_per_hit)
    try:
        import torch
        # events arrive in pinned host memory (as from a readout link) and are
        # submitted without a copy; each stays untouched until its result is in
        pool = [(torch.from_numpy(cl).pin_memory(), rc) for cl, rc in pool]
        tr.stream_configure(arena_bytes=args.stream_arena_gb << 30, max_batch_events=batch,
                            max_inflight=args.stream_inflight, no_copy=True,
                            max_batch_clusters=args.stream_batch_clusters)
        tr.stream_set_batching(args.stream_min_batch_clusters, args.stream_max_wait_us)
        rng = np.random.default_rng(5)
        n_req = args.stream_requests or int(rate * args.stream_seconds)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        picks = rng.integers(0, len(pool), n_req)
        # warm-up: one burst of a full batch (the result buffers reach their
        # working size), then a few single requests, drained
        for burst in (min(batch, len(pool)), 1, 1, 1, 1):
            warm = [tr.submit(pool[i][0], pool[i][1], 1) for i in range(burst)]
            for t in warm:
                while t is not None and tr.poll(t, 1000) is None:
                    pass
        lat = np.zeros(n_req)
        clusters = 0
        nxt, done = 0, 0
        outstanding = {}
        backlog = []
        t_submit = t_poll = 0.0
        n_tracks = 0
        # the client's own garbage collection would show as request latency:
        # off while timing
        import gc
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        last = 0.0
        max_gap, max_gap_at = 0.0, 0.0   # the longest pass of the client loop (a host-side stall)
        while done < n_req:
            now = time.perf_counter() - t0
            if now - last > max_gap:
                max_gap, max_gap_at = now - last, last
            last = now
            while nxt < n_req and arrivals[nxt] <= now:
                backlog.append(nxt)
                nxt += 1
            while backlog:
                i = backlog[0]
                cl, rc = pool[picks[i]]
                ts = time.perf_counter()
                t = tr.submit(cl, rc, 1, tag=i)
                t_submit += time.perf_counter() - ts
                if t is None:
                    break               # not admitted now (memory/slots): retry later
                outstanding[t] = i
                backlog.pop(0)
            # take every result that is ready, in the order the batches
            # finished (one call per result, no scan over pending tickets);
            # with nothing to submit, wait in the library until the next
            # arrival is due
            wait_us = 0
            if not backlog and nxt < n_req:
                wait_us = int(max(0.0, min(1e-4, arrivals[nxt] - (time.perf_counter() - t0))) * 1e6)
            while True:
                ts = time.perf_counter()
                got = tr.poll_any(wait_us)
                t_poll += time.perf_counter() - ts
                if got is None:
                    break
                wait_us = 0
                t, r = got
                n_tracks += len(r.tracks)   # the tracks are read in place
                tr.release(t)
                i = outstanding.pop(t)
                lat[i] = time.perf_counter() - t0 - arrivals[i]
                clusters += len(pool[picks[i]][0])
                done += 1
        wall = time.perf_counter() - t0
        gc.enable()
        st = tr.stream_stats()
    finally:
        tr.close()
    st["gpu_busy_frac"] = st["gpu_ms"] / (wall * 1e3)
    st["client_submit_s"] = t_submit
    st["client_poll_s"] = t_poll
    st["mean_batch_events"] = st["events"] / max(st["batches"], 1)
    return {"rate_hz": rate, "requests": n_req, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "loop": st,
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_ms": float(lat.max() * 1e3),
            "max_arrival_s": float(arrivals[int(np.argmax(lat))]),
            "client_max_gap_ms": max_gap * 1e3, "client_max_gap_at_s": max_gap_at,
            "clusters_per_s": clusters / wall, "events_per_s": n_req / wall, "wall_s": wall,
            "tracks": n_tracks, "client": "tpc_stream_poll_any + tpc_stream_release (results read in place)",
            "batches_in_flight": args.stream_inflight,
            "batch_clusters_max": args.stream_batch_clusters,
            "batching": {"min_batch_clusters": args.stream_min_batch_clusters,
                         "max_wait_us": args.stream_max_wait_us},
            "pool_events": len(pool), "mean_clusters_per_event": float(np.mean([len(p[0]) for p in pool])),
            "max_batch_events": batch, "workload": workload}


def run_e2e(L, tr, cl_np, rc_ptr, rc_np, B, N, world, sp, cap_t, cap_h, args):
    """Same metric through the C ABI with pinned HOST input and output: the
    H2D of the clusters and row counts and the D2H of the tracks are inside
    every timed step."""
    import ctypes as C
    import torch
    from paper_1712_09430_gb300 import capi
    from paper_1712_09430_gb300.tracker import TRACK_DTYPE
    pin_cl = torch.from_numpy(cl_np).pin_memory()
    host_tr = torch.empty(cap_t * TRACK_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    host_h = torch.empty(cap_h, dtype=torch.int32).pin_memory()
    hout = capi.tpc_output(host_tr.data_ptr(), host_h.data_ptr(), cap_t, cap_h, capi.TPC_MEM_HOST,
                           0, 0)

    def step_e2e():
        r = L.tpc_track_sectors(tr.h, C.c_void_p(pin_cl.data_ptr()), rc_ptr, B, capi.TPC_MEM_HOST,
                                C.byref(hout), sp)
        if r != capi.TPC_OK:
            raise RuntimeError(f"tpc_track_sectors (host): {tr.error()}")

    for _ in range(3):
        step_e2e()
    torch.cuda.synchronize()
    k2 = max(3, args.steps // 2)
    t1 = time.perf_counter()
    for _ in range(k2):
        step_e2e()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t1) / k2
    h2d = N * 16 + len(rc_np) * 4
    d2h = hout.n_tracks * TRACK_DTYPE.itemsize + hout.n_hits * 4 + 64
    return {"value": N * world / e2e_s, "unit": "clusters/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3, "steps": k2}


def run_e2e_stream(tr0, cl_np, rc_np, B, N, world, args):
    """Same metric end to end through the serving API: every step submits the
    8-event batch from pinned host memory (tpc_stream_submit, no copy) and
    takes its tracks from the library's pinned result buffers
    (tpc_stream_poll_view); two batches are in flight, so one batch's H2D and
    D2H overlap the other's kernels (the pipelining of Sec. 3.1)."""
    import torch
    from collections import deque
    from paper_1712_09430_gb300 import synth
    from paper_1712_09430_gb300.tracker import TRACK_DTYPE, Tracker
    p = tr0.params
    tr = Tracker(synth.row_x(), bz=0.5, exact_fp32=p.exact_fp32, bin_target=p.bin_target,
                 threads_per_row=p.threads_per_row, tracklets_per_warp=p.tracklets_per_warp,
                 schedule=p.schedule, lanes_per_hit=p.lanes_per_hit)
    try:
        pin = torch.from_numpy(cl_np).pin_memory()
        tr.stream_configure(arena_bytes=args.stream_arena_gb << 30, max_batch_events=B, max_inflight=2,
                            no_copy=True)
        state = {"tracks": 0, "hits": 0}

        def take(t):
            r = None
            while r is None:
                r = tr.poll_view(t, timeout_us=1000)
            state["tracks"] = len(r.tracks)
            state["hits"] = len(r.hit_ids)
            tr.release(t)

        def run(k):
            q = deque()
            for _ in range(k):
                t = tr.submit(pin, rc_np, B)
                while t is None:          # not admitted now: finish the oldest first
                    take(q.popleft())
                    t = tr.submit(pin, rc_np, B)
                q.append(t)
                if len(q) > 2:
                    take(q.popleft())
            while q:
                take(q.popleft())
        run(3)
        torch.cuda.synchronize()
        # the pipeline fills and drains once per timed run: enough steps that
        # this costs little
        k2 = max(20, args.steps)
        t1 = time.perf_counter()
        run(k2)
        e2e_s = (time.perf_counter() - t1) / k2
    finally:
        tr.close()
    h2d = N * 16 + len(rc_np) * 4
    d2h = state["tracks"] * TRACK_DTYPE.itemsize + state["hits"] * 4 + 64
    return {"value": N * world / e2e_s, "unit": "clusters/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3, "steps": k2,
            "api": "tpc_stream_submit (no copy) + tpc_stream_poll_view/release, two batches in flight: "
                   "H2D and D2H of one batch overlap the kernels of the other"}


def measured_traffic(kernel_sources, summary):
    """DRAM bytes per launch of the tracklet kernel from a committed ncu
    summary, valid only while the kernel's sources are the ones it was taken
    on (the SHA-1 of their concatenation is recorded in the summary); None
    otherwise."""
    import hashlib
    try:
        h = hashlib.sha1()
        for path in kernel_sources:
            h.update(open(path, "rb").read())
        src = h.hexdigest()
        fields = {}
        for line in open(summary):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                fields[k.strip().strip("`- ")] = v.strip().strip("`")
    except OSError:
        return None
    if fields.get("source_sha1") != src:
        return None
    try:
        return float(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# Byte model of the hot path, each stage reading its inputs and writing its
# outputs once: tracklet construction about 55 B per input cluster (about 2
# row steps per cluster x (8 B bin entry + 16 B candidate + 4 B hit id)); the
# whole step about 220 B per cluster.
TRACKLET_MODEL_BYTES_PER_CLUSTER = 55
STEP_MODEL_BYTES_PER_CLUSTER = 220
TRACKLET_KERNEL = "k_tracklets_sched"
TRACKLET_SOURCES = [os.path.join(ROOT, "paper_1712_09430_gb300", "csrc", f) for f in ("k_fp.cu", "tpc_dev.cuh")]
TRACKLET_TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "k_tracklets_sched_traffic_central8.md")


def algorithmic_bytes(tr, N, T):
    """Bytes the tracklet constructor moves by its own stage structure,
    counted exactly per tracklet by the kernel (TPC_DUMP_TRACKLET_WORK, from a
    call with params.count_work = 1):
    per row step the row grid record (16 B), per bin-table row read two offsets
    (8 B), per candidate cluster examined 8 B (its y, z), per Phase-2 cluster a
    4 B write, and per tracklet its 80 B start record in (the state after the
    seed chain, filtered by the seed kernel, and its row information) and 68 B
    of state out."""
    from paper_1712_09430_gb300 import capi
    w = tr.dump(capi.TPC_DUMP_TRACKLET_WORK).astype(np.int64)
    n_hits = int(tr.dump(capi.TPC_DUMP_TRACKLET_N)[0].astype(np.int64).sum())
    steps, binrows, cand, chain = (int(v) for v in w.sum(axis=1))
    b = 16 * steps + 8 * binrows + 8 * cand + 4 * n_hits + T * (80 + 68)
    return {"bytes": float(b), "row_steps": steps, "bin_rows": binrows, "candidates": cand,
            "chain_hits": chain, "tracklet_hits": n_hits,
            "model": "16*row_steps + 8*bin_rows + 8*candidates + 4*hits + 148*T"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=8, help="central events per step (per GPU)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--exact", action="store_true", help="time the -fmad=false build")
    ap.add_argument("--bin-target", type=float, default=0.25)
    ap.add_argument("--threads-per-row", type=int, default=128)
    ap.add_argument("--tracklets-per-warp", type=int, default=32)
    ap.add_argument("--lanes-per-hit", type=int, default=1,
                    help="lanes sharing one hit in the neighbour finder (1, 2, 4, 8)")
    ap.add_argument("--schedule", type=int, default=2,
                    help="0 unit by unit, 1 by start row, 2 by start row inside blocks of ~2 M clusters")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="use the given execution parameters instead of tuning them first")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling)")
    ap.add_argument("--plain-steps", type=int, default=3, help="steps of the plain per-sector form")
    ap.add_argument("--stream-rates", type=lambda v: [float(x) for x in v.split(",") if x.strip()],
                    default=[1000.0, 3000.0, 5000.0],
                    help="Poisson arrival rates (Hz) of the serving leg, comma separated; '' = off")
    ap.add_argument("--stream-seconds", type=float, default=3.0)
    ap.add_argument("--stream-central-rates", type=lambda v: [float(x) for x in v.split(",") if x.strip()],
                    default=[250.0, 500.0, 1000.0],
                    help="Poisson arrival rates (Hz) of central events through the serving API; '' = off")
    ap.add_argument("--refit-steps", type=int, default=10,
                    help="steps of the final-refit leg (0: skip)")
    ap.add_argument("--tf-collisions", type=int, default=50,
                    help="collisions of the continuous-readout time-frame leg (0: skip)")
    ap.add_argument("--tf-steps", type=int, default=5)
    ap.add_argument("--batch-sizes", type=lambda v: [int(x) for x in v.split(",") if x.strip()],
                    default=[1, 32], help="other central events per call to time beside --batch; '' = off")
    ap.add_argument("--tf-slices",
                    type=lambda v: [tuple(int(y) for y in x.split(":")) for x in v.split(",") if x.strip()],
                    default=[(47, 8), (44, 16), (42, 24), (43, 40), (44, 64)],
                    help="seed:collisions of each time-frame slice of the uneven-slice batch; the "
                         "default gives 0.9, 2.0, 3.2, 4.9 and 8.5 M clusters; '' = off")
    ap.add_argument("--stream-batch", type=int, default=16,
                    help="most events per serving batch (a large batch formed after a burst "
                         "holds all its requests until its last kernel)")
    ap.add_argument("--stream-arena-gb", type=int, default=16)
    ap.add_argument("--stream-inflight", type=int, default=2, help="serving batches in flight")
    ap.add_argument("--stream-batch-clusters", type=int, default=1 << 22,
                    help="most clusters in one serving batch (the library's default: 2^22)")
    ap.add_argument("--stream-min-batch-clusters", type=int, default=1 << 20,
                    help="serving: while a batch runs, form the next once this many clusters are "
                         "pending (0: whenever a slot is free)")
    ap.add_argument("--stream-max-wait-us", type=int, default=1000,
                    help="serving: ... or once the oldest pending request has waited this long")
    ap.add_argument("--stream-requests", type=int, default=0,
                    help="requests per serving rate (0: rate x --stream-seconds)")
    ap.add_argument("--pool", type=int, default=96, help="min-bias events in the serving pool")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
