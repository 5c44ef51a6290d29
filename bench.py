#!/usr/bin/env python3
"""Benchmark of the Voronoi point-inclusion test (arXiv 2007.15385) on GB300.

One step = one pip_test over the vehicle-footprint workload: a 12-vertex
convex footprint (2.4 m x 1.0 m ellipse) against 2^26 float32 lidar-like
points, packed inclusion bitmask out, bit-exact (float32 filter + exact
refine).  The metric is point x edge tests per second (full work: every point
meets every edge).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

At one GPU the line also carries a ``workloads`` object: the octagon, the
ragged GIS batch, the GIS all-pairs first hit, the integer hulls and the
collision penalty, each with its call and kernel times, HBM and FP32 rooflines
(the FP32 peak measured in the same run by a pure-FFMA kernel, beside the
nominal one), refine fraction, CUDA-graph replay, comparators and the oracle on
a bounded sample.  Under torchrun each rank runs the headline workload on its
own GPU (weak scaling, no data-path collective); rank 0 prints one JSON line.
``--impl reference`` times the CPU oracle (exact predicate, one thread) on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Gtests/s (point×edge) and % of HBM/FP32 roofline; "
          "Voronoi vs sign-of-offset/ray on GB300")
UNIT = "Gtests/s"
WORKLOAD = "vehicle_footprint"
NUM_POINTS = 1 << 26
FALLBACK_HBM_GBS = 6800.0

# dram bytes (read + write) per launch of the pipelined kernel on this
# workload, from one ncu capture of 2^25 points scaled by 2 to the 2^26-point
# launch, valid only while the kernel sources hash to the value recorded with it.
# keyed by the tile variant the autotuner picks (2: 24 points per lane x 2
# stages, 3: 20 x 2, 4: 24 x 2 at 16 consumer warps)
NCU_TRAFFIC = {"bytes_by_variant": {2: 548285440, 3: 548588032, 4: 548974592}, "sources_sha": "15dc8a5832480fdb"}
# GB300 HBM3e nominal bandwidth, reported beside the measured-peak fraction
NOMINAL_HBM_GBS = 7900.0
KERNEL_SOURCES = ["paper_2007_15385_gb300/csrc/pip_stream_tma.cuh",
                  "paper_2007_15385_gb300/csrc/pip_tma.cuh",
                  "paper_2007_15385_gb300/csrc/pip_kernels.cuh",
                  "paper_2007_15385_gb300/csrc/pip_internal.cuh",
                  "paper_2007_15385_gb300/csrc/pip_stream_launch.cuh",
                  "paper_2007_15385_gb300/csrc/pip_stream.cu"]


def sources_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the GPU works."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.period)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def cpu_baseline_run(w, sample: int) -> dict:
    """The oracle on the first `sample` points: the exact predicate on one
    thread (the value), the same on every host core (contiguous pieces, one
    per thread; the C calls release the GIL) and the literal fp64 Alg. 5 on
    one thread."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    pts = np.ascontiguousarray(w.points[:sample])
    n = int(w.edges()[0])
    oracle.inside_exact(w.vertices, pts[:1024])  # build + warm
    t0 = time.perf_counter()
    oracle.inside_exact(w.vertices, pts)
    dt = time.perf_counter() - t0
    threads = os.cpu_count() or 1
    pieces = np.array_split(pts, threads)
    with ThreadPoolExecutor(threads) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda q: oracle.inside_exact(w.vertices, np.ascontiguousarray(q)), pieces))
        dt_all = time.perf_counter() - t0
    half = pts[:sample // 2]
    t0 = time.perf_counter()
    oracle.voronoi_fp64(w.vertices, half)
    dt_f64 = time.perf_counter() - t0
    return {"value": sample * n / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "first %d of the %d points, oracle.inside_exact (exact orientation "
                      "predicate, early exit per point), single thread, %.2f s" % (sample, len(w.points), dt),
            "cpu_model": cpu_model(),
            "all_cores": {"value": sample * n / dt_all / 1e9, "cores": threads,
                          "sample": "the same points in %d contiguous pieces, one per thread, %.2f s"
                                    % (threads, dt_all)},
            "plain_fp64_alg5": {"value": len(half) * n / dt_f64 / 1e9, "cores": 1,
                                "sample": "first %d points, oracle.voronoi_fp64 (Alg. 5 in fp64 with "
                                          "its own ambiguity flag), single thread, %.2f s" % (len(half), dt_f64)}}


def run_reference(args):
    """--impl reference: the CPU oracle timed as the reference arm."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2007_15385_gb300 import workloads as wl
    w = wl.vehicle_footprint(m=NUM_POINTS)
    import oracle
    n = int(w.edges()[0])
    # size each step's sample so that warm-up + timed steps end within ~3 minutes
    probe = 1 << 16
    t0 = time.perf_counter()
    oracle.inside_exact(w.vertices, np.ascontiguousarray(w.points[:probe]))
    per_point = (time.perf_counter() - t0) / probe
    budget = 150.0 / max(1, args.steps + args.warmup)
    sample = int(min(1 << 24, max(1 << 14, budget / per_point)))
    sample = 1 << int(np.floor(np.log2(sample)))
    rng = np.random.default_rng(7)
    starts = rng.integers(0, NUM_POINTS - sample, size=args.steps + args.warmup)
    times = []
    for i, s in enumerate(starts):
        pts = np.ascontiguousarray(w.points[s:s + sample])
        t0 = time.perf_counter()
        oracle.inside_exact(w.vertices, pts)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = sample * n * len(times) / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "num_points": NUM_POINTS, "edges": n,
                   "sample_points_per_step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d consecutive points per step at seeded offsets, "
                                   "oracle.inside_exact, single thread" % sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def dist_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) as torchrun sets them; (1, 0, 0) alone."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x of all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    tt = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Weak scaling: every rank decides its own shard of units; the job's
    rate is all ranks' units over the slowest rank's time, in G units/s."""
    return units_per_rank * world / (ms * 1e-3) / 1e9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1,
                    help="GPUs of the job (one rank each under torch.distributed.run; weak scaling)")
    ap.add_argument("--steps", type=int, default=200, help="timed steps (one pip_test call each)")
    ap.add_argument("--warmup", type=int, default=20, help="untimed warm-up steps (at least 3)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"],
                    help="reference: the CPU oracle timed on bounded samples of the same workload")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing on the host")
    ap.add_argument("--calls-only", action="store_true",
                    help="with --workload: prepare, then only W + K calls of the workload's main call "
                         "(no tuning, graphs, comparators or oracle; a small target for profilers)")
    ap.add_argument("--disc", action="store_true",
                    help="with --calls-only: the workload's call with the disc filter (PIP_DISC)")
    ap.add_argument("--headline-only", action="store_true",
                    help="time only the headline step (no per-workload objects)")
    ap.add_argument("--no-comparators", action="store_true",
                    help="skip the sign-of-offset, ray-crossing and plain fp64 kernels")
    ap.add_argument("--points", type=int, default=NUM_POINTS,
                    help="points of the workload (default the full 2^26; smaller only for profiling)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "gis_batch", "gis_all_pairs", "integer_hulls",
                             "footprint_trajectory", "unit_circle_octagon", "paper_sweep", "gis_raster",
                             "inner_generator"],
                    help="which workload to time (the default is the headline)")
    ap.add_argument("--polygons", type=int, default=0,
                    help="number of polygons of the batch workloads (0: the workload's own; "
                         "smaller cases are for profiling)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="tile shape of the pipelined kernel (default: autotuned)")
    ap.add_argument("--min-warmup-s", type=float, default=1.0,
                    help="warm up for at least this long so that clocks settle")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "paper_sweep":
        return run_sweep(args)
    if args.workload == "gis_raster":
        return run_raster(args)
    if args.workload == "inner_generator":
        return run_inner_generator(args)
    if args.workload != WORKLOAD:
        return run_other(args)

    import torch
    import torch.distributed as dist

    from paper_2007_15385_gb300 import binding as B
    from paper_2007_15385_gb300 import workloads as wl

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # each rank decides its own shard of points against the same footprint
    w = wl.vehicle_footprint(m=args.points, shard=rank)
    M = w.num_points
    n = int(w.edges()[0])
    v = torch.from_numpy(w.vertices).to(dev)
    vo = torch.from_numpy(w.vertex_offsets).to(dev)
    p = torch.from_numpy(w.points).to(dev)
    mask = torch.empty((M + 31) // 32, dtype=torch.int32, device=dev)
    t = B.pip_prepare(v, vo, max_points=M)
    st, _ = B.pip_get_status(t)
    assert st == B.PIP_OK

    def barrier():
        if world > 1:
            dist.barrier()

    stream = torch.cuda.current_stream()
    # tile shape of the pipelined kernel, tuned on this workload (not timed)
    if args.variant >= 0:
        variant = args.variant
        B.pip_set_stream_variant(t, variant)
    else:
        variant, _ = B.pip_autotune_stream(t, p, mask, reps=5)
    clocks = ClockSampler(local)
    clocks.start()
    # warm-up: W steps, and at least 1 s of them so that clocks settle
    t_w = time.perf_counter()
    i = 0
    while i < args.warmup or time.perf_counter() - t_w < args.min_warmup_s:
        B.pip_test(t, p, mask=mask)
        i += 1
        if i % 100 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        B.pip_test(t, p, mask=mask)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    # the same K steps again with per-call events around the kernel (kept out
    # of the step time above: the events themselves take time on the stream)
    B.pip_timing(t, True)
    for _ in range(args.steps):
        B.pip_test(t, p, mask=mask)
    calls, bulk_ms, refine_ms = B.pip_timing_read(t)
    B.pip_timing(t, False)
    clk = clocks.stop()
    _, refine_count = B.pip_get_status(t)
    ms_step = ms_total / args.steps
    # the pipelined path (16-byte aligned points) is one kernel per step
    calls_launches = 1 if p.data_ptr() % 16 == 0 else 2
    tests_per_step = M * n
    value = whole_job_rate(tests_per_step, world, ms_step)

    # roofline of the dominant (bulk streaming) kernel
    bytes_per_launch = M * 8 + ((M + 31) // 32) * 4
    bulk_avg_ms = bulk_ms / max(1, calls)
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / (bulk_avg_ms * 1e-3) / 1e9
    traffic = (NCU_TRAFFIC["bytes_by_variant"].get(variant) if NCU_TRAFFIC["sources_sha"] == sources_sha()
               else None)

    # end to end through the public API with host buffers
    p_host = torch.from_numpy(w.points).pin_memory()
    mask_host = torch.empty_like(mask, device="cpu").pin_memory()
    for _ in range(3):
        B.pip_test_host(t, p_host, p, mask, mask_host)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 50))
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        B.pip_test_host(t, p_host, p, mask, mask_host)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev) / e2e_steps
    e2e_value = whole_job_rate(tests_per_step, world, e2e_ms)
    h2d_bytes, d2h_bytes = int(p_host.numel() * 4), int(mask_host.numel() * 4)
    # the host link alone: the same bytes as one plain host-to-device copy
    # (pinned memory, copy engine), the floor of the end-to-end step
    for _ in range(2):
        p.copy_(p_host, non_blocking=True)
    torch.cuda.synchronize()
    l0 = torch.cuda.Event(enable_timing=True)
    l1 = torch.cuda.Event(enable_timing=True)
    l0.record(stream)
    for _ in range(5):
        p.copy_(p_host, non_blocking=True)
    l1.record(stream)
    torch.cuda.synchronize()
    link_ms = l0.elapsed_time(l1) / 5
    link_gbs = h2d_bytes / (link_ms * 1e-3) / 1e9

    # same-chip comparators on the same workload (Alg. 2, Alg. 1, plain fp64 Alg. 5)
    comparators = {}
    if not args.no_comparators:
        for name, fn, reps in (("sign_of_offset_f32", B.pip_test_sign_of_offset, 20),
                               ("ray_crossing_f32", B.pip_test_ray_crossing, 20),
                               ("voronoi_plain_fp64", B.pip_test_voronoi_fp64, 3)):
            fn(t, p, mask=mask)
            torch.cuda.synchronize()
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(reps):
                fn(t, p, mask=mask)
            c1.record(stream)
            torch.cuda.synchronize()
            cms = c0.elapsed_time(c1) / reps
            comparators[name] = {"ms": cms, "Gtests_per_s": tests_per_step / (cms * 1e-3) / 1e9}

    # the sequential test's early break (PIP_EARLY_EXIT, warp-uniform): same
    # results, less work, reported as an effective rate apart from the value
    ems = time_steps(lambda: B.pip_test(t, p, mode=B.PIP_MASK | B.PIP_EARLY_EXIT, mask=mask), 20, 3, stream)
    early_exit = {"ms_per_step": ems, "effective_Gtests_per_s": tests_per_step / (ems * 1e-3) / 1e9,
                  "note": "PIP_EARLY_EXIT: a warp stops once all its points are decided outside"}

    # the disc filter (PIP_DISC): a point inside the inner disc about o or
    # outside the outer one is decided without its edges; same results, less
    # work, reported as an effective rate apart from the value, with its own
    # kernel time against the same HBM peak (the same bytes move)
    disc_fn = lambda: B.pip_test(t, p, mode=B.PIP_MASK | B.PIP_DISC, mask=mask)
    dms = time_steps(disc_fn, max(20, args.steps), 3, stream)
    B.pip_timing(t, True)
    for _ in range(max(20, args.steps)):
        disc_fn()
    dcalls, dbulk_ms, _ = B.pip_timing_read(t)
    B.pip_timing(t, False)
    dk_ms = dbulk_ms / max(1, dcalls)
    full_frac = disc_full_fraction(B, t, w)
    disc = {"ms_per_step": dms, "effective_Gtests_per_s": tests_per_step / (dms * 1e-3) / 1e9,
            "kernel_ms": dk_ms,
            "roofline": {"bound": "hbm", "achieved": bytes_per_launch / (dk_ms * 1e-3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": bytes_per_launch / (dk_ms * 1e-3) / 1e9 / peak,
                         "peak_kind": peak_kind + " hbm_gbs"},
            "full_test_fraction": full_frac,
            "note": "PIP_DISC: points inside the inner or outside the outer disc about o skip their edges; "
                    "full_test_fraction = the points between the discs (host count, float32 d2)"}

    # the signed margin (pip_margin) on the same points, apart from the step:
    # 8 B read + 4 B written per point, against the same HBM peak
    marg = torch.empty(M, dtype=torch.float32, device=dev)
    mms = time_steps(lambda: B.pip_margin(t, p, out=marg), 20, 3, stream)
    margin = {"ms": mms, "Gtests_per_s": tests_per_step / (mms * 1e-3) / 1e9,
              "achieved": M * 12 / (mms * 1e-3) / 1e9, "unit": "GB/s", "peak": peak,
              "frac": M * 12 / (mms * 1e-3) / 1e9 / peak, "bytes_per_point": 12}
    del marg

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_run(w, 1 << 25)

    # every other configuration on the same GPU, apart from the headline step:
    # one object per workload (N = 1 only; the scaling runs time the headline)
    workloads, fma_peak, wclk = None, None, None
    if world == 1 and not args.headline_only:
        del p_host, mask_host
        torch.cuda.empty_cache()
        fma_peak = measure_fma_peak(B, dev, stream)
        wclocks = ClockSampler(local)
        wclocks.start()
        workloads = {}
        for name in WORKLOADS:
            workloads[name] = bench_workload(name, B, wl, dev, stream, max(args.steps, 20), args.warmup, fma_peak,
                                             2070.0, with_cpu=not args.no_cpu_baseline)
            torch.cuda.empty_cache()
        wclk = wclocks.stop()
        for r in workloads.values():
            renominal(r, wclk.get("sm_mhz"))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "num_points": M, "edges": n,
                       "polygon": "12 vertices on a 2.4 m x 1.0 m ellipse",
                       "points": "60% uniform in a 40 m square, 40% in 200 Gaussian clusters (sigma 0.3 m)",
                       "output": "packed uint32 bitmask, bit-exact (float32 filter + exact refine)",
                       "l2": "no flush: the 512 MiB of points exceed the 129 MB L2 every step",
                       "refined_points_per_step": refine_count,
                       "stream_variant": variant},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
                    "call": "pip_test_host (C ABI: pieces copied on the tables' copy stream, "
                            "tested and read back on the caller's stream)",
                    "host_link": {"h2d_gbs": link_gbs, "copy_ms": link_ms,
                                  "note": "one plain %d-byte pinned host-to-device copy, the same run" % h2d_bytes}},
            "gpu_launches": calls_launches * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "peak_kind": peak_kind + " hbm_gbs",
                         "kernel": "stream_tma_kernel (float32 test + inline exact refine)",
                         "bytes_per_launch": bytes_per_launch, "kernel_ms": bulk_avg_ms,
                         "refine_kernel_ms": refine_ms / max(1, calls)},
            "comparators": comparators,
            "early_exit": early_exit,
            "disc_filter": disc,
            "margin": margin,
            "cpu_baseline": cpu,
        }
        if workloads is not None:
            line["fp32_fma_peak"] = fma_peak
            line["workloads"] = workloads
            line["workloads_clocks"] = wclk
        print(json.dumps(line))
    t.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def fp32_fma_peak_tflops(sm_mhz: float) -> tuple[float, int]:
    """Nominal: #SM x 128 FP32 lanes x 2 flop x clock (clock sampled during the run)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12, sms


def measure_fma_peak(B, dev, stream, reps: int = 5) -> dict:
    """Measured FP32 FMA throughput: pip_fma_peak (8 independent FMA chains per
    thread, 8 blocks of 256 threads per SM) timed with CUDA events."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(8 * sms * 256, dtype=torch.float32, device=dev)
    B.pip_fma_peak(sink)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fmas = 0
    for _ in range(reps):
        fmas += B.pip_fma_peak(sink)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"tflops": 2.0 * fmas / (ms * 1e-3) / 1e12, "kernel": "fma_peak_kernel (pip_fma_peak)",
            "ms_per_launch": ms / reps, "fmas_per_launch": fmas // reps}


def fma_roofline(flops: float, kernel_ms: float, measured: dict | None, sm_mhz: float) -> dict:
    """FP32 roofline of a kernel doing `flops` in `kernel_ms`, against the peak
    measured in this run and against the nominal one at the sampled clock."""
    nominal, sms = fp32_fma_peak_tflops(sm_mhz or 2070.0)
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    out = {"bound": "alu", "achieved": achieved, "unit": "TFLOP/s",
           "nominal_peak": nominal, "frac_of_nominal": achieved / nominal,
           "nominal_kind": "%d SMs x 128 FP32 FMA lanes x 2 flop x sampled SM clock" % sms}
    if measured:
        out.update({"peak": measured["tflops"], "frac": achieved / measured["tflops"],
                    "peak_kind": "measured in this run: pip_fma_peak, a pure FFMA kernel"})
    else:
        out.update({"peak": nominal, "frac": achieved / nominal, "peak_kind": "nominal"})
    return out


def renominal(d: dict, sm_mhz: float) -> None:
    """Re-states every FP32 roofline in `d` against the nominal peak at the SM
    clock sampled over the run (known only once the sampler stops)."""
    if not sm_mhz:
        return
    for k, r in d.items():
        if k.startswith("fma_roofline") and isinstance(r, dict):
            nominal, _ = fp32_fma_peak_tflops(sm_mhz)
            r["nominal_peak"] = nominal
            r["frac_of_nominal"] = r["achieved"] / nominal


def time_steps(fn, steps: int, warmup: int, stream) -> float:
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_sweep(args):
    """The paper's experiment (Sec. 6.2) on the GPU: one convex polygon of n =
    3..15 edges on the unit circle, random points around it, Voronoi against
    sign of offset, ray crossing and the plain fp64 Voronoi form, in batches of
    10^6 points (the paper's batch; L2-resident, launch-bound) and of 2^25
    points (HBM-bound)."""
    import torch

    from paper_2007_15385_gb300 import binding as B
    from paper_2007_15385_gb300 import workloads as wl

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    reps = max(3, args.steps)
    sizes = {"batch_1e6": 10 ** 6, "stream_2e25": 1 << 25}
    rows = {k: [] for k in sizes}
    for n in range(3, 16):
        big = wl.unit_circle_octagon(seed=100 + n, m=sizes["stream_2e25"], n=n)
        v = torch.from_numpy(big.vertices).to(dev)
        vo = torch.from_numpy(big.vertex_offsets).to(dev)
        t = B.pip_prepare(v, vo, max_points=big.num_points)
        p_all = torch.from_numpy(big.points).to(dev)
        for key, m in sizes.items():
            p = p_all[:m]
            mask = torch.empty((m + 31) // 32, dtype=torch.int32, device=dev)
            row = {"n": n}
            for name, fn in (("voronoi", lambda: B.pip_test(t, p, mask=mask)),
                             ("sign_of_offset", lambda: B.pip_test_sign_of_offset(t, p, mask=mask)),
                             ("ray_crossing", lambda: B.pip_test_ray_crossing(t, p, mask=mask)),
                             ("voronoi_plain_fp64", lambda: B.pip_test_voronoi_fp64(t, p, mask=mask))):
                r = reps if name != "voronoi_plain_fp64" or key == "batch_1e6" else 3
                ms = time_steps(fn, r, 3, stream)
                row[name] = {"ms": ms, "Gtests_per_s": m * n / (ms * 1e-3) / 1e9}
            rows[key].append(row)
        t.close()
    clk = clocks.stop()
    vor = [r["voronoi"]["Gtests_per_s"] for r in rows["batch_1e6"]]
    value = float(np.exp(np.mean(np.log(vor))))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": reps,
            "warmup": 3, "ms_per_step": float(np.mean([r["voronoi"]["ms"] for r in rows["batch_1e6"]])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "paper_sweep", "edges": "3..15", "polygon": "n sorted random angles on the unit circle",
                       "points": "uniform in [-1.5, 1.5]^2", "value": "geometric mean over n of Voronoi Gtests/s, 10^6-point batches"},
            "clocks": clk, "gpu_launches": 13 * 2 * 4 * (reps + 3), "sweep": rows}
    print(json.dumps(line))
    return 0


def run_inner_generator(args):
    """The inner-generator study (Sec. 3: any interior point may be p0): the
    float32 filter's refine fraction and the call's time with the centroid
    (Eq. 3-4), the vertex mean and the Chebyshev centre (largest inscribed
    circle, by LP on the host) as p0, on the first 1,024 GIS polygons with
    their points and on the 1,024 integer hulls with their points as float32
    (so that the filter, not the exact integer path, decides them)."""
    import torch

    from paper_2007_15385_gb300 import binding as B
    from paper_2007_15385_gb300 import workloads as wl

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    cases = {"gis_batch_1024": wl.gis_batch(num_polygons=args.polygons or 1024),
             "integer_hulls_f32_points": wl.integer_hulls(num_polygons=args.polygons or 1024)}
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    study = {}
    for cname, w in cases.items():
        v = torch.from_numpy(w.vertices).to(dev)
        vo = torch.from_numpy(w.vertex_offsets).to(dev)
        p = torch.from_numpy(w.points.astype(np.float32)).to(dev)
        po = torch.from_numpy(w.point_offsets).to(dev)
        mask = torch.empty((w.num_points + 31) // 32, dtype=torch.int32, device=dev)
        t0 = time.perf_counter()
        cheb = torch.from_numpy(wl.chebyshev_centres(w.vertices, w.vertex_offsets)).to(dev)
        lp_s = time.perf_counter() - t0
        rows = {}
        for kind, code, given in (("centroid", B.PIP_P0_CENTROID, None),
                                  ("vertex_mean", B.PIP_P0_VERTEX_MEAN, None),
                                  ("chebyshev_centre", B.PIP_P0_GIVEN, cheb)):
            t = B.pip_prepare_p0(v, vo, w.num_points, code, given)
            st, _ = B.pip_get_status(t)
            call = lambda: B.pip_test(t, p, po, mask=mask)
            ms = time_steps(call, args.steps, args.warmup, stream)
            B.pip_timing(t, True)
            for _ in range(args.steps):
                call()
            calls, bulk_ms, refine_ms = B.pip_timing_read(t)
            B.pip_timing(t, False)
            _, refined = B.pip_get_status(t)
            rows[kind] = {"status": st, "ms_per_call": ms, "bulk_ms": bulk_ms / max(1, calls),
                          "refine_ms": refine_ms / max(1, calls), "refined_points": refined,
                          "refine_fraction": refined / w.num_points,
                          "Gtests_per_s": w.tests() / (ms * 1e-3) / 1e9}
            t.close()
        study[cname] = {"num_polygons": w.num_polygons, "num_points": w.num_points, "lp_seconds": lp_s,
                        "p0": rows}
    clk = clocks.stop()
    g = study["gis_batch_1024"]["p0"]["centroid"]
    line = {"metric": METRIC, "value": g["Gtests_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": g["ms_per_call"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "inner_generator", "value": "GIS batch (1,024 polygons), centroid p0"},
            "clocks": clk, "gpu_launches": 4 * args.steps * 6, "study": study}
    print(json.dumps(line))
    return 0


def run_raster(args):
    """Pixel coverage (pip_rasterize) of the 4,096 GIS polygons on a 3840 x 2160
    frame spanning their [0, 10^4]^2 domain: first-hit id and mask per pixel."""
    import torch

    from paper_2007_15385_gb300 import binding as B
    from paper_2007_15385_gb300 import workloads as wl

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    w = wl.gis_batch(num_polygons=args.polygons) if args.polygons > 0 else wl.gis_batch()
    W, H = 3840, 2160
    dx, dy = float(np.float32(1e4 / W)), float(np.float32(1e4 / H))
    t = B.pip_prepare(torch.from_numpy(w.vertices).to(dev), torch.from_numpy(w.vertex_offsets).to(dev),
                      max_points=W * H)
    ids = torch.empty((H, W), dtype=torch.int32, device=dev)
    mask = torch.empty((H, (W + 31) // 32), dtype=torch.int32, device=dev)
    ws = torch.empty(B.pip_raster_workspace_bytes(t.num_polygons, W, H) + 16, dtype=torch.uint8, device=dev)
    call = lambda: B.pip_rasterize(t, W, H, 0.0, 0.0, dx, dy, first_hit=ids, mask=mask, workspace=ws)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    ms = time_steps(call, args.steps, args.warmup, stream)
    B.pip_timing(t, True)
    for _ in range(args.steps):
        call()
    calls, bulk_ms, refine_ms = B.pip_timing_read(t)
    B.pip_timing(t, False)
    _, refined = B.pip_get_status(t)
    clk = clocks.stop()
    covered = int((ids >= 0).sum().item())
    t.close()
    px = W * H
    line = {"metric": "pixels/s (pixel-centre coverage, first-hit id + mask)", "value": px / (ms * 1e-3) / 1e9,
            "unit": "Gpixels/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "gis_raster", "width": W, "height": H, "num_polygons": w.num_polygons,
                       "frame": "[0, 1e4]^2", "covered_pixels": covered},
            "clocks": clk, "gpu_launches": 4 * args.steps,
            "tile_and_finalize_ms": bulk_ms / max(1, calls), "refine_ms": refine_ms / max(1, calls),
            "refined_pixels_per_step": refined,
            "output_bytes_per_step": px * 4 + H * ((W + 31) // 32) * 4}
    print(json.dumps(line))
    return 0


def workload_cpu_baseline(name: str, w) -> dict:
    """The oracle on a bounded sample of one workload (about a second or two on
    one host thread), as Gtests/s in the full-work convention."""
    import oracle
    n = w.edges()
    if name in ("gis_batch", "integer_hulls"):
        K = 16 if name == "gis_batch" else 512
        vo, po = w.vertex_offsets, w.point_offsets
        v = w.vertices[:vo[K]]
        q = w.points[:po[K]]
        tests = int((np.diff(po[:K + 1]) * n[:K]).sum())
        t0 = time.perf_counter()
        oracle.inside_exact_ragged(v, vo[:K + 1], q, po[:K + 1])
        dt = time.perf_counter() - t0
        sample = "the first %d polygons with their %d points, oracle.inside_exact_ragged, one thread, %.2f s" % (
            K, len(q), dt)
    elif name == "gis_all_pairs":
        m = 4096
        tests = m * int(n.sum())
        t0 = time.perf_counter()
        oracle.first_hit_exact(w.vertices, w.vertex_offsets, w.points[:m])
        dt = time.perf_counter() - t0
        sample = "the first %d points against all %d polygons, oracle.first_hit_exact (early exit), one thread, " \
                 "%.2f s" % (m, w.num_polygons, dt)
    elif name == "footprint_trajectory":
        k = 4
        poses = w.extra["poses"][:k]
        tests = k * w.num_points * int(n[0])
        t0 = time.perf_counter()
        oracle.penalty(w.vertices.astype(np.float64), poses.astype(np.float64), w.points.astype(np.float64),
                       float(np.float32(w.extra["tau"])))
        dt = time.perf_counter() - t0
        sample = "the first %d poses x all %d points, oracle.penalty (loss and every gradient, fp64), one " \
                 "thread, %.2f s" % (k, w.num_points, dt)
    else:
        tests = w.num_points * int(n.sum())
        t0 = time.perf_counter()
        oracle.inside_exact(w.vertices, w.points)
        dt = time.perf_counter() - t0
        sample = "all %d points, oracle.inside_exact, one thread, %.2f s" % (w.num_points, dt)
    return {"value": tests / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}


WORKLOADS = ("unit_circle_octagon", "gis_batch", "gis_all_pairs", "integer_hulls", "footprint_trajectory")


def disc_full_fraction(B, t, w) -> float:
    """Share of the points between the disc filter's two discs (they take the
    full test), counted on the host from the exported thresholds with the
    kernels' float32 d2 (output formatting only)."""
    ex = B.pip_export_tables(t)
    offs = w.point_offsets if w.point_offsets is not None else np.array([0, len(w.points)])
    between = 0
    for j in range(len(offs) - 1):
        q = w.points[offs[j]:offs[j + 1]].astype(np.float32) - ex["origin"][j]
        d2 = q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1]
        between += int(np.count_nonzero((d2 >= ex["disc"][j][0]) & (d2 <= ex["disc"][j][1])))
    return between / max(1, len(w.points))


def bench_workload(name: str, B, wl, dev, stream, steps: int, warmup: int, fma_peak: dict | None,
                   sm_mhz: float, polygons: int = 0, with_cpu: bool = True) -> dict:
    """Every measurement of one workload other than the headline: the call's
    time, the kernels' times, the rooflines, the refine fraction, the call
    replayed as a CUDA graph, the comparators where they apply and the oracle
    on a bounded sample.  Inputs are resident in HBM before timing starts."""
    import torch
    gen = getattr(wl, name)
    w = gen(num_polygons=polygons) if polygons > 0 and name in ("gis_batch", "gis_all_pairs",
                                                                   "integer_hulls") else gen()
    v = torch.from_numpy(w.vertices).to(dev)
    vo = torch.from_numpy(w.vertex_offsets).to(dev)
    p = torch.from_numpy(w.points).to(dev)
    po = torch.from_numpy(w.point_offsets).to(dev) if w.point_offsets is not None else None
    M = w.num_points
    tests = w.tests()
    out = {"config": {"num_points": M, "num_polygons": w.num_polygons, "tests_per_step": tests}}
    if name == "footprint_trajectory":
        poses = torch.from_numpy(w.extra["poses"]).to(dev)
        tau = w.extra["tau"]
        ws = torch.empty(B.pip_penalty_workspace_bytes(len(w.vertices), len(poses), M),
                         dtype=torch.uint8, device=dev)
        n = len(w.vertices)
        tests = len(poses) * M * n
        fwd = time_steps(lambda: B.pip_penalty_forward(v, poses, p, tau, workspace=ws), steps, warmup, stream)
        bwd = time_steps(lambda: B.pip_penalty_backward(v, poses, p, tau, workspace=ws), steps, warmup, stream)
        out["config"].update({"num_poses": len(poses), "tau": tau, "tests_per_step": tests,
                              "pairs": len(poses) * M})
        # the cull (PIP_PENALTY_CULL): pairs provably beyond 120 tau of every
        # edge line left out; same loss and gradients up to the order of the
        # float32 partial sums, reported apart as effective rates
        cfwd = time_steps(lambda: B.pip_penalty_forward(v, poses, p, tau, workspace=ws, cull=True), steps, warmup,
                          stream)
        cbwd = time_steps(lambda: B.pip_penalty_backward(v, poses, p, tau, workspace=ws, cull=True), steps, warmup,
                          stream)
        out["culled"] = {"forward_ms": cfwd, "backward_ms": cbwd,
                         "effective_forward_Gtests_per_s": tests / (cfwd * 1e-3) / 1e9,
                         "effective_backward_Gtests_per_s": tests / (cbwd * 1e-3) / 1e9,
                         "note": "PIP_PENALTY_CULL: pairs whose float32 term and gradient are exactly 0 left out"}
        out.update({"ms_per_step": fwd, "Gtests_per_s": tests / (fwd * 1e-3) / 1e9,
                    "forward_ms": fwd, "backward_ms": bwd,
                    "forward_Gtests_per_s": tests / (fwd * 1e-3) / 1e9,
                    "backward_Gtests_per_s": tests / (bwd * 1e-3) / 1e9,
                    "gpu_launches_per_step": {"forward": 6, "backward": 7},
                    # every edge term is two FMAs (4 flops)
                    "fma_roofline": fma_roofline(4.0 * tests, fwd, fma_peak, sm_mhz),
                    "fma_roofline_backward": fma_roofline(4.0 * tests, bwd, fma_peak, sm_mhz)})
    else:
        t = B.pip_prepare(v, vo, max_points=M)
        mode = B.PIP_MASK | (B.PIP_FIRST_HIT if name == "gis_all_pairs" else 0)
        mask = torch.empty((M + 31) // 32, dtype=torch.int32, device=dev)
        hit = torch.empty(M, dtype=torch.int32, device=dev) if mode & B.PIP_FIRST_HIT else None
        call = lambda: B.pip_test(t, p, po, mode=mode, mask=mask, first_hit=hit)
        if po is not None and p.data_ptr() % 16 == 0:
            # tile shape of the pipelined batch kernel, tuned on this batch (not timed)
            out["batch_variant"], _ = B.pip_autotune_batch(t, p, po, mask, reps=3)
        ms = time_steps(call, steps, warmup, stream)
        # per-call kernel events in a separate pass, out of the step time
        B.pip_timing(t, True)
        for _ in range(steps):
            call()
        calls, bulk_ms, refine_ms = B.pip_timing_read(t)
        B.pip_timing(t, False)
        _, refined = B.pip_get_status(t)
        bulk = bulk_ms / max(1, calls)
        out.update({"ms_per_step": ms, "Gtests_per_s": tests / (ms * 1e-3) / 1e9,
                    "bulk_kernel_ms": bulk, "refine_kernel_ms": refine_ms / max(1, calls),
                    "refined_points_per_step": refined, "refine_fraction": refined / max(1, M)})
        # the whole call (setup, bulk, refine) captured once as a CUDA graph, replayed per step
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            call()
        stream.wait_stream(gs)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            call()
        out["graph_ms_per_step"] = time_steps(graph.replay, steps, 3, stream)
        del graph
        if name in ("gis_batch", "unit_circle_octagon"):
            # the early break (PIP_EARLY_EXIT): same results, less work
            ecall = lambda: B.pip_test(t, p, po, mode=mode | B.PIP_EARLY_EXIT, mask=mask, first_hit=hit)
            ems = time_steps(ecall, steps, 3, stream)
            out["early_exit"] = {"ms_per_step": ems, "effective_Gtests_per_s": tests / (ems * 1e-3) / 1e9,
                                 "note": "PIP_EARLY_EXIT: a warp stops once all its points are decided outside"}
        if name in ("gis_batch", "unit_circle_octagon"):
            # the disc filter (PIP_DISC): same results, less work, reported
            # apart as an effective rate with its kernel's HBM roofline
            dcall = lambda: B.pip_test(t, p, po, mode=mode | B.PIP_DISC, mask=mask, first_hit=hit)
            dms = time_steps(dcall, steps, 3, stream)
            B.pip_timing(t, True)
            for _ in range(steps):
                dcall()
            dcalls, dbulk_ms, drefine_ms = B.pip_timing_read(t)
            B.pip_timing(t, False)
            dk = dbulk_ms / max(1, dcalls)
            peak, kind = measured_peaks()
            nbytes = M * 8 + ((M + 31) // 32) * 4
            out["disc_filter"] = {"ms_per_step": dms, "effective_Gtests_per_s": tests / (dms * 1e-3) / 1e9,
                                  "bulk_kernel_ms": dk, "refine_kernel_ms": drefine_ms / max(1, dcalls),
                                  "roofline": {"bound": "hbm", "achieved": nbytes / (dk * 1e-3) / 1e9,
                                               "peak": peak, "unit": "GB/s",
                                               "frac": nbytes / (dk * 1e-3) / 1e9 / peak,
                                               "peak_kind": kind + " hbm_gbs",
                                               "call_frac": nbytes / (dms * 1e-3) / 1e9 / peak},
                                  "full_test_fraction": disc_full_fraction(B, t, w),
                                  "note": "PIP_DISC: points inside the inner or outside the outer disc about o "
                                          "skip their edges (full_test_fraction: the points between the discs)"}
        if name == "gis_all_pairs":
            # bounding-box cull and early stop (PIP_CULL): same results, less work;
            # reported apart as an effective rate, not as the full-work value
            cull = lambda: B.pip_test(t, p, po, mode=mode | B.PIP_CULL, mask=mask, first_hit=hit)
            cms = time_steps(cull, steps, 3, stream)
            out["culled"] = {"ms_per_step": cms, "effective_Gtests_per_s": tests / (cms * 1e-3) / 1e9,
                             "note": "PIP_CULL: polygons skipped per warp by bounding box, early stop"}
        # our kernels per call: batch = the persistent kernel and the refine
        # (integer polygons with integer points: the persistent kernel alone);
        # all pairs = bulk, finalize, refine; one polygon = the pipelined
        # kernel (refine inline), or bulk + refine for unaligned points
        if po is not None:
            out["gpu_launches_per_step"] = 1 if w.points.dtype == np.int32 and w.vertices.dtype == np.int32 else 2
        elif w.num_polygons > 1:
            out["gpu_launches_per_step"] = 3
        else:
            out["gpu_launches_per_step"] = 1 if p.data_ptr() % 16 == 0 else 2
        if name in ("gis_all_pairs", "gis_batch", "integer_hulls"):
            # every test is two FMAs (4 flops): s_k = t_k - x w_kx - y w_ky
            out["fma_roofline"] = fma_roofline(4.0 * tests, bulk, fma_peak, sm_mhz)
        if name in ("gis_batch", "integer_hulls", "unit_circle_octagon"):
            peak, kind = measured_peaks()
            nbytes = M * 8 + ((M + 31) // 32) * 4
            out["roofline"] = {"bound": "hbm", "achieved": nbytes / (bulk * 1e-3) / 1e9, "peak": peak,
                               "unit": "GB/s", "frac": nbytes / (bulk * 1e-3) / 1e9 / peak,
                               "peak_kind": kind + " hbm_gbs", "bytes_per_launch": nbytes,
                               "kernel_ms": bulk, "call_frac": nbytes / (ms * 1e-3) / 1e9 / peak}
        if name in ("gis_batch", "integer_hulls", "unit_circle_octagon"):
            # the paper's comparators on the same points and polygons (float32
            # listings; integer hulls as float32, exact below 2^24)
            tc, pc = t, p
            if w.vertices.dtype != np.float32:
                tc = B.pip_prepare(v.float(), vo, max_points=M)
                pc = p.float()
            comps = {}
            for cname, fn in (("sign_of_offset_f32", B.pip_test_sign_of_offset),
                              ("ray_crossing_f32", B.pip_test_ray_crossing),
                              ("voronoi_plain_fp64", B.pip_test_voronoi_fp64)):
                cmask = torch.empty_like(mask)
                cms = time_steps(lambda: fn(tc, pc, po, mask=cmask), 5 if "fp64" in cname else steps, 2, stream)
                comps[cname] = {"ms": cms, "Gtests_per_s": tests / (cms * 1e-3) / 1e9}
            out["comparators"] = comps
            if tc is not t:
                tc.close()
        t.close()
    if with_cpu:
        out["cpu_baseline"] = workload_cpu_baseline(name, w)
    return out


def run_calls_only(args, B, wl, dev, stream):
    """--calls-only: the workload's main call W + K times after its prepare,
    nothing else on the GPU; prints the mean time of the K timed calls."""
    gen = getattr(wl, args.workload)
    w = gen(num_polygons=args.polygons) if args.polygons > 0 and args.workload in (
        "gis_batch", "gis_all_pairs", "integer_hulls") else gen()
    import torch
    v = torch.from_numpy(w.vertices).to(dev)
    p = torch.from_numpy(w.points).to(dev)
    if args.workload == "footprint_trajectory":
        poses = torch.from_numpy(w.extra["poses"]).to(dev)
        ws = torch.empty(B.pip_penalty_workspace_bytes(len(w.vertices), len(poses), w.num_points),
                         dtype=torch.uint8, device=dev)
        call = lambda: B.pip_penalty_backward(v, poses, p, w.extra["tau"], workspace=ws)
    else:
        vo = torch.from_numpy(w.vertex_offsets).to(dev)
        po = torch.from_numpy(w.point_offsets).to(dev) if w.point_offsets is not None else None
        t = B.pip_prepare(v, vo, max_points=w.num_points)
        mode = B.PIP_MASK | (B.PIP_FIRST_HIT if args.workload == "gis_all_pairs" else 0)
        if args.disc:
            mode |= B.PIP_DISC
        mask = torch.empty((w.num_points + 31) // 32, dtype=torch.int32, device=dev)
        hit = torch.empty(w.num_points, dtype=torch.int32, device=dev) if mode & B.PIP_FIRST_HIT else None
        call = lambda: B.pip_test(t, p, po, mode=mode, mask=mask, first_hit=hit)
    ms = time_steps(call, args.steps, args.warmup, stream)
    print(json.dumps({"workload": args.workload, "calls_only": True, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_call": ms}))
    return 0


def run_other(args):
    """One JSON line for a workload other than the headline (same metric and unit)."""
    import torch

    from paper_2007_15385_gb300 import binding as B
    from paper_2007_15385_gb300 import workloads as wl

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    if args.calls_only:
        return run_calls_only(args, B, wl, dev, stream)
    fma_peak = measure_fma_peak(B, dev, stream)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    r = bench_workload(args.workload, B, wl, dev, stream, args.steps, args.warmup, fma_peak, 2070.0,
                       polygons=args.polygons, with_cpu=not args.no_cpu_baseline)
    clk = clocks.stop()
    renominal(r, clk.get("sm_mhz"))
    launches = r.pop("gpu_launches_per_step")
    if isinstance(launches, dict):
        launches = sum(launches.values())
    line = {"metric": METRIC, "value": r.pop("Gtests_per_s"), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict({"workload": args.workload}, **r.pop("config")),
            "clocks": clk, "gpu_launches": launches * args.steps, "fp32_fma_peak": fma_peak}
    line.update(r)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
