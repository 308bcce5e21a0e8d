"""Benchmark: MG8 label propagation on a GB300, one JSON line on stdout.

A step is one whole run of the hot path on one synthetic graph resident in HBM: degree
binning, synchronous sweeps to convergence (at most 20, pick-less every 8, tol 0.05) and
the modularity of the result -- one ``lpa_detect_ex`` call.  ``value`` is edges processed
per second (sum over steps of iterations * m, divided by the CUDA-event time of the
timed steps).  ``e2e`` is the same metric through ``lpa_detect_host`` with the graph in
page-locked host memory (host-to-device copy of the CSR and device-to-host copy of the
labels inside the timed region).  On the default workload the line also carries
``forms``: short runs of the batched form (the first 256 graphs of the batched family,
against one call per graph) and of the served form (the full arrival stream, 4000 timed
requests, against first-in-first-out one-at-a-time solves), each with its own warm-up,
timing and clock record (``--no-forms`` leaves them out).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload lfr26|rmat22|pp1000|lfr26s|lfr22|sbm256|sbm4096|serve]
                  [--mode mg|bm|exact] [--k K] [--unclamped] [--rescan] [--tune]
                  [--skip-cpu] [--no-forms]

Under torchrun (N > 1) every rank solves its own replica (the single-graph path does not
shard; scaling is weak) and rank 0 prints the line with the max time over ranks.
``--impl reference`` times the CPU oracle (the only reference this method has) on the
host cores, rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "MG8-LPA edges/sec/iteration"
UNIT = "edges/s"


def metric_name(args) -> str:
    """The headline metric for MG with k = 8; the same quantity for another mode, k or
    ablation variant is named after it."""
    if args.mode == "mg":
        name = f"MG{args.k}"
        if args.unclamped:
            name += "-literal"
        if args.rescan:
            name += "-rescan"
    else:
        name = {"bm": "BM", "exact": "exact"}[args.mode]
    return f"{name}-LPA edges/sec/iteration"

# DRAM traffic of one MG k = 8 sweep, from an ncu capture of a small case of the same
# family (dram__bytes_read.sum + dram__bytes_write.sum of the lane kernel, the whole sweep
# there since its rows have no hubs) scaled to the workload below by the ratio of their
# algorithmic bytes, with the hash of the sweep kernel source it was taken with.  If the
# source changes, traffic is reported as null until a new capture.
SWEEP_TRAFFIC = {"src_sha256": "21c06732b4c919e67beb9c7084dae2c298a2eedb244b24fd57d363b1cb381a7e",
                 "workload": "lfr26", "captured_on": "lfr26s",
                 "captured_bytes_per_launch": 10243403648,
                 "captured_algorithmic_bytes": 5479657280}

WORKLOADS = {
    "lfr26": "LFR-style heavy-tailed planted partition, n=2^26, degree power law 2.1 on "
             "[4, 65536], community sizes power law 1.5 on [20, 1e6], mu=0.2, integer "
             "weights 1..8, community-contiguous ids, seed 0",
    "lfr22": "LFR-style heavy-tailed planted partition as lfr26 but n=2^22 (profiling size)",
    "lfr26s": "LFR-style as lfr26 but degrees power law 2.1 on [2, 32] (mean about 5): a "
              "profiling size whose label array (256 MB) still exceeds L2",
    "rmat22": "R-MAT scale 22, edge factor 16, (a,b,c)=(0.57,0.19,0.19), symmetrised, "
              "duplicates merged with summed weights, seed 0",
    "pp1000": "planted partition, 1000 vertices in 10 communities, p_in=0.1, p_out=0.005, "
              "unit weights, seed 0",
    "sbm256": "batched form: graphs 0..255 of the uneven planted-partition family (n "
              "log-uniform in [100, 2e5], mean degree U[8, 64], communities log-uniform in "
              "[4, 500] capped at n/20, 80 % internal, unit weights), seed 0",
    "sbm4096": "batched form: graphs 0..4095 of the same family, seed 0",
}
BATCH_COUNT = {"sbm256": 256, "sbm4096": 4096}
BATCH_METRIC = "MG8-LPA batched graphs/s"
WORKLOADS["serve"] = ("served form: Poisson arrivals at 2000 requests/s (seeded exponential "
                      "gaps), each request a graph drawn from a pool held in page-locked host "
                      "memory: graphs 0..511 of the batched family plus, for 5 % of requests, "
                      "one of 8 R-MAT scale-20 graphs; host-to-device copy at arrival counted "
                      "in latency; 4000 timed requests per step after 700 per warm-up step")
SERVE_METRIC = "MG8-LPA served p99 latency"


def make_graph(name: str, threads: int | None = None) -> synth.Graph:
    if name == "lfr26":
        return synth.lfr(n=2**26, gamma_d=2.1, dmin=4, dmax=65536, gamma_c=1.5, cmin=20,
                         cmax=10**6, mu=0.2, wmax=8, seed=0, threads=threads)
    if name == "lfr26s":
        return synth.lfr(n=2**26, gamma_d=2.1, dmin=2, dmax=32, gamma_c=1.5, cmin=20,
                         cmax=10**6, mu=0.2, wmax=8, seed=0, threads=threads)
    if name == "lfr22":
        return synth.lfr(n=2**22, gamma_d=2.1, dmin=4, dmax=65536, gamma_c=1.5, cmin=20,
                         cmax=10**6, mu=0.2, wmax=8, seed=0, threads=threads)
    if name == "rmat22":
        return synth.rmat(scale=22, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=0,
                          threads=threads)
    if name == "pp1000":
        return synth.planted_partition(n=1000, ncomm=10, p_in=0.1, p_out=0.005, seed=0)
    raise ValueError(name)


def sweep_src_sha() -> str:
    h = hashlib.sha256()
    for f in ("lpa_sweep.cu", "lpa_sweep_impl.cuh", "lpa_fold.cuh", "lpa_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2411_19901_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def mark(self, which: str):
        """Host time at the start / end of the timed region."""
        setattr(self, which, time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(",") for r in self.file.read().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "start", None), getattr(self, "end", None)
        parsed = []
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(r[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + r[0].split(".")[1]) if "." in r[0] else 0.0
                parsed.append((ts, float(r[2]), float(r[3]), float(r[4]), r[6:10]))
            except (ValueError, IndexError):
                continue
        inside = [p for p in parsed if t0 is not None and t0 - 0.2 <= p[0] <= t1 + 0.2]
        for ts, a, b, c, flags in (inside or parsed):
            sm.append(a)
            smax.append(b)
            power.append(c)
            for name, val in zip(names, flags):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None,
            "samples": len(sm),
            "samples_in_timed_region": len(inside),
            "reasons": sorted(reasons),
        }


# ------------------------------------------------------------------ helpers


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def physical_gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        parts = [p for p in vis.split(",") if p.strip()]
        if local_rank < len(parts) and parts[local_rank].strip().isdigit():
            return int(parts[local_rank])
    return local_rank


# Approximate host bytes of each workload's CSR (offsets, indices, weights).
GRAPH_BYTES = {"lfr26": 13 << 30, "lfr26s": 6 << 30, "rmat22": 2 << 30}


def _bcast_from_rank0(obj):
    """rank 0's value of obj on every rank (torch.distributed must be initialised)."""
    import torch.distributed as dist

    box = [obj]
    dist.broadcast_object_list(box, src=0)
    return box[0]


def share_graph(name: str, world: int, rank: int, barrier,
                need_bytes: int | None = None, free_bytes: int | None = None,
                local_world: int | None = None, bcast=None) -> tuple[synth.Graph, float]:
    """Rank 0 generates; with several ranks the others map rank 0's arrays from disk.

    Rank 0 alone decides whether the graph is shared, and broadcasts the decision, so every
    rank takes the same path: it is shared only when every rank runs on rank 0's node
    (LOCAL_WORLD_SIZE == WORLD_SIZE, so all see rank 0's temporary directory) and that
    directory has room for two copies of the graph.  Otherwise every rank generates its
    own copy (same seed, same graph; the host cores split between ranks).  free_bytes and
    local_world override what rank 0 reads from the system (tests)."""
    t0 = time.perf_counter()
    if world == 1:
        g = make_graph(name)
        return g, time.perf_counter() - t0
    import shutil

    need = GRAPH_BYTES.get(name, 1 << 30) if need_bytes is None else need_bytes
    if local_world is None:
        local_world = int(os.environ.get("LOCAL_WORLD_SIZE", str(world)))
    if free_bytes is None:
        free_bytes = shutil.disk_usage(tempfile.gettempdir()).free
    shared = (bcast or _bcast_from_rank0)(bool(local_world == world and free_bytes > 2 * need))
    if not shared:
        g = make_graph(name, threads=max(1, (os.cpu_count() or 1) // world))
        return g, time.perf_counter() - t0
    d = os.path.join(tempfile.gettempdir(), f"lpa_bench_{name}")
    if rank == 0:
        g = make_graph(name)
        os.makedirs(d, exist_ok=True)
        np.save(os.path.join(d, "offsets.npy"), g.offsets)
        np.save(os.path.join(d, "indices.npy"), g.indices)
        if g.weights is not None:
            np.save(os.path.join(d, "weights.npy"), g.weights)
    barrier()
    if rank != 0:
        off = np.load(os.path.join(d, "offsets.npy"), mmap_mode="r")
        idx = np.load(os.path.join(d, "indices.npy"), mmap_mode="r")
        wp = os.path.join(d, "weights.npy")
        w = np.load(wp, mmap_mode="r") if os.path.exists(wp) else None
        g = synth.Graph(off, idx, w, name)
    return g, time.perf_counter() - t0


def aggregate_over_ranks(times_ms, counts, world: int, device):
    """Whole-job figures: the max of each time and the sum of each count over ranks."""
    if world == 1:
        return [float(t) for t in times_ms], [float(c) for c in counts]
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x) for x in times_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()], [float(x) for x in c.tolist()]


def sweep_bytes(n: int, m: int, weighted: bool) -> int:
    """Algorithmic bytes of one sweep: per CSR entry its index, weight and the gathered
    neighbour label (12 B, 8 B with unit weights); per vertex its offset, old label, new
    label and its place in the degree order (8 + 4 + 4 + 4 = 20 B)."""
    return (12 if weighted else 8) * m + 20 * n


def sweep_kernel_label(args, weighted: bool) -> str:
    """The kernels one timed sweep launches, for the roofline line."""
    wf = "weighted" if weighted else "unit weights"
    if args.mode == "exact":
        return f"one sweep: sweep_exact_kernel (per-vertex hashtable, {wf})"
    if args.mode == "bm":
        sk = "BMState"
    else:
        sk = f"MGLiteral<{args.k}>" if args.unclamped else f"MGSketch<{args.k}>"
        if args.rescan:
            sk += ", rescan"
    return (f"one sweep: sweep_hub_kernel and sweep_lane_kernel <{sk}, {wf}> "
            "(concurrent, fork/join)")


def oracle_sweeps(g: synth.Graph, mode: str, seconds: float, max_reps: int, k: int = 8,
                  unclamped: bool = False, rescan: bool = False):
    """Time full oracle sweeps (iteration 0 from identity labels) on all host cores."""
    import oracle

    om = {"mg": oracle.MG, "bm": oracle.BM, "exact": oracle.EXACT}[mode]
    threads = os.cpu_count() or 1
    offs = np.ascontiguousarray(g.offsets)
    idx = np.ascontiguousarray(g.indices)
    w = None if g.weights is None else np.ascontiguousarray(g.weights)
    c0 = np.arange(g.n, dtype=np.int32)
    times = []
    while len(times) < max_reps and (not times or sum(times) < seconds):  # at least one
        t = time.perf_counter()
        oracle.move(offs, idx, w, c0, mode=om, k=k, pick_less=True, threads=threads,
                    unclamped=unclamped, rescan=rescan)
        times.append(time.perf_counter() - t)
    return times, threads


# ------------------------------------------------------------------ arms


def oracle_batch_rate(gs, mode: str, seconds: float):
    """Full oracle runs, graph after graph, on all host cores for about ``seconds``."""
    import oracle

    om = {"mg": oracle.MG, "bm": oracle.BM, "exact": oracle.EXACT}[mode]
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    done = 0
    for g in gs:
        oracle.lpa(g.offsets, g.indices, g.weights, mode=om, k=8, tol=0.05, max_iter=20,
                   threads=threads)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt, threads


def oracle_serve_latencies(gpool, mode: str, seconds: float):
    """Requests drawn as in the served workload, each a full oracle run on all host cores,
    one at a time with no queueing; returns the per-request times (ms) and the threads."""
    import oracle

    rng = np.random.default_rng(12345)
    threads = os.cpu_count() or 1
    om = {"mg": oracle.MG, "bm": oracle.BM, "exact": oracle.EXACT}[mode]
    lat = []
    t0 = time.perf_counter()
    while not lat or time.perf_counter() - t0 < seconds:
        j = int(512 + rng.integers(0, 8)) if rng.random() < 0.05 else int(rng.integers(0, 512))
        g = gpool[j]
        t = time.perf_counter()
        oracle.lpa(g.offsets, g.indices, g.weights, mode=om, threads=threads)
        lat.append(1e3 * (time.perf_counter() - t))
    return lat, threads


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    if args.workload in BATCH_COUNT:
        gs = make_batch(BATCH_COUNT[args.workload])
        rates = []
        for step in range(args.warmup + args.steps):
            rate, done, dt, threads = oracle_batch_rate(gs, args.mode, 10.0)
            if step >= args.warmup:
                rates.append(rate)
        value = sum(rates) / len(rates)
        sample = f"full oracle runs of the batch's first graphs, about 10 s per step"
        print(json.dumps({
            "impl": "reference", "metric": BATCH_METRIC, "value": value, "unit": "graphs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * len(gs) / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}",
                       "graphs": len(gs), "mode": args.mode, "k": 8},
            "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }), flush=True)
        return
    if args.workload == "serve":
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
            gpool = pool.map(_gen_serve, range(520), chunksize=4)
        lat, threads = oracle_serve_latencies(gpool, args.mode, 10.0 * max(args.steps, 1) / 5 + 5.0)
        p99 = float(np.percentile(lat, 99))
        print(json.dumps({
            "impl": "reference", "metric": SERVE_METRIC, "value": p99, "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(sum(lat)), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serve: {WORKLOADS['serve']}", "mode": args.mode, "k": 8},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": p99,
            "cpu_baseline": {"value": p99, "unit": "ms", "cores": threads, "kind": "oracle",
                             "sample": f"{len(lat)} requests from the same pool, each a full "
                                       "oracle run on all host cores, served one at a time "
                                       "with no queueing (a lower bound on its latency)"},
            "e2e": {"value": p99, "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
        }), flush=True)
        return
    g = make_graph(args.workload)
    import oracle  # noqa: F401  (the reference arm is the CPU oracle)

    om_times, threads = [], 0
    for step in range(args.warmup + args.steps):
        ts, threads = oracle_sweeps(g, args.mode, 0.0, 1, k=args.k, unclamped=args.unclamped,
                                    rescan=args.rescan)
        if step >= args.warmup:
            om_times += ts
    value = len(om_times) * g.m / sum(om_times)
    sample = f"{len(om_times)} full oracle sweeps (iteration 0 from identity labels) of the graph"
    line = {
        "impl": "reference", "metric": metric_name(args), "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(om_times) / len(om_times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(args, g),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(args, g):
    return {
        "workload": f"{args.workload}: {WORKLOADS[args.workload]}",
        "n": g.n, "m": g.m, "mode": args.mode, "k": args.k, "tol": 0.05, "max_iter": 20,
        "mg_variant": {"unclamped": args.unclamped, "rescan": args.rescan},
        "pl_period": 8, "weights": "int-valued fp32" if g.weights is not None else "unit",
        "l2": "inputs larger than L2 (no flush)" if g.m * 8 > 129e6 else
              "inputs smaller than L2 (warm cache)",
        "parallelism": "replicas" if args.gpus > 1 else "single GPU",
    }


def run_ours(args):
    import torch

    import paper_2411_19901_gb300 as lpa
    from paper_2411_19901_gb300 import build

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")

        def barrier():
            dist.barrier()
    else:
        def barrier():
            pass
    dev = torch.device("cuda", local)
    build.build()
    g, gen_s = share_graph(args.workload, world, rank, barrier)
    n, m = g.n, g.m
    weighted = g.weights is not None

    # page-locked host copies (the e2e inputs) and device copies (the value inputs)
    pin = world == 1
    h_off = torch.from_numpy(np.ascontiguousarray(g.offsets))
    h_idx = torch.from_numpy(np.ascontiguousarray(g.indices))
    h_w = torch.from_numpy(np.ascontiguousarray(g.weights)) if weighted else None
    if pin:
        h_off, h_idx = h_off.pin_memory(), h_idx.pin_memory()
        h_w = h_w.pin_memory() if weighted else None
    d_off = h_off.to(dev)
    d_idx = h_idx.to(dev)
    d_w = h_w.to(dev) if weighted else None
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the launch choices: the defaults, or with --tune the tuner's pick for this graph
    # (timed before the timed region; results are identical under every choice)
    tuning, tune_table, tune_s = None, None, 0.0
    if args.tune:
        from paper_2411_19901_gb300 import tune as _tune

        t0 = time.perf_counter()
        tuning, tune_table = _tune.tune_graph(d_off, d_idx, d_w, mode=args.mode, k=args.k,
                                              reps=1, stream=stream)
        tune_s = time.perf_counter() - t0

    def options(tun, **kw):
        return lpa.make_options(validate=False, stream=stream, unclamped=args.unclamped,
                                rescan=args.rescan, tuning=tun, **kw)

    ws_bytes = max(lpa.lpa_workspace_size_ex(n, m, args.mode, args.k, options(t))
                   for t in (None, tuning))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    opt = options(tuning, timing=True, modularity=True, workspace=ws)

    def step():
        st = lpa.lpa_stats()
        lpa.lpa_detect_ex(d_off, d_idx, d_w, n, m, args.mode, args.k, 0.05, 20, labels, st, opt)
        return st.to_dict()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier()
    clocks = ClockSampler(physical_gpu_index(local))
    launches0 = lpa.lpa_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    time.sleep(0.5)  # let nvidia-smi start sampling
    torch.cuda.synchronize(dev)
    clocks.mark("start")
    ev0.record(stream)
    stats = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark("end")
    barrier()
    clk = clocks.stop()
    launches = lpa.lpa_launch_count() - launches0
    elapsed_ms = ev0.elapsed_time(ev1)
    edges = sum(s["iterations"] * m for s in stats)
    sweeps = sum(s["iterations"] for s in stats)
    sweep_ms = sum(s["sweep_ms"] for s in stats)

    # end to end through the host-memory entry point: one untimed call first (it grows
    # the library's device pool by the staging buffers), then e2e_steps timed calls, each
    # with its host-to-device copies and its labels back to host memory
    e2e_steps = max(1, min(args.steps, 3))
    h_lab = torch.empty(n, dtype=torch.int32, pin_memory=pin)
    e2e_stats = []

    def e2e_call():
        st = lpa.lpa_stats()
        lpa.lpa_detect_host(h_off.numpy(), h_idx.numpy(), h_w.numpy() if weighted else None,
                            n, m, args.mode, args.k, 0.05, 20, h_lab.numpy(), st,
                            options(tuning, modularity=True, workspace=ws))
        return st.to_dict()

    e2e_call()
    torch.cuda.synchronize(dev)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_host = time.perf_counter()
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_stats.append(e2e_call())
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = max(e0.elapsed_time(e1), 1e3 * (time.perf_counter() - t_host))
    barrier()
    e2e_edges = sum(s["iterations"] * m for s in e2e_stats)

    # with --tune, the same steps under the default launch choices, for comparison
    fixed = None
    if args.tune:
        fopt = options(None, timing=True, modularity=True, workspace=ws)
        lpa.lpa_detect_ex(d_off, d_idx, d_w, n, m, args.mode, args.k, 0.05, 20, labels,
                          lpa.lpa_stats(), fopt)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        f0.record(stream)
        fst = []
        for _ in range(args.steps):
            st = lpa.lpa_stats()
            lpa.lpa_detect_ex(d_off, d_idx, d_w, n, m, args.mode, args.k, 0.05, 20, labels, st,
                              fopt)
            fst.append(st.to_dict())
        f1.record(stream)
        torch.cuda.synchronize(dev)
        fms = f0.elapsed_time(f1)
        fixed = {"value": sum(s["iterations"] * m for s in fst) / (fms * 1e-3),
                 "ms_per_step": fms / args.steps,
                 "sweep_ms": sum(s["sweep_ms"] for s in fst) / max(sum(s["iterations"] for s in fst), 1)}

    # the standalone modularity entry point (Eq. 1) on the final labels, outside the timed
    # region: CUDA events around lpa_modularity_ex calls, after one untimed call
    mopt = lpa.make_options(validate=False, stream=stream)
    lpa.lpa_modularity_ex(d_off, d_idx, d_w, n, m, labels, mopt)
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(3):
        q_alone = lpa.lpa_modularity_ex(d_off, d_idx, d_w, n, m, labels, mopt)
    m1.record(stream)
    torch.cuda.synchronize(dev)
    mod_ms = m0.elapsed_time(m1) / 3
    mod_bytes = (12 if weighted else 8) * m + 16 * n

    (elapsed_ms, e2e_ms), (edges_all, e2e_edges_all) = aggregate_over_ranks(
        [elapsed_ms, e2e_ms], [edges, e2e_edges], world, dev)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    peak, peak_kind = measured_hbm_peak()
    launch_ms = sweep_ms / max(sweeps, 1)
    alg_bytes = sweep_bytes(n, m, weighted) + (sweep_bytes(0, m, weighted) if args.rescan else 0)
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    traffic = None
    default_sketch = args.mode == "mg" and args.k == 8 and not (args.unclamped or args.rescan)
    if (default_sketch and SWEEP_TRAFFIC["src_sha256"] == sweep_src_sha()
            and args.workload in (SWEEP_TRAFFIC["workload"], SWEEP_TRAFFIC["captured_on"])):
        # scaled by algorithmic bytes: traffic per algorithmic byte as on the small case
        traffic = round(SWEEP_TRAFFIC["captured_bytes_per_launch"] * alg_bytes
                        / SWEEP_TRAFFIC["captured_algorithmic_bytes"])
    cpu = None
    if world == 1 and not args.skip_cpu:
        times, threads = oracle_sweeps(g, args.mode, seconds=10.0, max_reps=3, k=args.k,
                                       unclamped=args.unclamped, rescan=args.rescan)
        cpu = {"value": len(times) * m / sum(times), "unit": UNIT, "cores": threads,
               "kind": "oracle",
               "sample": f"{len(times)} full oracle sweep(s) (iteration 0 from identity "
                         f"labels) of the same graph, {sum(times):.1f} s"}
    h2d = 8 * (n + 1) + 4 * m + (4 * m if weighted else 0)
    d2h = 4 * n + 64 + 32 + 64 + 8 * 20
    line = {
        "metric": metric_name(args), "value": edges_all / (elapsed_ms * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(args, g),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": sweep_kernel_label(args, weighted),
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "launch_ms": launch_ms, "peak_source": f"{peak_kind} hbm_gbs",
                     # the second fraction: measured DRAM bytes of one sweep over its time
                     "traffic_source": (f"ncu dram bytes of the lane kernel on "
                                        f"{SWEEP_TRAFFIC['captured_on']}, scaled by "
                                        "algorithmic bytes") if traffic else None,
                     "dram_achieved": (traffic / (launch_ms * 1e-3) / 1e9) if traffic else None,
                     "dram_frac": (traffic / (launch_ms * 1e-3) / 1e9 / peak) if traffic else None},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_edges_all / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "pinned_host_memory": pin},
        "gpu_launches": launches,
        "clocks": clk,
        "iterations": [s["iterations"] for s in stats],
        "sweep_ms_iter": [round(x, 3) for x in stats[-1]["sweep_ms_iter"]],
        "modularity": stats[-1]["modularity"],
        "tuning": ({"chosen": tuning, "tuner_s": tune_s, "candidates": len(tune_table),
                    "fixed_defaults": fixed,
                    "table": [[r["tuning"], round(r["ms"], 3)] for r in tune_table]}
                   if args.tune else {"chosen": "defaults"}),
        "modularity_standalone": {"ms": mod_ms, "q": q_alone, "algorithmic_bytes": mod_bytes,
                                  "achieved_gbs": mod_bytes / (mod_ms * 1e-3) / 1e9,
                                  "call": "lpa_modularity_ex (no plan), mean of 3"},
        "setup_ms": stats[-1]["setup_ms"],
        "generate_s": gen_s,
    }
    if world == 1 and default_sketch and args.workload == "lfr26" and not args.no_forms:
        # the batched and served forms, measured after the headline in the same run on the
        # freed device (their own warm-up, timed region and clock record each)
        del ws, d_off, d_idx, d_w, labels, h_lab
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
        lpa.lpa_release_memory()
        line["forms"] = measure_forms(args)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


FORM_KEYS = {
    "batched": ("metric", "value", "unit", "ms_per_step", "steps", "warmup",
                "one_call_per_graph", "e2e", "iterations_max", "iterations_mean",
                "gpu_launches", "clocks", "generate_s"),
    "served": ("metric", "p50_ms", "p99_ms", "mean_ms", "max_ms", "throughput_per_s",
               "by_kind", "one_at_a_time", "bit_equal_sampled", "sampled", "step_ms",
               "steps_over_5ms", "in_flight_mean", "steps", "warmup", "gpu_launches", "clocks",
               "generate_s"),
}


def measure_forms(args) -> dict:
    """Short runs of the batched form (the first 256 graphs of the batched family, 3 timed
    batches) and of the served form (the full arrival stream and request pool, 4000 timed
    requests), without their oracle baselines.  A failure is reported in place of the
    numbers; it never stops the headline line."""
    import argparse as _ap

    out = {}
    for form, workload, steps in (("batched", "sbm256", 3), ("served", "serve", 1)):
        sub = _ap.Namespace(**vars(args))
        sub.workload, sub.steps, sub.warmup, sub.tune, sub.skip_cpu = workload, steps, 3, False, True
        t0 = time.perf_counter()
        try:
            line = run_batch(sub, emit=False) if form == "batched" else run_serve(sub, emit=False)
            res = {k: line[k] for k in FORM_KEYS[form] if k in line}
            res["config"] = line["config"]
            if form == "batched":
                res["roofline_frac"] = line["roofline"]["frac"]
        except Exception as exc:  # noqa: BLE001 -- reported in the line, not raised
            res = {"error": f"{type(exc).__name__}: {exc}"}
        res["wall_s"] = round(time.perf_counter() - t0, 1)
        out[form] = res
        try:
            import torch

            import paper_2411_19901_gb300 as lpa

            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            lpa.lpa_release_memory()
        except Exception:  # noqa: BLE001
            pass
    return out


def _gen_member(g):
    return synth.sbm_member(g, seed=0)


def make_batch(count: int):
    """The batch's graphs, generated on all host cores (a spawn pool: no CUDA state is
    inherited by the workers)."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(min(count, os.cpu_count() or 1)) as pool:
        return pool.map(_gen_member, range(count), chunksize=4)


def run_batch(args, emit: bool = True):
    """Batched form: one lpa_batch_detect over the whole batch per step, against one
    lpa_detect_ex per graph.  Unit: graphs per second over the batch.  Returns the JSON
    line (rank 0), printing it when emit."""
    world, rank, local = dist_env()
    t0 = time.perf_counter()
    gs = make_batch(BATCH_COUNT[args.workload])
    gen_s = time.perf_counter() - t0
    import torch

    import paper_2411_19901_gb300 as lpa
    from paper_2411_19901_gb300 import build

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        barrier = dist.barrier
    else:
        def barrier():
            pass
    dev = torch.device("cuda", local)
    build.build()
    count = len(gs)
    n_all = sum(g.n for g in gs)
    m_all = sum(g.m for g in gs)
    h = [(torch.from_numpy(g.offsets), torch.from_numpy(g.indices)) for g in gs]
    d = [(o.to(dev), i.to(dev), None, torch.empty(g.n, dtype=torch.int32, device=dev))
         for (o, i), g in zip(h, gs)]
    stream = torch.cuda.current_stream(dev)
    tuning, tune_table, tune_s = None, None, 0.0
    if args.tune:  # the tuner's pick for this batch, timed before the timed region
        from paper_2411_19901_gb300 import tune as _tune

        t0 = time.perf_counter()
        tuning, tune_table = _tune.tune_batch(d, mode=args.mode, k=8, reps=1, stream=stream)
        tune_s = time.perf_counter() - t0
    opt = lpa.make_options(validate=False, stream=stream, tuning=tuning)

    def step(o=None):
        return lpa.lpa_batch_detect(d, mode=args.mode, k=8, tol=0.05, max_iter=20,
                                    opt=o or opt)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier()
    clocks = ClockSampler(physical_gpu_index(local))
    launches0 = lpa.lpa_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    time.sleep(0.5)
    torch.cuda.synchronize(dev)
    clocks.mark("start")
    ev0.record(stream)
    results = [step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark("end")
    barrier()
    clk = clocks.stop()
    launches = lpa.lpa_launch_count() - launches0
    elapsed_ms = ev0.elapsed_time(ev1)
    stats = results[-1][0]
    fixed = None
    if args.tune:  # the same steps under the default launch choices
        fopt = lpa.make_options(validate=False, stream=stream)
        step(fopt)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        f0.record(stream)
        for _ in range(args.steps):
            step(fopt)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        fms = f0.elapsed_time(f1) / args.steps
        fixed = {"value": count / (fms * 1e-3), "ms_per_step": fms}
    # one call per graph (the same work, one plan and run per graph)
    one_steps = 1
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(one_steps):
        for (o, i, w, out) in d:
            st = lpa.lpa_stats()
            lpa.lpa_detect_ex(o, i, w, int(o.numel() - 1), int(i.numel()), args.mode, 8, 0.05,
                              20, out, st, opt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    one_ms = e0.elapsed_time(e1) / one_steps
    # end to end: host graphs in, labels out, every step
    pin = world == 1
    hp = [(o.pin_memory(), i.pin_memory()) if pin else (o, i) for (o, i) in h]
    h_out = [torch.empty(g.n, dtype=torch.int32, pin_memory=pin) for g in gs]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_host = time.perf_counter()
    e2.record(stream)
    for _ in range(e2e_steps):
        for (o, i), (do, di, _, _) in zip(hp, d):
            do.copy_(o, non_blocking=True)
            di.copy_(i, non_blocking=True)
        step()
        for ho, (_, _, _, dout) in zip(h_out, d):
            ho.copy_(dout, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = max(e2.elapsed_time(e3), 1e3 * (time.perf_counter() - t_host)) / e2e_steps
    (elapsed_ms, e2e_ms), (graphs_all, e2e_graphs_all) = aggregate_over_ranks(
        [elapsed_ms, e2e_ms * e2e_steps], [count * args.steps, count * e2e_steps], world, dev)
    if rank != 0:
        return
    iters = [s["iterations"] for s in stats]
    useful = sum(it * sweep_bytes(g.n, g.m, g.weights is not None) for it, g in zip(iters, gs))
    cpu = None
    if world == 1 and not args.skip_cpu:
        rate, done, dt, threads = oracle_batch_rate(gs, args.mode, 10.0)
        cpu = {"value": rate, "unit": "graphs/s", "cores": threads, "kind": "oracle",
               "sample": f"full oracle runs of the batch's first {done} graphs, {dt:.1f} s"}
    peak, peak_kind = measured_hbm_peak()
    step_ms = elapsed_ms / args.steps
    line = {
        "metric": BATCH_METRIC, "value": graphs_all / (elapsed_ms * 1e-3), "unit": "graphs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "graphs": count,
                   "n": n_all, "m": m_all, "mode": args.mode, "k": 8, "tol": 0.05,
                   "max_iter": 20, "pl_period": 8, "weights": "unit",
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "single GPU"
                   if world == 1 else "replicas"},
        "one_call_per_graph": {"value": count / (one_ms * 1e-3), "unit": "graphs/s",
                               "ms": one_ms},
        "roofline": {"bound": "hbm", "achieved": useful / (step_ms * 1e-3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": useful / (step_ms * 1e-3) / 1e9 / peak,
                     "traffic": None, "kernel": "whole batched step (useful sweep bytes: "
                     "sum over graphs of its iterations x (8 or 12) m + 20 n)",
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_graphs_all / (e2e_ms * 1e-3), "unit": "graphs/s",
                "h2d_bytes_per_step": sum(8 * (g.n + 1) + 4 * g.m for g in gs),
                "d2h_bytes_per_step": sum(4 * g.n for g in gs), "pinned_host_memory": pin},
        "gpu_launches": launches,
        "clocks": clk,
        "iterations_max": max(iters), "iterations_mean": sum(iters) / len(iters),
        "tuning": ({"chosen": tuning, "tuner_s": tune_s, "candidates": len(tune_table),
                    "fixed_defaults": fixed,
                    "table": [[r["tuning"], round(r["ms"], 3)] for r in tune_table]}
                   if args.tune else {"chosen": "defaults"}),
        "generate_s": gen_s,
    }
    if emit:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return line


def _gen_serve(i):
    if i < 512:
        return synth.sbm_member(i, seed=0)
    return synth.rmat(scale=20, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=i - 512)


def run_serve(args, emit: bool = True):
    """Served form: requests arrive by a Poisson process; each step of the host loop
    submits the requests that have arrived (copying their graph to the device), runs one
    lpa_server_step and polls.  Latency = completion (host clock after the step that
    finished the request) - arrival.  Returns the JSON line (rank 0), printing it when
    emit."""
    import multiprocessing as mp

    world, rank, local = dist_env()
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        gpool = pool.map(_gen_serve, range(520), chunksize=4)
    gen_s = time.perf_counter() - t0
    import torch

    import paper_2411_19901_gb300 as lpa
    from paper_2411_19901_gb300 import build

    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    build.build()
    host = [(torch.from_numpy(g.offsets).pin_memory(), torch.from_numpy(g.indices).pin_memory(),
             None if g.weights is None else torch.from_numpy(g.weights).pin_memory())
            for g in gpool]
    rng = np.random.default_rng(12345 + rank)
    lam = 2000.0
    n_warm, n_timed = 700 * args.warmup, 4000 * args.steps
    total = n_warm + n_timed
    gaps = rng.exponential(1.0 / lam, total)
    arrive = np.cumsum(gaps)
    pick = np.where(rng.random(total) < 0.05, 512 + rng.integers(0, 8, total),
                    rng.integers(0, 512, total))
    stream = torch.cuda.current_stream(dev)
    # admission budget: the resident graphs' footprint stays under 32 GB (requests beyond
    # it wait in the server's queue, and their wait counts in their latency)
    srv = lpa.Server(mode=args.mode, k=8, tol=0.05, max_iter=20, hbm_budget_bytes=32 << 30,
                     validate=False, stream=stream)
    clocks = ClockSampler(physical_gpu_index(local))
    launches0 = lpa.lpa_launch_count()
    inflight = {}
    done_at = np.full(total, np.nan)
    iters = np.zeros(total, dtype=np.int64)
    outputs = {}
    check = set(int(x) for x in rng.choice(np.arange(n_warm, total), size=min(16, n_timed),
                                           replace=False))
    nxt = 0
    steps = 0
    step_time = 0.0
    inflight_sum = 0
    step_admit, step_plain = [], []  # host ms of steps that admitted requests / did not
    step_log = []  # (host ms, requests admitted, requests in flight) of every step
    torch.cuda.synchronize(dev)
    start = time.perf_counter()
    clocks.mark("start")
    while nxt < total or inflight:
        now = time.perf_counter() - start
        if not inflight and nxt < total and arrive[nxt] > now:
            time.sleep(max(0.0, arrive[nxt] - now))
            now = time.perf_counter() - start
        admitted = 0
        while nxt < total and arrive[nxt] <= now:
            ho, hi, hw = host[pick[nxt]]
            do = ho.to(dev, non_blocking=True)
            di = hi.to(dev, non_blocking=True)
            dw = None if hw is None else hw.to(dev, non_blocking=True)
            out = torch.empty(do.numel() - 1, dtype=torch.int32, device=dev)
            inflight[srv.submit(do, di, dw, out)] = (nxt, out)
            nxt += 1
            admitted += 1
        t_step = time.perf_counter()
        srv.step()
        steps += 1
        t_done = time.perf_counter() - start
        dt_step = time.perf_counter() - t_step
        step_time += dt_step
        (step_admit if admitted else step_plain).append(1e3 * dt_step)
        step_log.append((1e3 * dt_step, admitted, len(inflight)))
        inflight_sum += len(inflight)
        for tk in srv.drain():
            st = srv.poll(tk)
            i, out = inflight.pop(tk)
            done_at[i] = t_done
            iters[i] = st["iterations"]
            if i in check:
                outputs[i] = out
    torch.cuda.synchronize(dev)
    clocks.mark("end")
    clk = clocks.stop()
    launches = lpa.lpa_launch_count() - launches0
    srv.close()
    lat = (done_at - arrive)[n_warm:] * 1e3
    span = done_at[n_warm:].max() - arrive[n_warm]
    # bit equality: sampled requests against the same graph solved alone
    equal = True
    for i, out in outputs.items():
        ho, hi, hw = host[pick[i]]
        solo, _ = lpa.detect(ho.to(dev), hi.to(dev), None if hw is None else hw.to(dev),
                             mode=args.mode, validate=False)
        equal = equal and bool(torch.equal(solo, out))
    one = serve_one_at_a_time(lpa, host, gpool, arrive, pick, n_warm, args, stream)
    if rank != 0:
        return
    entries = np.array([gpool[j].m for j in pick])
    kind = np.where(pick[n_warm:] >= 512, "rmat20", "sbm")

    def pct(x, q):
        return float(np.percentile(x, q)) if len(x) else None

    def mean(x):
        return float(np.mean(x)) if len(x) else None
    cpu = None
    if world == 1 and not args.skip_cpu:
        olat, threads = oracle_serve_latencies(gpool, args.mode, 10.0)
        cpu = {"value": float(np.percentile(olat, 99)), "unit": "ms", "cores": threads,
               "kind": "oracle",
               "sample": f"{len(olat)} requests from the same pool, each a full oracle run on "
                         "all host cores, served one at a time with no queueing"}
    line = {
        "metric": SERVE_METRIC, "value": float(np.percentile(lat, 99)), "unit": "ms",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * span / max(args.steps, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serve: {WORKLOADS['serve']}", "requests_timed": int(n_timed),
                   "requests_warmup": int(n_warm), "offered_per_s": lam, "mode": args.mode,
                   "k": 8, "tol": 0.05, "max_iter": 20, "pl_period": 8,
                   "hbm_budget_bytes": 32 << 30, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": "single GPU" if world == 1 else "replicas"},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
        "throughput_per_s": float(n_timed / span),
        "edge_visits_per_s": float((iters[n_warm:] * entries[n_warm:]).sum() / span),
        "by_kind": {k: {"requests": int((kind == k).sum()), "p50_ms": pct(lat[kind == k], 50),
                        "p99_ms": pct(lat[kind == k], 99)} for k in ("sbm", "rmat20")},
        "one_at_a_time": one,
        "server_steps": steps, "step_ms_mean": 1e3 * step_time / max(steps, 1),
        "step_ms": {"admitting": {"steps": len(step_admit), "mean": mean(step_admit),
                                  "p99": pct(step_admit, 99)},
                    "sweep_only": {"steps": len(step_plain), "mean": mean(step_plain),
                                   "p99": pct(step_plain, 99)}},
        "slowest_steps": [{"ms": round(ms, 3), "admitted": a, "in_flight": f}
                          for ms, a, f in sorted(step_log, reverse=True)[:5]],
        "steps_over_5ms": int(sum(1 for ms, _, _ in step_log if ms > 5.0)),
        # latency by the number of sweeps a request needed (its steps in the server)
        "by_iterations": {b: {"requests": int(sel.sum()), "p50_ms": pct(lat[sel], 50),
                              "p99_ms": pct(lat[sel], 99)}
                          for b, sel in (("<=10", iters[n_warm:] <= 10),
                                         ("11-19", (iters[n_warm:] > 10) & (iters[n_warm:] < 20)),
                                         ("20", iters[n_warm:] >= 20))},
        "in_flight_mean": inflight_sum / max(steps, 1),
        "bit_equal_sampled": equal, "sampled": len(outputs),
        "roofline": None, "cpu_baseline": cpu,
        "e2e": {"value": float(np.percentile(lat, 99)), "unit": "ms",
                "h2d_bytes_per_step": int(sum(8 * (gpool[j].n + 1) + 4 * gpool[j].m
                                             for j in pick[n_warm:]) / max(args.steps, 1)),
                "d2h_bytes_per_step": 0,
                "note": "latency is end to end: host-to-device copy at arrival included"},
        "gpu_launches": launches, "clocks": clk, "generate_s": gen_s,
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def serve_one_at_a_time(lpa, host, gpool, arrive, pick, n_warm, args, stream):
    """The same arrival stream served first come, first served by one lpa_detect_host call
    per request on the same GPU (graph copied in from page-locked memory, labels copied
    back); latency = completion - arrival, over the requests after the warm-up ones."""
    import torch

    total = len(arrive)
    opt = lpa.make_options(validate=False, stream=stream)
    out = torch.empty(max(g.n for g in gpool), dtype=torch.int32, pin_memory=True)
    done_at = np.zeros(total)
    start = time.perf_counter()
    for i in range(total):
        now = time.perf_counter() - start
        if arrive[i] > now:
            time.sleep(arrive[i] - now)
        ho, hi, hw = host[pick[i]]
        g = gpool[pick[i]]
        lpa.lpa_detect_host(ho.numpy(), hi.numpy(), None if hw is None else hw.numpy(), g.n,
                            g.m, args.mode, 8, 0.05, 20, out.numpy(), None, opt)
        done_at[i] = time.perf_counter() - start
    lat = (done_at - arrive)[n_warm:] * 1e3
    span = done_at[n_warm:].max() - arrive[n_warm]
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "throughput_per_s": float((total - n_warm) / span),
            "how": "FIFO, one lpa_detect_host per request (host graph in, labels out)"}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="lfr26")
    ap.add_argument("--mode", choices=["mg", "bm", "exact"], default="mg")
    ap.add_argument("--k", type=int, choices=[1, 2, 4, 8, 16, 32], default=8,
                    help="MG sketch slots (single-graph workloads)")
    ap.add_argument("--unclamped", action="store_true",
                    help="MG ablation: the accumulate exactly as printed (LPA_MG_UNCLAMPED)")
    ap.add_argument("--rescan", action="store_true",
                    help="MG ablation: the double scan of Sec. 4.4 (LPA_RESCAN)")
    ap.add_argument("--skip-cpu", action="store_true",
                    help="leave out the oracle's cpu_baseline (for ablation tables; the "
                         "default run always reports it)")
    ap.add_argument("--no-forms", action="store_true",
                    help="leave out the short batched and served runs that the default "
                         "workload reports under 'forms'")
    ap.add_argument("--tune", action="store_true",
                    help="time the autotuner's candidates first and run the timed steps with "
                         "its pick (the default launch choices are timed beside it)")
    args = ap.parse_args()
    if args.mode != "mg" and (args.k != 8 or args.unclamped or args.rescan):
        ap.error("--k, --unclamped and --rescan apply to --mode mg")
    if args.warmup < 3:
        print("note: the timing rules want at least 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in BATCH_COUNT:
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
