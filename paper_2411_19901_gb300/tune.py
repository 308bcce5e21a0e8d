"""Autotuner over the launch choices that never change a result (``lpa_tuning``).

The paper tunes its GPU kernel by hand (the switch degree and block shape of Sec. 4.2);
here every launch choice that leaves the labels alone -- the binning window, the lane
CTA size and whether the hub kernels run beside the lane kernel -- is timed on the
caller's own graph (or batch) and the fastest is kept.  Results are identical under
every candidate (the leaf partition and merge order are fixed by the row lengths alone),
which the GPU tests check.

Winners are cached in a JSON file keyed by a coarse signature of the workload (sizes in
powers of two, weights, mode and k), so a later run of the same kind of graph reuses them
without timing again.  Timing uses CUDA events on the calls' stream; every candidate is
warmed up once first.
"""
from __future__ import annotations

import itertools
import json
import math
import os

from . import lpa as _lpa

WINDOWS = (4096, 8192, 16384)
LANE_THREADS = (64, 128, 256)


def _full_sketch(mode: str, k: int) -> bool:
    """Sketches built with every lane CTA size."""
    return mode == "bm" or (mode == "mg" and k == 8)


def candidates(weighted: bool, mode: str = "mg", k: int = 8) -> list[dict]:
    """Every tuning the library accepts for this kind of call (exact mode: the default)."""
    if mode == "exact":
        return [{}]
    sizes = LANE_THREADS if _full_sketch(mode, k) else (128,)
    return [{"window": w, "lane_threads": t, "serial_hubs": s}
            for w, t, s in itertools.product(WINDOWS, sizes, (0, 1))]


def signature(kind: str, n: int, m: int, weighted: bool, mode: str, k: int,
              count: int = 1) -> str:
    """Coarse workload key: sizes rounded to powers of two."""
    lg = lambda x: int(round(math.log2(max(x, 1))))  # noqa: E731
    return f"{kind}:n2^{lg(n)}:m2^{lg(m)}:count2^{lg(count)}:{'w' if weighted else 'unit'}:{mode}{k}"


def _time_ms(run, reps: int, stream) -> float:
    import torch

    run()  # warm-up: the library's memory pool grows, code is loaded
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _search(run_with, cands: list[dict], reps: int, stream) -> tuple[dict, list[dict]]:
    table = []
    for c in cands:
        table.append({"tuning": c, "ms": _time_ms(lambda: run_with(c), reps, stream)})
    best = min(table, key=lambda r: r["ms"])
    return best["tuning"], table


def _load(cache: str | None) -> dict:
    if cache and os.path.exists(cache):
        with open(cache) as f:
            return json.load(f)
    return {}


def _store(cache: str | None, key: str, best: dict, table: list[dict]) -> None:
    if not cache:
        return
    data = _load(cache)
    data[key] = {"best": best, "table": table}
    tmp = f"{cache}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, cache)


def tune_graph(offsets, indices, weights=None, mode: str = "mg", k: int = 8, tol: float = 0.05,
               max_iter: int = 20, reps: int = 2, cache: str | None = None, stream=None,
               retune: bool = False) -> tuple[dict, list[dict]]:
    """Fastest tuning for whole runs (lpa_detect_ex) on this device graph; returns it and
    the timing table.  A cached winner for the same signature is returned without timing
    unless ``retune``."""
    import torch

    n, m = int(offsets.numel() - 1), int(indices.numel())
    key = signature("graph", n, m, weights is not None, mode, k)
    hit = _load(cache).get(key)
    if hit and not retune:
        return hit["best"], hit["table"]
    stream = stream or torch.cuda.current_stream()
    labels = torch.empty(n, dtype=torch.int32, device=offsets.device)

    def run_with(c):
        opt = _lpa.make_options(validate=False, stream=stream, tuning=c)
        _lpa.lpa_detect_ex(offsets, indices, weights, n, m, mode, k, tol, max_iter, labels,
                           None, opt)

    best, table = _search(run_with, candidates(weights is not None, mode, k), reps, stream)
    _store(cache, key, best, table)
    return best, table


def tune_batch(graphs, mode: str = "mg", k: int = 8, tol: float = 0.05, max_iter: int = 20,
               reps: int = 1, cache: str | None = None, stream=None,
               retune: bool = False) -> tuple[dict, list[dict]]:
    """Fastest tuning for lpa_batch_detect on these graphs (tuples as lpa_batch_detect
    takes them); returns it and the timing table."""
    import torch

    n = sum(int(g[0].numel() - 1) for g in graphs)
    m = sum(int(g[1].numel()) for g in graphs)
    weighted = any(g[2] is not None for g in graphs)
    key = signature("batch", n, m, weighted, mode, k, count=len(graphs))
    hit = _load(cache).get(key)
    if hit and not retune:
        return hit["best"], hit["table"]
    stream = stream or torch.cuda.current_stream()

    def run_with(c):
        opt = _lpa.make_options(validate=False, stream=stream, tuning=c)
        _lpa.lpa_batch_detect(graphs, mode=mode, k=k, tol=tol, max_iter=max_iter, opt=opt)

    best, table = _search(run_with, candidates(weighted, mode, k), reps, stream)
    _store(cache, key, best, table)
    return best, table
