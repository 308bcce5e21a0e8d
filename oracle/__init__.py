"""CPU oracle for memory-efficient label propagation (arxiv 2411.19901).

TEST INFRASTRUCTURE ONLY.  Plain, slow C (``lpa_oracle.c``) that restates the paper's
method: Eq. 3 label choice, the weighted Misra-Gries sketch of Sec. 4.1 / Alg. 2 with
partial sketches merged as in Sec. 4.3, the weighted Boyer-Moore rule of Sec. 4.7 /
Alg. 3, the driver of Alg. 1 (`lpa`) and modularity, Eq. 1.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import this package.  It shares no code
with the CUDA library and never imports it.

Functions whose result is pinned only by agreement with the GPU path (full runs on large
graphs) are "parity unpinned" against the paper, which prints no worked example; every
building block below is pinned by the tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

EXACT, MG, BM = 0, 1, 2
PRUNE, UNCLAMPED, RESCAN = 1, 2, 4  # variant flags (pruning, paper-literal MG, double scan)

_c_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_c_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_c_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP, no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lpa_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = [
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
            "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra",
            _SRC, "-o", tmp,
        ]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    lib.oracle_leaf_count.restype = ctypes.c_int32
    lib.oracle_leaf_count.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
    lib.oracle_mg_sketch.restype = ctypes.c_int
    lib.oracle_mg_sketch.argtypes = [
        _c_i32p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_int32, _c_i32p, _c_f32p,
    ]
    lib.oracle_bm_sketch.restype = ctypes.c_int
    lib.oracle_bm_sketch.argtypes = [
        _c_i32p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
    ]
    lib.oracle_choose.restype = ctypes.c_int32
    lib.oracle_choose.argtypes = [
        ctypes.c_int32, _c_i64p, _c_i32p, ctypes.c_void_p, _c_i32p, ctypes.c_int32,
        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
    ]
    lib.oracle_move.restype = ctypes.c_int64
    lib.oracle_move.argtypes = [
        ctypes.c_int32, _c_i64p, _c_i32p, ctypes.c_void_p, _c_i32p, _c_i32p,
        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_int32,
    ]
    lib.oracle_lpa.restype = ctypes.c_int
    lib.oracle_lpa.argtypes = [
        ctypes.c_int32, _c_i64p, _c_i32p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_void_p, _c_i32p, _c_i64p, ctypes.POINTER(ctypes.c_int32),
        ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
    ]
    lib.oracle_mg_sketch_ex.restype = ctypes.c_int
    lib.oracle_mg_sketch_ex.argtypes = [
        _c_i32p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_int32, ctypes.c_int32, _c_i32p, _c_f32p,
    ]
    lib.oracle_move_ex.restype = ctypes.c_int64
    lib.oracle_move_ex.argtypes = [
        ctypes.c_int32, _c_i64p, _c_i32p, ctypes.c_void_p, _c_i32p, _c_i32p, ctypes.c_void_p,
        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
    ]
    lib.oracle_lpa_ex.restype = ctypes.c_int
    lib.oracle_lpa_ex.argtypes = [
        ctypes.c_int32, _c_i64p, _c_i32p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
        ctypes.c_int32, ctypes.c_void_p, _c_i32p, _c_i64p, _c_i64p,
        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
    ]
    lib.oracle_modularity.restype = ctypes.c_double
    lib.oracle_modularity.argtypes = [
        ctypes.c_int32, _c_i64p, _c_i32p, ctypes.c_void_p, _c_i32p,
    ]
    _lib = lib
    return lib


def _wptr(weights):
    if weights is None:
        return None
    assert weights.dtype == np.float32 and weights.flags.c_contiguous
    return weights.ctypes.data


def _graph(offsets, indices, weights):
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    if weights is not None:
        weights = np.ascontiguousarray(weights, dtype=np.float32)
    if indices.size == 0:  # ndpointer wants a real buffer
        indices = np.zeros(1, dtype=np.int32)
    return offsets, indices, weights


def leaf_count(d: int, e0: int = 64, lmax: int = 256) -> int:
    """Number of partial sketches (leaves) for a row of ``d`` CSR positions."""
    return int(_load().oracle_leaf_count(d, e0, lmax))


def mg_sketch(labels, weights=None, k: int = 8, e0: int = 64, lmax: int = 256,
              unclamped: bool = False):
    """Final MG sketch (keys, vals) of a (label, weight) sequence; label < 0 = skip.

    The clamped sketch reports key -1 for empty slots; ``unclamped`` (the paper-literal
    accumulate) returns the raw slots, whose values may be negative and whose empty slots
    may keep a stale key."""
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    keys = np.empty(k, dtype=np.int32)
    vals = np.empty(k, dtype=np.float32)
    lab_buf = lab if lab.size else np.zeros(1, dtype=np.int32)
    if unclamped:
        rc = _load().oracle_mg_sketch_ex(lab_buf, _wptr(w), lab.size, k, e0, lmax, UNCLAMPED,
                                         keys, vals)
    else:
        rc = _load().oracle_mg_sketch(lab_buf, _wptr(w), lab.size, k, e0, lmax, keys, vals)
    if rc != 0:
        raise ValueError("oracle_mg_sketch: bad arguments")
    return keys, vals


def bm_sketch(labels, weights=None, own_label: int = 0, e0: int = 64, lmax: int = 256):
    """Winning (c#, w#) of weighted BM over a sequence; label < 0 = skip."""
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    c = ctypes.c_int32()
    wv = ctypes.c_float()
    lab_buf = lab if lab.size else np.zeros(1, dtype=np.int32)
    rc = _load().oracle_bm_sketch(lab_buf, _wptr(w), lab.size, own_label, e0, lmax,
                                  ctypes.byref(c), ctypes.byref(wv))
    if rc != 0:
        raise ValueError("oracle_bm_sketch: bad arguments")
    return int(c.value), float(wv.value)


def choose(i, offsets, indices, weights, c_prev, mode=MG, k=8, e0=64, lmax=256) -> int:
    """Label vertex ``i`` would pick from ``c_prev`` (before pick-less), -1 if none."""
    offsets, indices, weights = _graph(offsets, indices, weights)
    c_prev = np.ascontiguousarray(c_prev, dtype=np.int32)
    return int(_load().oracle_choose(i, offsets, indices, _wptr(weights), c_prev, mode, k,
                                     e0, lmax))


def _flags(prune=False, unclamped=False, rescan=False) -> int:
    return (PRUNE if prune else 0) | (UNCLAMPED if unclamped else 0) | (RESCAN if rescan else 0)


def move(offsets, indices, weights, c_prev, mode=MG, k=8, e0=64, lmax=256,
         pick_less=False, threads=1, active=None, unclamped=False, rescan=False,
         return_scanned=False):
    """One synchronous sweep; returns (c_next, dN), plus the CSR entries of the swept
    rows when ``return_scanned``.  ``active`` (bool/uint8 per vertex, optional) limits
    the sweep to those vertices; the others keep their label."""
    offsets, indices, weights = _graph(offsets, indices, weights)
    n = offsets.size - 1
    c_prev = np.ascontiguousarray(c_prev, dtype=np.int32)
    c_next = np.empty(max(n, 1), dtype=np.int32)
    act = None
    if active is not None:
        act = np.ascontiguousarray(np.asarray(active).astype(np.uint8))
    scanned = ctypes.c_int64()
    dn = _load().oracle_move_ex(n, offsets, indices, _wptr(weights),
                                c_prev if n else np.zeros(1, np.int32), c_next,
                                act.ctypes.data if act is not None and n else None, mode, k,
                                e0, lmax, int(bool(pick_less)),
                                _flags(unclamped=unclamped, rescan=rescan), threads,
                                ctypes.byref(scanned))
    if return_scanned:
        return c_next[:n], int(dn), int(scanned.value)
    return c_next[:n], int(dn)


def lpa(offsets, indices, weights=None, mode=MG, k=8, tol=0.05, max_iter=20, rho=8,
        e0=64, lmax=256, labels_in=None, threads=1, prune=False, unclamped=False,
        rescan=False):
    """Full run.  Returns dict(labels, changed, scanned, iterations, converged); scanned
    lists the CSR entries swept per iteration (all m unless ``prune``)."""
    offsets, indices, weights = _graph(offsets, indices, weights)
    n = offsets.size - 1
    labels = np.empty(max(n, 1), dtype=np.int32)
    changed = np.zeros(max(max_iter, 1), dtype=np.int64)
    scanned = np.zeros(max(max_iter, 1), dtype=np.int64)
    it = ctypes.c_int32()
    conv = ctypes.c_int32()
    lin = None
    if labels_in is not None:
        lin_arr = np.ascontiguousarray(labels_in, dtype=np.int32)
        lin = lin_arr.ctypes.data
    rc = _load().oracle_lpa_ex(n, offsets, indices, _wptr(weights), mode, k, tol, max_iter,
                               rho, e0, lmax, _flags(prune, unclamped, rescan), lin, labels,
                               changed, scanned, ctypes.byref(it), ctypes.byref(conv),
                               threads)
    if rc != 0:
        raise ValueError("oracle_lpa: bad arguments")
    return {
        "labels": labels[:n].copy(),
        "changed": changed[: it.value].copy(),
        "scanned": scanned[: it.value].copy(),
        "iterations": int(it.value),
        "converged": bool(conv.value),
    }


def modularity(offsets, indices, weights, labels) -> float:
    """Modularity Q (Eq. 1, community form) in fp64."""
    offsets, indices, weights = _graph(offsets, indices, weights)
    n = offsets.size - 1
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    if n == 0:
        return 0.0
    return float(_load().oracle_modularity(n, offsets, indices, _wptr(weights), labels))
