"""Seeded synthetic graphs shared by the CUDA library's tests/benchmarks and the oracle.

The paper measures on SuiteSparse web and social graphs (Sec. 5.1.3, Table 1) that are
not available here; the generators below produce graphs of the same shape instead.
This module holds no part of label propagation itself, only inputs: symmetric CSR
(int64 offsets, int32 neighbour ids sorted per row, fp32 integer-valued weights).

The heavy generators are C (``graphgen.c``, OpenMP, thread-count independent); small
test graphs come from numpy's seeded PCG64.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")


@dataclasses.dataclass
class Graph:
    """Symmetric CSR graph.  ``weights`` None means every weight is 1."""

    offsets: np.ndarray  # int64 [n + 1]
    indices: np.ndarray  # int32 [m]
    weights: np.ndarray | None  # float32 [m] or None
    name: str = ""
    communities: np.ndarray | None = None  # planted community per vertex, if known

    @property
    def n(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def m(self) -> int:
        return int(self.indices.size)

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)


class _CSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("offsets", ctypes.POINTER(ctypes.c_int64)),
        ("indices", ctypes.POINTER(ctypes.c_int32)),
        ("weights", ctypes.POINTER(ctypes.c_float)),
    ]


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` with gcc and OpenMP."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-Wall",
             _SRC, "-o", tmp, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_CSR)
        lib.gg_free.argtypes = [P]
        lib.gg_planted_partition.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_uint64, P]
        lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                ctypes.c_int, P]
        lib.gg_lfr.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                               ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                               ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                               ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                               ctypes.c_void_p, P]
        lib.gg_sbm_member.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_double, P]
        for f in (lib.gg_planted_partition, lib.gg_rmat, lib.gg_lfr, lib.gg_sbm_member):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _take(csr: _CSR, unit: bool, name: str) -> Graph:
    n, m = int(csr.n), int(csr.m)
    try:
        off = np.ctypeslib.as_array(csr.offsets, shape=(n + 1,)).copy()
        idx = (np.ctypeslib.as_array(csr.indices, shape=(m,)).copy() if m
               else np.zeros(0, dtype=np.int32))
        w = None
        if not unit:
            w = (np.ctypeslib.as_array(csr.weights, shape=(m,)).copy() if m
                 else np.zeros(0, dtype=np.float32))
    finally:
        _load().gg_free(ctypes.byref(csr))
    return Graph(off, idx, w, name)


def _threads(threads):
    return int(threads) if threads else (os.cpu_count() or 1)


def planted_partition(n=1000, ncomm=10, p_in=0.1, p_out=0.005, seed=0,
                      unit_weights_array=True) -> Graph:
    """Planted partition: pairs i < j in lexicographic order, one uniform each."""
    csr = _CSR()
    if _load().gg_planted_partition(n, ncomm, p_in, p_out, seed, ctypes.byref(csr)) != 0:
        raise ValueError("planted_partition: bad arguments")
    g = _take(csr, unit=not unit_weights_array, name=f"planted_partition_n{n}_seed{seed}")
    csize = n // ncomm if ncomm <= n else 1
    g.communities = np.minimum(np.arange(n) // csize, ncomm - 1).astype(np.int32)
    return g


def rmat(scale=22, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=0, threads=None) -> Graph:
    """R-MAT, symmetrised, self-loops dropped, duplicates merged by summing weights."""
    csr = _CSR()
    if _load().gg_rmat(scale, edge_factor, a, b, c, seed, _threads(threads),
                       ctypes.byref(csr)) != 0:
        raise ValueError("rmat: bad arguments or out of memory")
    return _take(csr, unit=False, name=f"rmat{scale}_ef{edge_factor}_seed{seed}")


def lfr(n=2**26, gamma_d=2.1, dmin=4, dmax=65536, gamma_c=1.5, cmin=20, cmax=10**6,
        mu=0.2, wmax=8, seed=0, permute=False, threads=None) -> Graph:
    """LFR-style heavy-tailed planted partition with integer weights in 1..wmax."""
    csr = _CSR()
    comm = np.empty(n, dtype=np.int32)
    rc = _load().gg_lfr(n, gamma_d, dmin, dmax, gamma_c, cmin, cmax, mu, wmax, seed,
                        int(bool(permute)), _threads(threads), comm.ctypes.data,
                        ctypes.byref(csr))
    if rc != 0:
        raise ValueError("lfr: bad arguments or out of memory")
    g = _take(csr, unit=False, name=f"lfr_n{n}_seed{seed}{'_perm' if permute else ''}")
    g.communities = comm
    return g


def sbm_member(g, seed=0, nmin=100, nmax=200_000, dmin=8.0, dmax=64.0, cmin=4, cmax=500,
               p_in=0.8) -> Graph:
    """Graph ``g`` of the batched workload (uneven planted-partition graphs)."""
    csr = _CSR()
    rc = _load().gg_sbm_member(seed, g, nmin, nmax, dmin, dmax, cmin, cmax, p_in,
                               ctypes.byref(csr))
    if rc != 0:
        raise ValueError("sbm_member: bad arguments")
    return _take(csr, unit=True, name=f"sbm_{seed}_{g}")


def random_graph(n, avg_degree, seed, wmax=0, self_loops=0.0, zero_weights=0.0,
                 hubs=(), power=None) -> Graph:
    """Small seeded test graph (numpy PCG64), symmetric, neighbours sorted.

    ``wmax`` 0 gives unit weights (weights None), otherwise integers in 1..wmax.
    ``self_loops``/``zero_weights`` are per-vertex / per-edge probabilities.
    ``hubs`` lists (vertex, degree) pairs that get that many extra random neighbours.
    ``power`` draws per-vertex target degrees from a power law with that exponent.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if power is not None:
        u = rng.random(n)
        deg = np.floor((1 - u) ** (-1.0 / (power - 1.0)) * max(avg_degree / 3.0, 1.0))
        deg = np.minimum(deg, max(n - 1, 1)).astype(np.int64)
        src = np.repeat(np.arange(n), deg)
        dst = rng.integers(0, n, size=src.size)
    else:
        ne = int(n * avg_degree / 2)
        src = rng.integers(0, max(n, 1), size=ne)
        dst = rng.integers(0, max(n, 1), size=ne)
    extra_s, extra_d = [src], [dst]
    for v, d in hubs:
        extra_s.append(np.full(d, v))
        extra_d.append(rng.integers(0, n, size=d))
    src = np.concatenate(extra_s).astype(np.int64)
    dst = np.concatenate(extra_d).astype(np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    a, b = np.minimum(src, dst), np.maximum(src, dst)
    key = np.unique(a * n + b)
    a, b = key // n, key % n
    if wmax:
        wu = rng.integers(1, wmax + 1, size=a.size).astype(np.float32)
        wu[rng.random(a.size) < zero_weights] = 0.0
    else:
        wu = np.ones(a.size, dtype=np.float32)
    s_all = np.concatenate([a, b])
    d_all = np.concatenate([b, a])
    w_all = np.concatenate([wu, wu])
    if self_loops > 0:
        loops = np.nonzero(rng.random(n) < self_loops)[0]
        s_all = np.concatenate([s_all, loops])
        d_all = np.concatenate([d_all, loops])
        lw = (rng.integers(1, wmax + 1, size=loops.size).astype(np.float32) if wmax
              else np.ones(loops.size, dtype=np.float32))
        w_all = np.concatenate([w_all, lw])
    order = np.lexsort((d_all, s_all))
    s_all, d_all, w_all = s_all[order], d_all[order], w_all[order]
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.add.at(offsets, s_all + 1, 1)
    offsets = np.cumsum(offsets).astype(np.int64)
    return Graph(offsets, d_all.astype(np.int32),
                 None if not wmax else w_all.astype(np.float32),
                 f"random_n{n}_d{avg_degree}_s{seed}")


def cliques(r, s) -> Graph:
    """r disjoint cliques of size s (ids contiguous per clique), unit weights."""
    rows, cols = [], []
    for q in range(r):
        base = q * s
        for i in range(s):
            for j in range(s):
                if i != j:
                    rows.append(base + i)
                    cols.append(base + j)
    n = r * s
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int32)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.add.at(offsets, rows + 1, 1)
    return Graph(np.cumsum(offsets).astype(np.int64), cols, None, f"cliques_{r}x{s}")


def from_edges(n, edges, weights=None) -> Graph:
    """Symmetric CSR from an undirected edge list (no dedup); rows sorted."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = (np.ones(len(e), dtype=np.float32) if weights is None
         else np.asarray(weights, dtype=np.float32))
    s = np.concatenate([e[:, 0], e[:, 1]])
    d = np.concatenate([e[:, 1], e[:, 0]])
    ww = np.concatenate([w, w])
    loops = e[:, 0] == e[:, 1]
    if loops.any():  # a self-loop is stored once
        keep = np.concatenate([np.ones(len(e), bool), ~loops])
        s, d, ww = s[keep], d[keep], ww[keep]
    order = np.lexsort((d, s))
    s, d, ww = s[order], d[order], ww[order]
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.add.at(offsets, s + 1, 1)
    return Graph(np.cumsum(offsets).astype(np.int64), d.astype(np.int32),
                 None if weights is None else ww.astype(np.float32), "edges")
