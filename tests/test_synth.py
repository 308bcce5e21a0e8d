"""The seeded synthetic inputs (CPU only): every generator yields a symmetric CSR with
sorted rows and the documented structure, identically for a given seed and for any
number of generator threads.  These graphs stand in for the paper's SuiteSparse graphs,
so their shape is part of what the benchmark measures."""
import numpy as np
import pytest

import synth


def edge_set(g):
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets))
    return rows, g.indices.astype(np.int64)


def check_csr(g, unit=None, loops_allowed=False):
    assert g.offsets[0] == 0 and g.offsets[-1] == g.m
    assert np.all(np.diff(g.offsets) >= 0)
    assert g.indices.dtype == np.int32 and g.offsets.dtype == np.int64
    if g.m:
        assert g.indices.min() >= 0 and g.indices.max() < g.n
    r, c = edge_set(g)
    if not loops_allowed:
        assert not np.any(r == c), "self-loop"
    # rows sorted, no repeated neighbour
    key = r * g.n + c
    assert np.all(np.diff(key) > 0), "rows not sorted or a repeated pair"
    # symmetric, with symmetric weights
    order = np.argsort(c * g.n + r, kind="stable")
    assert np.array_equal((c * g.n + r)[order], key), "not symmetric"
    if g.weights is not None:
        assert g.weights.dtype == np.float32
        assert np.array_equal(g.weights[order], g.weights), "w_ij != w_ji"
        assert np.all(g.weights > 0)
    if unit is True:
        assert g.weights is None or np.all(g.weights == 1.0)


def test_planted_partition_config1():
    g = synth.planted_partition(n=1000, ncomm=10, p_in=0.1, p_out=0.005, seed=0)
    check_csr(g, unit=True)
    assert (g.n, g.m) == (1000, 14170)  # the size the parity tests and bench.py quote
    # more internal than external pairs, as p_in / p_out and the block sizes imply
    r, c = edge_set(g)
    internal = np.mean(r // 100 == c // 100)
    assert 0.6 < internal < 0.75  # expected 4950 * 0.1 / (4950 * 0.1 + 45000 * 0.005) = 0.69
    h = synth.planted_partition(n=1000, ncomm=10, p_in=0.1, p_out=0.005, seed=0)
    assert np.array_equal(g.indices, h.indices)


def test_rmat_structure_and_weights():
    g = synth.rmat(scale=12, edge_factor=16, seed=3)
    check_csr(g)
    # every generated edge adds weight 1 to both directions; self-loops are dropped
    tot = float(g.weights.sum())
    assert tot == np.round(tot) and tot <= 2 * 16 * 4096 and tot > 1.8 * 16 * 4096
    assert np.all(g.weights == np.round(g.weights))
    # heavy-tailed: the largest degree far above the mean
    d = np.diff(g.offsets)
    assert d.max() > 20 * d.mean()
    a = synth.rmat(scale=12, edge_factor=16, seed=3, threads=1)
    b = synth.rmat(scale=12, edge_factor=16, seed=3, threads=4)
    assert np.array_equal(a.indices, b.indices) and np.array_equal(a.weights, b.weights)


def test_lfr_structure_mixing_and_threads():
    n = 1 << 14
    g = synth.lfr(n=n, dmax=2048, cmax=4000, seed=5)
    check_csr(g)
    assert set(np.unique(g.weights)).issubset({float(x) for x in range(1, 9)})
    d = np.diff(g.offsets)
    assert d.max() <= 2048 and d.mean() > 8
    # the planted communities: about 80 % of the entries stay inside (mu = 0.2), and the
    # communities occupy contiguous id ranges
    assert g.communities is not None
    r, c = edge_set(g)
    inside = np.mean(g.communities[r] == g.communities[c])
    assert 0.7 < inside < 0.9
    change = np.count_nonzero(np.diff(g.communities) != 0)
    assert change == np.unique(g.communities).size - 1, "community ids not contiguous"
    h = synth.lfr(n=n, dmax=2048, cmax=4000, seed=5, threads=1)
    assert np.array_equal(g.indices, h.indices) and np.array_equal(g.weights, h.weights)


@pytest.mark.parametrize("member", [0, 1, 7])
def test_sbm_member_structure(member):
    g = synth.sbm_member(member, seed=0, nmax=20000)
    check_csr(g, unit=True)
    assert 100 <= g.n <= 20000
    assert 4 <= g.m / g.n <= 70


def test_small_constructions():
    g = synth.cliques(3, 4)
    check_csr(g, unit=True)
    assert g.m == 3 * 4 * 3
    e = synth.from_edges(4, [[0, 1], [1, 2], [2, 2]], [2.0, 3.0, 5.0])
    check_csr(e, loops_allowed=True)
    assert e.m == 5  # the self-loop is stored once
    rg = synth.random_graph(500, 8, seed=1, wmax=4, self_loops=0.1, power=2.2, hubs=[(3, 300)])
    check_csr(rg, loops_allowed=True)
    # 300 extra random neighbours out of 500 vertices, repeats merged: about 225 distinct
    assert np.diff(rg.offsets)[3] > 200
