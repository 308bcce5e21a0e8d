"""Pins for the oracle's sweep, driver and modularity (CPU only).

Checks come from outside the oracle: brute-force Eq. 3 on every small graph, whole runs
worked by hand (tests/golden/driver_cases.json), the closed forms for disjoint cliques,
and modularity by its all-pairs definition (Eq. 1 read as a sum over all vertex pairs)
and its closed forms.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import synth

MODES = {"exact": oracle.EXACT, "mg": oracle.MG, "bm": oracle.BM}


def _brute_choice(g, i, c_prev):
    """Eq. 3 by enumeration of every label: argmax_c sum_{j != i, C_j = c} w_ij."""
    n = g.n
    best, bestK = -1, 0.0
    for c in range(n):
        K = 0.0
        for p in range(g.offsets[i], g.offsets[i + 1]):
            j = int(g.indices[p])
            w = 1.0 if g.weights is None else float(g.weights[p])
            if j != i and w > 0 and c_prev[j] == c:
                K += w
        if K > bestK:  # strict: ties keep the smaller c
            best, bestK = c, K
    return best


def _all_graphs(n, rng):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        edges = [pairs[b] for b in range(len(pairs)) if mask >> b & 1]
        w = rng.integers(1, 4, size=len(edges)).astype(np.float32)
        yield synth.from_edges(n, edges, w if len(edges) else None)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_exact_choice_brute_force_all_small_graphs(n):
    rng = np.random.default_rng(n)
    for g in _all_graphs(n, rng):
        for _ in range(3):
            c_prev = rng.integers(0, n, size=n).astype(np.int32)
            want = [_brute_choice(g, i, c_prev) for i in range(n)]
            got = [oracle.choose(i, g.offsets, g.indices, g.weights, c_prev, mode=oracle.EXACT)
                   for i in range(n)]
            assert got == want
            # MG with k >= n - 1 sees at most k distinct labels: exactly Eq. 3
            got_mg = [oracle.choose(i, g.offsets, g.indices, g.weights, c_prev, mode=oracle.MG,
                                    k=8) for i in range(n)]
            assert got_mg == want


def test_move_commit_rule_and_count():
    # commit (Alg. 1 move step): a different label, and a smaller one under pick-less
    rng = np.random.default_rng(3)
    g = synth.random_graph(60, 5, seed=3, wmax=4)
    for pick_less in (False, True):
        c_prev = rng.integers(0, 60, size=60).astype(np.int32)
        c_next, dn = oracle.move(g.offsets, g.indices, g.weights, c_prev, mode=oracle.EXACT,
                                 pick_less=pick_less)
        changed = 0
        for i in range(60):
            c = _brute_choice(g, i, c_prev)
            if c >= 0 and c != c_prev[i] and (not pick_less or c < c_prev[i]):
                assert c_next[i] == c
                changed += 1
            else:
                assert c_next[i] == c_prev[i]
        assert dn == changed


def test_golden_driver_cases(golden_dir):
    with open(os.path.join(golden_dir, "driver_cases.json")) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        g = synth.from_edges(case["n"], case["edges"], case.get("weights"))
        for mode in case["modes"]:
            r = oracle.lpa(g.offsets, g.indices, g.weights, mode=MODES[mode],
                           k=case.get("k", 8), tol=case["tol"], max_iter=case["max_iter"],
                           rho=case["rho"])
            exp = case["expected"]
            assert r["labels"].tolist() == exp["labels"], (case["name"], mode)
            assert r["changed"].tolist() == exp["changed"], (case["name"], mode)
            assert r["iterations"] == exp["iterations"], (case["name"], mode)
            assert r["converged"] == exp["converged"], (case["name"], mode)
            if "modularity" in case:
                q = oracle.modularity(g.offsets, g.indices, g.weights, r["labels"])
                assert q == pytest.approx(case["modularity"], abs=1e-15), case["name"]


@pytest.mark.parametrize("r,s", [(1, 2), (3, 4), (5, 9), (2, 3)])
@pytest.mark.parametrize("mode", ["exact", "mg"])
def test_disjoint_cliques_small(r, s, mode):
    # s <= k + 1: each vertex sees s-1 <= k distinct labels; iteration 0 (pick-less)
    # moves every vertex to its clique's smallest id, iteration 1 changes nothing
    g = synth.cliques(r, s)
    res = oracle.lpa(g.offsets, g.indices, None, mode=MODES[mode], k=8)
    assert res["labels"].tolist() == [q * s for q in range(r) for _ in range(s)]
    assert res["changed"].tolist() == [r * (s - 1), 0]
    assert res["iterations"] == 2 and res["converged"]
    q = oracle.modularity(g.offsets, g.indices, None, res["labels"])
    assert q == pytest.approx(1.0 - 1.0 / r, abs=1e-15)


@pytest.mark.parametrize("mode", ["mg", "bm"])
def test_disjoint_large_cliques_monochrome(mode):
    r, s = 6, 40  # s > k + 1: the sketch decrements, yet each clique ends one label
    g = synth.cliques(r, s)
    res = oracle.lpa(g.offsets, g.indices, None, mode=MODES[mode], k=8, max_iter=20)
    lab = res["labels"].reshape(r, s)
    assert all(len(set(row)) == 1 for row in lab.tolist())
    assert len(set(lab[:, 0].tolist())) == r
    q = oracle.modularity(g.offsets, g.indices, None, res["labels"])
    assert q == pytest.approx(1.0 - 1.0 / r, abs=1e-15)


def _q_all_pairs(g, labels):
    """Eq. 1 left form over all ordered vertex pairs: (1/2m) sum_ij [A_ij - K_i K_j / 2m] d(C_i, C_j)."""
    n = g.n
    A = np.zeros((n, n))
    for i in range(n):
        for p in range(g.offsets[i], g.offsets[i + 1]):
            A[i, g.indices[p]] += 1.0 if g.weights is None else float(g.weights[p])
    K = A.sum(axis=1)
    two_m = K.sum()
    if two_m == 0:
        return 0.0
    same = labels[:, None] == labels[None, :]
    return float(((A - np.outer(K, K) / two_m) * same).sum() / two_m)


def test_modularity_matches_all_pairs_definition():
    rng = np.random.default_rng(9)
    for t in range(40):
        n = int(rng.integers(1, 40))
        g = synth.random_graph(n, float(rng.uniform(0, 6)), seed=t, wmax=int(rng.integers(0, 5)),
                               self_loops=0.1 if t % 3 == 0 else 0.0)
        labels = rng.integers(0, max(1, n // 3), size=n).astype(np.int32)
        q = oracle.modularity(g.offsets, g.indices, g.weights, labels)
        assert q == pytest.approx(_q_all_pairs(g, labels), abs=1e-12)
        assert -0.5 - 1e-12 <= q <= 1.0 + 1e-12


def test_modularity_closed_forms():
    g = synth.random_graph(200, 8, seed=4, wmax=5)
    w = g.weights.astype(np.float64)
    K = np.add.reduceat(w, g.offsets[:-1]) if g.m else np.zeros(g.n)
    K[np.diff(g.offsets) == 0] = 0.0
    two_m = w.sum()
    singletons = np.arange(g.n, dtype=np.int32)
    q = oracle.modularity(g.offsets, g.indices, g.weights, singletons)
    assert q == pytest.approx(-np.sum((K / two_m) ** 2), rel=1e-12)
    one = np.zeros(g.n, dtype=np.int32)
    assert oracle.modularity(g.offsets, g.indices, g.weights, one) == pytest.approx(0.0, abs=1e-15)


def test_empty_graph_and_bad_args():
    off = np.zeros(1, dtype=np.int64)
    r = oracle.lpa(off, np.zeros(0, np.int32), None)
    assert r["iterations"] == 0 and r["converged"] and r["labels"].size == 0
    g = synth.cliques(2, 3)
    with pytest.raises(ValueError):
        oracle.lpa(g.offsets, g.indices, None, mode=7)


def test_warm_start_is_one_sweep_from_given_labels():
    g = synth.planted_partition()
    rng = np.random.default_rng(2)
    lab = rng.integers(0, 50, size=g.n).astype(np.int32)
    r = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, rho=0, labels_in=lab,
                   max_iter=1)
    c_next, dn = oracle.move(g.offsets, g.indices, g.weights, lab, mode=oracle.MG)
    assert np.array_equal(r["labels"], c_next) and r["changed"].tolist() == [dn]


def test_threads_do_not_change_results():
    g = synth.random_graph(3000, 12, seed=8, wmax=8, power=2.2)
    for mode in (oracle.EXACT, oracle.MG, oracle.BM):
        a = oracle.lpa(g.offsets, g.indices, g.weights, mode=mode, threads=1, e0=2)
        b = oracle.lpa(g.offsets, g.indices, g.weights, mode=mode, threads=4, e0=2)
        assert np.array_equal(a["labels"], b["labels"])
        assert np.array_equal(a["changed"], b["changed"])


def test_convergence_test_is_strict():
    """Alg. 1 stops when dN / N < tau: a sweep with dN / N exactly tau does not stop.
    Triangle 0-1-2 labelled (5, 5, 9) plus 17 isolated vertices (N = 20): only vertex 2
    moves in the first sweep (to 5), so dN / N = 1 / 20, the same double as 0.05."""
    g = synth.from_edges(20, [[0, 1], [1, 2], [0, 2]])
    lab = np.arange(20, dtype=np.int32)
    lab[:3] = [5, 5, 9]
    assert 1.0 / 20.0 == 0.05
    r = oracle.lpa(g.offsets, g.indices, None, mode=oracle.MG, rho=0, tol=0.05, labels_in=lab)
    assert r["changed"].tolist() == [1, 0] and r["iterations"] == 2 and r["converged"]
    above = float(np.nextafter(0.05, 1.0))
    r = oracle.lpa(g.offsets, g.indices, None, mode=oracle.MG, rho=0, tol=above, labels_in=lab)
    assert r["changed"].tolist() == [1] and r["iterations"] == 1 and r["converged"]
    assert r["labels"][:3].tolist() == [5, 5, 5]
