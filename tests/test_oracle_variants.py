"""Pins for the oracle's variant paths (CPU only): pruning by unprocessed flags (the
"mark j as unprocessed" step of Alg. 1), the paper-literal Misra-Gries accumulate
(Alg. 2 without sharing), the double scan of Sec. 4.4 and textbook weighted Boyer-Moore.

None of these re-derives the oracle's own code: pruning is checked against an independent
Python replay of the rule around full sweeps and against the fact that, with pick-less
off, a vertex none of whose neighbours moved would choose what it chose before (so
pruning cannot change MG or exact results); the literal sketch against hand-worked
sequences and the textbook Misra-Gries counters it equals for unit weights; the double
scan against exact K_{i->c} of the sketch's candidates computed with numpy; textbook BM
against the k = 1 clamped sketch.
"""
from collections import defaultdict

import numpy as np
import pytest

import oracle
import synth


def _graphs():
    return [
        synth.random_graph(300, 8, seed=1, wmax=5, power=2.2),
        synth.random_graph(500, 12, seed=2, wmax=1, power=2.0, hubs=[(3, 200)]),
        synth.planted_partition(200, 4, 0.2, 0.01, seed=3),
        synth.cliques(5, 7),
    ]


# ------------------------------------------------------------------ pruning


@pytest.mark.parametrize("mode", [oracle.MG, oracle.EXACT])
def test_pruning_does_not_change_mg_or_exact_without_pick_less(mode):
    # symmetric graphs, self-loops skipped: a vertex whose neighbours kept their labels
    # sees the same neighbourhood and chooses the same label again, which it already holds
    for g in _graphs():
        a = oracle.lpa(g.offsets, g.indices, g.weights, mode=mode, rho=0, max_iter=12,
                       tol=0.0)
        b = oracle.lpa(g.offsets, g.indices, g.weights, mode=mode, rho=0, max_iter=12,
                       tol=0.0, prune=True)
        assert np.array_equal(a["labels"], b["labels"])
        assert a["changed"].tolist() == b["changed"].tolist()
        assert a["scanned"].tolist() == [g.m] * a["iterations"]
        assert b["scanned"][0] == g.m and all(s <= g.m for s in b["scanned"])


def _replay_pruned(g, mode, rho, max_iter, tol):
    """Pruned driver restated with full sweeps: sweep everyone, keep only the active
    vertices' moves, then activate every vertex listed in a changed vertex's row."""
    n = g.n
    deg = np.diff(g.offsets)
    C = np.arange(n, dtype=np.int32)
    active = np.ones(n, dtype=bool)
    changed, scanned = [], []
    for l in range(max_iter):
        pl = rho > 0 and l % rho == 0
        full, _ = oracle.move(g.offsets, g.indices, g.weights, C, mode=mode, pick_less=pl)
        nxt = np.where(active, full, C)
        moved = np.nonzero(nxt != C)[0]
        changed.append(len(moved))
        scanned.append(int(deg[active].sum()))
        active = np.zeros(n, dtype=bool)
        for i in moved:
            active[g.indices[g.offsets[i]:g.offsets[i + 1]]] = True
        C = nxt.astype(np.int32)
        if not pl and len(moved) / n < tol:
            break
    return C, changed, scanned


@pytest.mark.parametrize("mode", [oracle.MG, oracle.BM, oracle.EXACT])
@pytest.mark.parametrize("rho", [0, 8, 3])
def test_pruned_driver_matches_an_independent_replay(mode, rho):
    for g in _graphs():
        want_c, want_dn, want_sc = _replay_pruned(g, mode, rho, 15, 0.05)
        got = oracle.lpa(g.offsets, g.indices, g.weights, mode=mode, rho=rho, max_iter=15,
                         tol=0.05, prune=True)
        assert np.array_equal(got["labels"], want_c)
        assert got["changed"].tolist() == want_dn
        assert got["scanned"].tolist() == want_sc


def test_move_with_an_active_mask_keeps_inactive_labels():
    g = _graphs()[0]
    c = np.random.default_rng(4).integers(0, 50, g.n).astype(np.int32)
    act = np.random.default_rng(5).random(g.n) < 0.3
    full, _ = oracle.move(g.offsets, g.indices, g.weights, c)
    part, dn, sc = oracle.move(g.offsets, g.indices, g.weights, c, active=act,
                               return_scanned=True)
    assert np.array_equal(part, np.where(act, full, c))
    assert dn == int((part != c).sum())
    assert sc == int(np.diff(g.offsets)[act].sum())


# ------------------------------------------------------------------ literal MG


def test_literal_mg_drives_weights_negative():
    # k = 1, (y,1), (z,10), (x,5) x 3: the literal rule subtracts every non-matching
    # weight from the one slot: 1 - 10 - 5 - 5 - 5 = -24, and no label is chosen
    y, z, x = 3, 7, 5
    keys, vals = oracle.mg_sketch([y, z, x, x, x], [1, 10, 5, 5, 5], k=1, unclamped=True)
    assert keys.tolist() == [y] and vals.tolist() == [-24.0]
    # the clamped sketch keeps x, the true heavy hitter (15 of 26 > 26 / 2)
    keys, vals = oracle.mg_sketch([y, z, x, x, x], [1, 10, 5, 5, 5], k=1)
    assert keys.tolist() == [x] and vals.tolist() == [6.0]


def test_literal_mg_stale_key_matches_an_empty_slot():
    # k = 2, unit weights: a, b fill both slots; c empties both (a, b stay as stale
    # keys); b then matches its stale slot 1 instead of taking the lowest empty slot 0
    a, b, c = 1, 2, 3
    keys, vals = oracle.mg_sketch([a, b, c, b, b], None, k=2, unclamped=True)
    assert keys.tolist() == [a, b] and vals.tolist() == [0.0, 2.0]
    keys, vals = oracle.mg_sketch([a, b, c, b, b], None, k=2)
    assert keys.tolist() == [b, -1] and vals.tolist() == [2.0, 0.0]


def _textbook_mg(seq, k):
    counters = {}
    for x in seq:
        if x in counters:
            counters[x] += 1
        elif len(counters) < k:
            counters[x] = 1
        else:
            for key in list(counters):
                counters[key] -= 1
                if counters[key] == 0:
                    del counters[key]
    return counters


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_literal_mg_with_unit_weights_is_textbook_mg(k):
    rng = np.random.default_rng(10 + k)
    for _ in range(200):
        d = int(rng.integers(0, 120))
        labels = rng.zipf(1.6, d).clip(0, 40).astype(np.int32)
        keys, vals = oracle.mg_sketch(labels, None, k=k, unclamped=True)
        got = {int(kk): float(v) for kk, v in zip(keys, vals) if v > 0}
        want = {kk: float(v) for kk, v in _textbook_mg(labels.tolist(), k).items()}
        assert got == want


# ------------------------------------------------------------------ double scan


def _star(labels, weights):
    """Vertex 0 joined to vertices 1..d; returns (graph, c_prev) whose row 0 carries the
    given label sequence; vertex 0's own label is n - 1 (never a neighbour's label)."""
    d = len(labels)
    edges = np.stack([np.zeros(d, np.int64), np.arange(1, d + 1)], axis=1)
    g = synth.from_edges(d + 2, edges, np.asarray(weights, np.float32))
    c = np.arange(d + 2, dtype=np.int32)
    c[1:d + 1] = labels
    c[0] = d + 1
    return g, c


@pytest.mark.parametrize("k,e0", [(2, 64), (4, 64), (8, 64), (2, 2), (4, 1)])
def test_double_scan_picks_the_heaviest_candidate(k, e0):
    rng = np.random.default_rng(20 + k + e0)
    for _ in range(100):
        d = int(rng.integers(1, 200))
        labels = rng.zipf(1.4, d).clip(1, 30).astype(np.int32)
        weights = rng.integers(1, 6, d).astype(np.float32)
        g, c = _star(labels, weights)
        row = slice(g.offsets[0], g.offsets[1])
        seq_l = c[g.indices[row]]
        seq_w = g.weights[row]
        keys, vals = oracle.mg_sketch(seq_l, seq_w, k=k, e0=e0)
        cand = [int(kk) for kk, v in zip(keys, vals) if v > 0]
        K = defaultdict(float)
        for lab, w in zip(seq_l.tolist(), seq_w.tolist()):
            K[lab] += w
        # no candidate left (every slot cancelled): no move, the own label stays
        want = min(cand, key=lambda lab: (-K[lab], lab)) if cand else c[0]
        nxt, _ = oracle.move(g.offsets, g.indices, g.weights, c, k=k, e0=e0, rescan=True)
        assert nxt[0] == want


def test_double_scan_equals_exact_when_no_decrement_fires():
    # at most k distinct neighbour labels: the sketch holds every label with its exact
    # weight, so single scan, double scan and Eq. 3 agree
    rng = np.random.default_rng(30)
    for _ in range(100):
        d = int(rng.integers(1, 300))
        labels = rng.integers(1, 9, d).astype(np.int32)   # <= 8 distinct
        weights = rng.integers(1, 9, d).astype(np.float32)
        g, c = _star(labels, weights)
        a, _ = oracle.move(g.offsets, g.indices, g.weights, c, mode=oracle.EXACT)
        b, _ = oracle.move(g.offsets, g.indices, g.weights, c, k=8, rescan=True)
        s, _ = oracle.move(g.offsets, g.indices, g.weights, c, k=8)
        assert a[0] == b[0] == s[0]


def test_variant_flags_are_mg_only():
    g = _graphs()[0]
    for mode in (oracle.BM, oracle.EXACT):
        with pytest.raises(ValueError):
            oracle.lpa(g.offsets, g.indices, g.weights, mode=mode, unclamped=True)
        with pytest.raises(ValueError):
            oracle.lpa(g.offsets, g.indices, g.weights, mode=mode, rescan=True)


# ------------------------------------------------------------------ textbook BM


def test_textbook_weighted_bm_is_the_k1_sketch():
    """Textbook weighted Boyer-Moore (cancel: the heavier side keeps the difference)
    equals the clamped Misra-Gries sketch with one slot."""
    rng = np.random.default_rng(40)
    for _ in range(300):
        d = int(rng.integers(0, 100))
        labels = rng.integers(0, 6, d).astype(np.int32)
        weights = rng.integers(1, 7, d).astype(np.float32)
        cand, wt = None, 0.0
        for lab, w in zip(labels.tolist(), weights.tolist()):
            if wt == 0.0:
                cand, wt = lab, w
            elif lab == cand:
                wt += w
            elif w > wt:
                cand, wt = lab, w - wt
            else:
                wt -= w
        keys, vals = oracle.mg_sketch(labels, weights, k=1, e0=10**6)
        got = (int(keys[0]), float(vals[0])) if vals[0] > 0 else None
        assert got == ((cand, wt) if wt > 0 else None)
