"""Pins for the oracle's sketches (CPU only).

Nothing here re-derives the oracle's own code: the checks are hand-worked examples
(tests/golden, each with its passage), the textbook Misra-Gries algorithm that the
weighted sketch must reduce to with unit weights (Sec. 3.5), the Misra-Gries error
bound and heavy-hitter guarantee (Sec. 3.5 and Sec. 4.4: every label above K_i/(k+1)
survives), exactness when a row has at most k distinct labels, and the mass balance
W - sum(S_v) = (k+1) * (total decrement).
"""
import json
import os
from collections import Counter, defaultdict

import numpy as np
import pytest

import oracle


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)["cases"]


def test_golden_mg_cases(golden_dir):
    for case in _load(golden_dir, "mg_sketch_cases.json"):
        keys, vals = oracle.mg_sketch(case["labels"], case["weights"], k=case["k"],
                                      e0=case["e0"], lmax=case["lmax"])
        got = [[int(kk), float(v)] for kk, v in zip(keys, vals)]
        assert got == case["expected_slots"], case["name"]
        occ = [(float(v), int(kk)) for kk, v in zip(keys, vals) if v > 0]
        choice = min(occ, key=lambda t: (-t[0], t[1]))[1] if occ else -1
        assert choice == case["expected_choice"], case["name"]


def test_golden_bm_cases(golden_dir):
    for case in _load(golden_dir, "bm_cases.json"):
        c, w = oracle.bm_sketch(case["labels"], case["weights"], own_label=case["own_label"],
                                e0=case["e0"], lmax=case["lmax"])
        assert [c, w] == case["expected"], case["name"]


@pytest.mark.parametrize("d,e0,lmax,L", [
    (0, 64, 256, 1), (1, 64, 256, 1), (127, 64, 256, 1), (128, 64, 256, 2),
    (255, 64, 256, 2), (256, 64, 256, 4), (4095, 64, 256, 32), (4096, 64, 256, 64),
    (16383, 64, 256, 128), (16384, 64, 256, 256), (65536, 64, 256, 256),
    (1, 1, 256, 1), (2, 1, 256, 2), (3, 1, 256, 2), (4, 1, 256, 4), (7, 1, 4, 4),
    (10**6, 1, 1, 1), (5, 2, 256, 2), (6, 3, 256, 2), (7, 3, 256, 2), (12, 3, 256, 4),
])
def test_leaf_count_table(d, e0, lmax, L):
    # L(d) = 1 if d < 2*e0 else min(lmax, largest power of two p with p*e0 <= d)
    assert oracle.leaf_count(d, e0, lmax) == L


def _textbook_mg(seq, k):
    """Misra-Gries (1982) frequent items with k counters, unit increments (Sec. 3.5)."""
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


@pytest.mark.parametrize("k", [1, 2, 3, 8, 16])
def test_unit_weights_single_leaf_is_textbook_mg(k):
    rng = np.random.default_rng(100 + k)
    for _ in range(300):
        d = int(rng.integers(0, 120))
        labels = rng.integers(0, int(rng.integers(1, 3 * k + 3)), size=d)
        keys, vals = oracle.mg_sketch(labels, None, k=k, e0=64, lmax=256)
        got = {int(kk): float(v) for kk, v in zip(keys, vals) if v > 0}
        want = {kk: float(v) for kk, v in _textbook_mg(labels.tolist(), k).items()}
        assert got == want


def _check_mg_bounds(labels, weights, k, e0, lmax):
    keys, vals = oracle.mg_sketch(labels, weights, k=k, e0=e0, lmax=lmax)
    K = defaultdict(float)
    for c, w in zip(labels, weights):
        if c >= 0 and w > 0:
            K[int(c)] += float(w)
    W = sum(K.values())
    assert np.all(vals >= 0)
    occ = {int(kk): float(v) for kk, v in zip(keys, vals) if v > 0}
    assert len(occ) == int(np.sum(vals > 0)), "an occupied label appears twice"
    assert all(kk == -1 for kk, v in zip(keys, vals) if v == 0)
    mass = W - sum(occ.values())
    # mass balance: each decrement of delta removes delta from k slots and from w
    assert mass >= 0 and mass % (k + 1) == 0
    D = mass / (k + 1)
    for c, kc in K.items():
        vc = occ.get(c, 0.0)
        assert vc <= kc, (c, vc, kc)
        assert vc >= kc - D, (c, vc, kc, D)  # Misra-Gries error bound
        if kc > W / (k + 1):
            assert c in occ  # heavy hitters survive
    for c in occ:
        assert c in K


@pytest.mark.parametrize("k", [1, 2, 4, 8])
@pytest.mark.parametrize("e0,lmax", [(1, 256), (2, 4), (3, 256), (64, 256), (1, 1), (5, 32)])
def test_mg_bound_and_mass_with_merges(k, e0, lmax):
    rng = np.random.default_rng(7 * k + e0 + lmax)
    for _ in range(150):
        d = int(rng.integers(0, 400))
        nlab = int(rng.integers(1, 4 * k + 4))
        # skewed label distribution so heavy hitters exist
        p = rng.dirichlet(np.full(nlab, 0.3))
        labels = rng.choice(nlab, size=d, p=p).astype(np.int32)
        labels[rng.random(d) < 0.03] = -1  # self-loop positions
        weights = rng.integers(0, 9, size=d).astype(np.float32)  # zeros are skipped
        _check_mg_bounds(labels, weights, k, e0, lmax)


@pytest.mark.parametrize("e0,lmax", [(1, 256), (2, 8), (64, 256)])
def test_mg_exact_when_at_most_k_distinct(e0, lmax):
    rng = np.random.default_rng(e0 * 31 + lmax)
    k = 8
    for _ in range(200):
        d = int(rng.integers(1, 600))
        pool = rng.choice(10**6, size=int(rng.integers(1, k + 1)), replace=False)
        labels = rng.choice(pool, size=d).astype(np.int32)
        weights = rng.integers(1, 9, size=d).astype(np.float32)
        keys, vals = oracle.mg_sketch(labels, weights, k=k, e0=e0, lmax=lmax)
        got = {int(kk): float(v) for kk, v in zip(keys, vals) if v > 0}
        want = defaultdict(float)
        for c, w in zip(labels, weights):
            want[int(c)] += float(w)
        assert got == dict(want)


def test_single_leaf_settings_agree():
    # lmax = 1 and e0 >= d/2 both make one leaf: one sequential fold
    rng = np.random.default_rng(5)
    for _ in range(100):
        d = int(rng.integers(0, 3000))
        labels = rng.integers(0, 30, size=d).astype(np.int32)
        weights = rng.integers(1, 5, size=d).astype(np.float32)
        a = oracle.mg_sketch(labels, weights, k=8, e0=1, lmax=1)
        b = oracle.mg_sketch(labels, weights, k=8, e0=10**6, lmax=256)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _bm_rule(labels, weights, own, lo, hi):
    """The weighted BM rule of Sec. 4.7 as printed, over positions [lo, hi)."""
    c, w = own, 0.0
    for p in range(lo, hi):
        lab, wp = int(labels[p]), float(weights[p])
        if lab < 0 or wp <= 0:
            continue
        if lab == c:
            w += wp
        elif w > wp:
            w -= wp
        else:
            c, w = lab, wp
    return c, w


def test_bm_random_rows_against_rule():
    rng = np.random.default_rng(11)
    for _ in range(400):
        d = int(rng.integers(0, 700))
        labels = rng.integers(-1, 12, size=d).astype(np.int32)
        weights = rng.integers(0, 6, size=d).astype(np.float32)
        own = int(rng.integers(0, 12))
        e0, lmax = [(64, 256), (1, 256), (3, 4), (1, 1)][int(rng.integers(0, 4))]
        L = oracle.leaf_count(d, e0, lmax)
        best = None
        for l in range(L):
            st = _bm_rule(labels, weights, own, (l * d) // L, ((l + 1) * d) // L)
            if best is None or st[1] > best[1] or (st[1] == best[1] and st[0] < best[0]):
                best = st
        got = oracle.bm_sketch(labels, weights, own_label=own, e0=e0, lmax=lmax)
        assert got == (best[0], float(best[1]))


def test_bad_parameters_rejected():
    with pytest.raises(ValueError):
        oracle.mg_sketch([1, 2], None, k=0)
    with pytest.raises(ValueError):
        oracle.mg_sketch([1, 2], None, k=33)
    with pytest.raises(ValueError):
        oracle.mg_sketch([1, 2], None, k=8, lmax=3)


def test_empty_sequence():
    keys, vals = oracle.mg_sketch([], None, k=8)
    assert np.all(keys == -1) and np.all(vals == 0)
    assert Counter(oracle.bm_sketch([], None, own_label=4)) == Counter((4, 0.0))
