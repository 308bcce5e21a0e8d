"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

Labels and per-sweep change counts must match bit for bit (integer-valued fp32 weights
make every sketch sum exact); modularity must agree within 1e-9 relative.  Graphs are
seeded and synthetic, sized so the oracle finishes in seconds while still spanning many
chunks, hub CTAs and ragged tails.
"""
import zlib

import numpy as np
import pytest

import oracle
import synth
from tolerance import q_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMODE = {"exact": oracle.EXACT, "mg": oracle.MG, "bm": oracle.BM}


@pytest.fixture(scope="module")
def lpa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_19901_gb300 import build

    build.build()
    import paper_2411_19901_gb300 as mod

    return mod


def to_dev(g):
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    idx = torch.from_numpy(g.indices if g.m else np.zeros(0, np.int32)).to(dev)
    w = None if g.weights is None else torch.from_numpy(g.weights).to(dev)
    return off, idx, w




# graphs that reach every kernel path: short rows (one leaf), 2..32 leaves in chunks,
# hub CTAs (rows longer than a chunk, or > 32 leaves), self-loops, zero weights
def graph_zoo():
    return {
        "powerlaw_w": synth.random_graph(6000, 14, seed=1, wmax=8, power=2.1,
                                         hubs=[(5, 5000), (77, 300), (901, 4097), (3000, 129)],
                                         self_loops=0.05, zero_weights=0.02),
        "powerlaw_unit": synth.random_graph(5000, 10, seed=2, power=2.3,
                                            hubs=[(1, 4200), (2, 2000), (4999, 128)]),
        "uniform_w": synth.random_graph(3001, 24, seed=3, wmax=3),
        "sparse_isolated": synth.random_graph(4000, 0.7, seed=4, wmax=5),
    }


PARAMS = [(64, 256), (1, 256), (3, 4), (1, 1), (16, 32)]


@pytest.mark.parametrize("name", ["powerlaw_w", "powerlaw_unit", "uniform_w", "sparse_isolated"])
@pytest.mark.parametrize("e0,lmax", PARAMS)
@pytest.mark.parametrize("mode,k", [("mg", 8), ("mg", 1), ("mg", 2), ("mg", 4), ("mg", 16),
                                    ("mg", 32), ("bm", 1), ("exact", 1)])
def test_sweep_matches_oracle(lpa, name, e0, lmax, mode, k):
    if mode == "exact" and (e0, lmax) != (64, 256):
        pytest.skip("leaf parameters do not affect the exact mode")
    if mode == "mg" and k != 8 and (e0, lmax) not in ((64, 256), (1, 256)):
        pytest.skip("k sweep on two leaf settings")
    g = graph_zoo()[name]
    off, idx, w = to_dev(g)
    rng = np.random.default_rng(zlib.crc32(f"{name}/{e0}/{lmax}/{mode}/{k}".encode()))
    plan = lpa.Plan(off, idx, w, mode=mode, k=k, leaf_e0=e0, leaf_max=lmax)
    try:
        for labeling in ("identity", "few", "many"):
            if labeling == "identity":
                c_prev = np.arange(g.n, dtype=np.int32)
            elif labeling == "few":
                c_prev = rng.integers(0, max(2, g.n // 400), size=g.n).astype(np.int32)
            else:
                c_prev = rng.integers(0, max(2, g.n // 8), size=g.n).astype(np.int32)
            cp = torch.from_numpy(c_prev).cuda()
            for pick_less in (False, True):
                cn = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
                dn = plan.sweep(cp, cn, pick_less)
                want, want_dn = oracle.move(g.offsets, g.indices, g.weights, c_prev,
                                            mode=OMODE[mode], k=k, e0=e0, lmax=lmax,
                                            pick_less=pick_less, threads=4)
                got = cn.cpu().numpy()
                bad = np.nonzero(got != want)[0]
                assert bad.size == 0, (labeling, pick_less, bad[:10], got[bad[:10]], want[bad[:10]])
                assert dn == want_dn
    finally:
        plan.close()


@pytest.mark.parametrize("mode", ["mg", "exact", "bm"])
def test_config1_full_run(lpa, mode):
    g = synth.planted_partition(n=1000, ncomm=10, p_in=0.1, p_out=0.005, seed=0)
    off, idx, w = to_dev(g)
    labels, st = lpa.detect(off, idx, w, mode=mode, k=8, tol=0.05, max_iter=20)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode], k=8, tol=0.05,
                     max_iter=20)
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    assert st["changed"] == ref["changed"].tolist()
    assert st["iterations"] == ref["iterations"] and st["converged"] == ref["converged"]
    q = lpa.modularity(off, idx, w, labels)
    assert q_close(q, oracle.modularity(g.offsets, g.indices, g.weights, ref["labels"]))


@pytest.mark.parametrize("mode", ["mg", "bm", "exact"])
@pytest.mark.parametrize("weighted", [True, False])
def test_per_iteration_labels(lpa, mode, weighted):
    g = synth.random_graph(20000, 12, seed=11, wmax=8 if weighted else 0, power=2.1,
                           hubs=[(7, 9000), (8, 600)])
    off, idx, w = to_dev(g)
    plan = lpa.Plan(off, idx, w, mode=mode, k=8)
    gpu = torch.arange(g.n, dtype=torch.int32, device="cuda")
    nxt = torch.empty_like(gpu)
    ref = np.arange(g.n, dtype=np.int32)
    try:
        for l in range(12):
            pl = l % 8 == 0
            dn = plan.sweep(gpu, nxt, pl)
            ref, ref_dn = oracle.move(g.offsets, g.indices, g.weights, ref, mode=OMODE[mode],
                                      k=8, pick_less=pl, threads=4)
            assert np.array_equal(nxt.cpu().numpy(), ref), f"iteration {l}"
            assert dn == ref_dn, f"iteration {l}"
            gpu, nxt = nxt, gpu
    finally:
        plan.close()


def test_full_run_matches_and_is_deterministic(lpa):
    g = synth.random_graph(30000, 16, seed=5, wmax=8, power=2.1, hubs=[(3, 12000)])
    off, idx, w = to_dev(g)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, threads=4)
    a, sa = lpa.detect(off, idx, w, mode="mg")
    b, sb = lpa.detect(off, idx, w, mode="mg", timing=True)
    assert np.array_equal(a.cpu().numpy(), ref["labels"])
    assert torch.equal(a, b) and sa["changed"] == sb["changed"] == ref["changed"].tolist()
    assert sb["sweep_ms"] > 0


@pytest.mark.parametrize("mode", ["mg", "bm", "exact"])
def test_edge_cases(lpa, mode):
    cases = {
        "single_vertex": synth.from_edges(1, np.zeros((0, 2))),
        "no_edges": synth.from_edges(5, np.zeros((0, 2))),
        "self_loops_only": synth.from_edges(3, [[0, 0], [1, 1]], [2.0, 3.0]),
        "k2": synth.from_edges(2, [[0, 1]]),
        "star_big": synth.from_edges(70001, [[0, j] for j in range(1, 70001)],
                                     list(np.arange(70000) % 5 + 1)),
    }
    for name, g in cases.items():
        off, idx, w = to_dev(g)
        labels, st = lpa.detect(off, idx, w, mode=mode, k=8)
        ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode], k=8)
        assert np.array_equal(labels.cpu().numpy(), ref["labels"]), name
        assert st["changed"] == ref["changed"].tolist(), name
        assert st["iterations"] == ref["iterations"], name


def test_empty_graph(lpa):
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    idx = torch.zeros(0, dtype=torch.int32, device="cuda")
    labels, st = lpa.detect(off, idx, None, mode="mg")
    assert labels.numel() == 0 and st["iterations"] == 0 and st["converged"]
    assert lpa.modularity(off, idx, None, labels) == 0.0


def test_degree_thresholds(lpa):
    # rows of exactly 127, 128, 255, 256, 4095, 4096, 4097 positions around the leaf and
    # chunk boundaries, in a graph whose other rows are short
    n = 12000
    edges = []
    rng = np.random.default_rng(21)
    for v, d in ((10, 127), (20, 128), (30, 255), (40, 256), (50, 4095), (60, 4096), (70, 4097)):
        nb = rng.choice(np.arange(100, n), size=d, replace=False)
        edges += [[v, int(j)] for j in nb]
    edges += rng.integers(100, n, size=(30000, 2)).tolist()
    edges = [e for e in edges if e[0] != e[1]]
    key = {(min(a, b), max(a, b)) for a, b in edges}
    edges = sorted(key)
    w = rng.integers(1, 9, size=len(edges)).astype(np.float32)
    g = synth.from_edges(n, edges, w)
    off, idx, wt = to_dev(g)
    labs = rng.integers(0, 60, size=n).astype(np.int32)
    for mode in ("mg", "bm", "exact"):
        with lpa.Plan(off, idx, wt, mode=mode, k=8) as plan:
            cn = torch.empty(n, dtype=torch.int32, device="cuda")
            dn = plan.sweep(torch.from_numpy(labs).cuda(), cn, False)
        want, wdn = oracle.move(g.offsets, g.indices, g.weights, labs, mode=OMODE[mode], k=8)
        assert np.array_equal(cn.cpu().numpy(), want) and dn == wdn, mode


def test_modularity_matches_oracle(lpa):
    rng = np.random.default_rng(8)
    for t in range(6):
        g = synth.random_graph(int(rng.integers(2, 5000)), float(rng.uniform(1, 30)), seed=t,
                               wmax=int(rng.integers(0, 9)), self_loops=0.02)
        off, idx, w = to_dev(g)
        for labels in (np.arange(g.n), np.zeros(g.n), rng.integers(0, max(1, g.n // 50), g.n)):
            labels = labels.astype(np.int32)
            q = lpa.modularity(off, idx, w, torch.from_numpy(labels).cuda())
            assert q_close(q, oracle.modularity(g.offsets, g.indices, g.weights, labels))


# The standalone pass splits each 256-vertex tile's positions evenly over its warps, so
# rows are cut between warps and steps; a hub spans many warps, runs of isolated vertices
# leave empty rows, and label runs of every length meet the per-run Sigma_c atomics.
@pytest.mark.parametrize("case", ["hubs_fractional", "sparse_integer", "unit"])
def test_standalone_modularity_cut_rows_match_oracle(lpa, case):
    if case == "hubs_fractional":
        g = synth.random_graph(20000, 12, seed=5, wmax=8, power=2.1,
                               hubs=[(3, 19000), (700, 5000), (701, 4000), (19999, 9000)],
                               self_loops=0.02, zero_weights=0.03)
        g.weights = (g.weights.astype(np.float64) * 0.37 + 0.011 * (g.weights > 0)).astype(
            np.float32)
    elif case == "sparse_integer":
        g = synth.random_graph(30000, 0.6, seed=6, wmax=5, self_loops=0.01)
    else:
        g = synth.random_graph(9000, 40, seed=7, power=2.1, hubs=[(100, 8000)])
    off, idx, w = to_dev(g)
    rng = np.random.default_rng(11)
    n = g.n
    for labels in (np.arange(n), np.zeros(n), np.arange(n) // 7, np.arange(n) % 2,
                   rng.integers(0, max(1, n // 300), n), np.repeat(rng.integers(0, n, n // 50 + 1), 50)[:n]):
        labels = np.ascontiguousarray(labels.astype(np.int32))
        q = lpa.modularity(off, idx, w, torch.from_numpy(labels).cuda())
        assert q_close(q, oracle.modularity(g.offsets, g.indices, g.weights, labels)), case


def test_validation_rejects_bad_input(lpa):
    g = synth.random_graph(500, 6, seed=9, wmax=4)
    off, idx, w = to_dev(g)
    bad_idx = idx.clone()
    bad_idx[17] = g.n  # out of range
    with pytest.raises(lpa.LpaError, match="index"):
        lpa.detect(off, bad_idx, w)
    bad_w = w.clone()
    bad_w[3] = -1.0
    with pytest.raises(lpa.LpaError, match="weight"):
        lpa.detect(off, idx, bad_w)
    bad_w[3] = float("nan")
    with pytest.raises(lpa.LpaError, match="weight"):
        lpa.detect(off, idx, bad_w)
    bad_off = off.clone()
    bad_off[100] = bad_off[101] + 1
    with pytest.raises(lpa.LpaError, match="offsets"):
        lpa.detect(bad_off, idx, w)
    lab = torch.full((g.n,), g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(lpa.LpaError, match="labels_in"):
        lpa.detect(off, idx, w, labels_in=lab)
    with pytest.raises(lpa.LpaError):
        lpa.detect(off, idx, w, mode="mg", k=3)
    with pytest.raises(lpa.LpaError):
        lpa.detect(off, idx, w, leaf_max=3)
    with pytest.raises(lpa.LpaError):
        lpa.detect(off, idx, w, max_iter=lpa.lpa.LPA_MAX_ITER + 1)
    with pytest.raises(lpa.LpaError, match="overlap"):
        with lpa.Plan(off, idx, w) as plan:
            x = torch.zeros(g.n + 5, dtype=torch.int32, device="cuda")
            plan.sweep(x[:g.n], x[3:g.n + 3])


def test_workspace_stream_warm_start_and_host_entry(lpa):
    g = synth.random_graph(8000, 10, seed=12, wmax=6, power=2.2, hubs=[(1, 5000)])
    off, idx, w = to_dev(g)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG)
    for mode in ("mg", "exact"):
        nbytes = lpa.lpa_workspace_size(g.n, g.m, mode)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            labels, st = lpa.detect(off, idx, w, mode=mode, workspace=ws, stream=s)
        s.synchronize()
        r = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode])
        assert np.array_equal(labels.cpu().numpy(), r["labels"]), mode
    # a smaller leaf_e0 needs the options-aware bound; the plain bound is refused
    r1 = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, e0=1)
    o1 = lpa.make_options(leaf_e0=1)
    ws = torch.empty(lpa.lpa_workspace_size_ex(g.n, g.m, "mg", 8, o1), dtype=torch.uint8, device="cuda")
    labels, st = lpa.detect(off, idx, w, mode="mg", leaf_e0=1, workspace=ws)
    assert np.array_equal(labels.cpu().numpy(), r1["labels"])
    small = torch.empty(lpa.lpa_workspace_size(g.n, g.m, "mg"), dtype=torch.uint8, device="cuda")
    with pytest.raises(lpa.LpaError, match="workspace"):
        lpa.detect(off, idx, w, mode="mg", leaf_e0=1, workspace=small)
    # warm start: one sweep from given labels, no pick-less
    lab = np.random.default_rng(3).integers(0, 100, g.n).astype(np.int32)
    labels, st = lpa.detect(off, idx, w, mode="mg", labels_in=torch.from_numpy(lab).cuda(),
                            pl_period=0, max_iter=1)
    want, dn = oracle.move(g.offsets, g.indices, g.weights, lab, mode=oracle.MG)
    assert np.array_equal(labels.cpu().numpy(), want) and st["changed"] == [dn]
    # host-memory entry point
    out = np.empty(g.n, dtype=np.int32)
    stats = lpa.lpa_stats()
    lpa.lpa_detect_host(g.offsets, g.indices, g.weights, g.n, g.m, "mg", 8, 0.05, 20, out,
                        stats, lpa.make_options())
    assert np.array_equal(out, ref["labels"])
    assert stats.to_dict()["changed"] == ref["changed"].tolist()


def test_memory_pool_release_and_reuse(lpa):
    """Pool-backed allocations survive a release between calls: results stay exact."""
    g = synth.random_graph(5000, 10, seed=21, wmax=4, power=2.2, hubs=[(3, 4200)])
    off, idx, w = to_dev(g)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG)
    for _ in range(2):
        labels, _ = lpa.detect(off, idx, w, mode="mg")
        assert np.array_equal(labels.cpu().numpy(), ref["labels"])
        lpa.lpa_release_memory()
    h = np.empty(g.n, dtype=np.int32)
    lpa.lpa_detect_host(g.offsets, g.indices, g.weights, g.n, g.m, "mg", 8, 0.05, 20, h)
    assert np.array_equal(h, ref["labels"])


def test_convergence_test_is_strict_on_the_device(lpa):
    """dN / N exactly equal to tol does not stop the run (Alg. 1's strict test), on the
    device as in the oracle: triangle (5, 5, 9) plus 17 isolated vertices, N = 20."""
    g = synth.from_edges(20, [[0, 1], [1, 2], [0, 2]])
    off, idx, w = to_dev(g)
    lab = np.arange(20, dtype=np.int32)
    lab[:3] = [5, 5, 9]
    for tol in (0.05, float(np.nextafter(0.05, 1.0))):
        labels, st = lpa.detect(off, idx, w, mode="mg", tol=tol, pl_period=0,
                                labels_in=torch.from_numpy(lab).cuda())
        ref = oracle.lpa(g.offsets, g.indices, None, mode=oracle.MG, rho=0, tol=tol, labels_in=lab)
        assert st["changed"] == ref["changed"].tolist() and st["iterations"] == ref["iterations"]
        assert np.array_equal(labels.cpu().numpy(), ref["labels"])


# Weights of every magnitude the sketch sums meet: integers up to about 2^20 (fp32 sums
# of a row stay exact), just above, and fractional ones (sums round, so the leaf order
# decides the bits).  Weights stay symmetric: each is an elementwise map of an integer
# weight in 1..8.
@pytest.mark.parametrize("weights", ["packed_max", "just_over", "fractional"])
@pytest.mark.parametrize("mode", ["mg", "bm"])
def test_weight_formats_match_oracle(lpa, weights, mode):
    g = synth.random_graph(3000, 18, seed=41, wmax=8, power=2.1, hubs=[(7, 2900), (11, 300)],
                           self_loops=0.03, zero_weights=0.02)
    scale = {"packed_max": lambda x: x * 131071.0,    # largest 1048568 < 2^20
             "just_over": lambda x: x * 131072.0,     # 8 * 2^17 = 2^20 does not fit
             "fractional": lambda x: x + 0.25 * (x > 0)}[weights]
    g.weights = scale(g.weights.astype(np.float64)).astype(np.float32)
    off, idx, w = to_dev(g)
    rng = np.random.default_rng(3)
    plan = lpa.Plan(off, idx, w, mode=mode, k=8)
    try:
        for c_prev in (np.arange(g.n, dtype=np.int32),
                       rng.integers(0, 40, size=g.n).astype(np.int32)):
            cn = torch.empty(g.n, dtype=torch.int32, device="cuda")
            dn = plan.sweep(torch.from_numpy(c_prev).cuda(), cn, False)
            want, want_dn = oracle.move(g.offsets, g.indices, g.weights, c_prev,
                                        mode=OMODE[mode], k=8, threads=4)
            assert np.array_equal(cn.cpu().numpy(), want) and dn == want_dn
    finally:
        plan.close()
    labels, st = lpa.detect(off, idx, w, mode=mode, k=8, modularity=True)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode], k=8)
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    assert st["changed"] == ref["changed"].tolist()
    assert q_close(st["modularity"],
                   oracle.modularity(g.offsets, g.indices, g.weights, ref["labels"]))
