"""Parity of the batched form (lpa_batch_detect) with the oracle run graph by graph.

Each graph of the batch must end with the labels, iteration count, convergence flag and
per-sweep change counts of an independent oracle run: the block-diagonal packing shifts
a graph's ids by a constant, which keeps every tie-break and pick-less decision, and
each graph keeps its own stop test.
"""
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


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def batch_graphs():
    gs = [
        synth.from_edges(0, np.zeros((0, 2), np.int64)),            # empty
        synth.from_edges(1, np.zeros((0, 2), np.int64)),            # one isolated vertex
        synth.from_edges(2, [[0, 1]]),                              # K2
        synth.cliques(4, 6),
        synth.planted_partition(n=1000, ncomm=10, p_in=0.1, p_out=0.005, seed=0),
        synth.random_graph(3000, 10, seed=5, wmax=6, power=2.2, hubs=[(3, 4500), (9, 700)]),
        synth.random_graph(500, 4, seed=6),                         # unit weights
        synth.random_graph(2000, 20, seed=7, wmax=3, self_loops=0.05, zero_weights=0.02),
    ]
    gs += [synth.sbm_member(g, seed=1, nmin=100, nmax=3000) for g in range(12)]
    return gs


def run_batch(lpa, gs, mode, k=8, **opts):
    tensors = []
    for g in gs:
        w = None if g.weights is None else dev(g.weights, np.float32)
        tensors.append((dev(g.offsets, np.int64),
                        dev(g.indices if g.m else np.zeros(0, np.int32), np.int32), w,
                        torch.full((max(g.n, 1),), -5, dtype=torch.int32, device="cuda")[:g.n]))
    stats, changed = lpa.lpa_batch_detect(tensors, mode=mode, k=k, tol=0.05, max_iter=20,
                                          opt=lpa.make_options(**opts))
    return [t[3].cpu().numpy() for t in tensors], stats, changed


@pytest.mark.parametrize("mode,k,e0", [("mg", 8, 64), ("mg", 4, 1), ("bm", 1, 64),
                                       ("exact", 1, 64)])
def test_batch_matches_oracle_per_graph(lpa, mode, k, e0):
    gs = batch_graphs()
    labels, stats, changed = run_batch(lpa, gs, mode, k=k, leaf_e0=e0)
    for i, g in enumerate(gs):
        ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode], k=k, e0=e0,
                         tol=0.05, max_iter=20, threads=4)
        assert np.array_equal(labels[i], ref["labels"]), i
        assert stats[i]["iterations"] == ref["iterations"], i
        assert stats[i]["converged"] == ref["converged"], i
        assert changed[i, :ref["iterations"]].tolist() == ref["changed"].tolist(), i
        assert stats[i]["edges_scanned"] == ref["iterations"] * g.m


def test_batch_with_pruning_and_rescan(lpa):
    gs = batch_graphs()
    labels, stats, changed = run_batch(lpa, gs, "mg", prune=True, rescan=True)
    for i, g in enumerate(gs):
        ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, tol=0.05,
                         max_iter=20, prune=True, rescan=True, threads=4)
        assert np.array_equal(labels[i], ref["labels"]), i
        assert changed[i, :ref["iterations"]].tolist() == ref["changed"].tolist(), i
        assert stats[i]["edges_scanned"] == -1


def test_batch_equals_one_call_per_graph(lpa):
    gs = [synth.sbm_member(g, seed=2, nmin=1000, nmax=20000) for g in range(6)]
    labels, stats, _ = run_batch(lpa, gs, "mg")
    for i, g in enumerate(gs):
        w = None if g.weights is None else dev(g.weights, np.float32)
        one, st = lpa.detect(dev(g.offsets, np.int64), dev(g.indices, np.int32), w, mode="mg")
        assert np.array_equal(labels[i], one.cpu().numpy())
        assert stats[i]["iterations"] == st["iterations"]


def test_batch_validation_and_edge_cases(lpa):
    good = synth.cliques(2, 5)
    bad_idx = good.indices.copy()
    bad_idx[3] = good.n + 7
    t = [(dev(good.offsets, np.int64), dev(good.indices, np.int32), None,
          torch.empty(good.n, dtype=torch.int32, device="cuda")),
         (dev(good.offsets, np.int64), dev(bad_idx, np.int32), None,
          torch.empty(good.n, dtype=torch.int32, device="cuda"))]
    with pytest.raises(lpa.LpaError, match="index out of range"):
        lpa.lpa_batch_detect(t, mode="mg")
    stats, changed = lpa.lpa_batch_detect([], mode="mg")
    assert stats == [] and changed.shape[0] == 0
    with pytest.raises(lpa.LpaError, match="labels_in"):
        lpa.lpa_batch_detect(t[:1], mode="mg",
                             opt=lpa.make_options(labels_in=torch.zeros(good.n, dtype=torch.int32,
                                                                        device="cuda")))


def test_batch_modularity_per_graph(lpa):
    gs = batch_graphs()
    labels, stats, _ = run_batch(lpa, gs, "mg", modularity=True)
    for i, g in enumerate(gs):
        ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, threads=4)
        assert np.array_equal(labels[i], ref["labels"]), i
        q = oracle.modularity(g.offsets, g.indices, g.weights, ref["labels"]) if g.n else 0.0
        assert q_close(stats[i]["modularity"], q), (i, stats[i], q)
    with pytest.raises(lpa.LpaError, match="sketch mode"):
        run_batch(lpa, gs[:3], "exact", modularity=True)
