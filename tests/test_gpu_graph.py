"""Runs recorded as one CUDA graph (LPA_GRAPH) give the bits of the direct launches.

A plan records its run once and launches the recorded graph again while labels_out, tol,
max_iter and the flags stay the same; a warm start changes only the contents behind the
plan's labels_in pointer, which the replayed graph reads afresh.  The batched form records
its sweeps per call.  Every result is checked against the CPU oracle (labels, per-sweep
change counts, iterations; modularity within 1e-9 relative), on the legacy default
stream and on a stream of the caller's.
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


def to_dev(g):
    off = torch.from_numpy(g.offsets).cuda()
    idx = torch.from_numpy(g.indices).cuda()
    w = None if g.weights is None else torch.from_numpy(g.weights).cuda()
    return off, idx, w


def graph():
    return synth.random_graph(6000, 14, seed=21, wmax=8, power=2.1,
                              hubs=[(5, 5000), (77, 300), (901, 4097)], self_loops=0.03,
                              zero_weights=0.02)


def check_run(g, st, got, ref, want_q=False):
    assert np.array_equal(got, ref["labels"])
    assert st["changed"] == ref["changed"].tolist()
    assert st["iterations"] == ref["iterations"] and st["converged"] == ref["converged"]
    if want_q:
        assert q_close(st["modularity"], oracle.modularity(g.offsets, g.indices, g.weights,
                                                           ref["labels"]))


@pytest.mark.parametrize("mode,k,prune", [("mg", 8, False), ("mg", 8, True), ("bm", 1, False),
                                          ("exact", 1, False)])
@pytest.mark.parametrize("own_stream", [False, True])
def test_plan_replays_its_recorded_run(lpa, mode, k, prune, own_stream):
    g = graph()
    off, idx, w = to_dev(g)
    side = torch.cuda.Stream() if own_stream else None
    want_q = mode != "exact"
    out = torch.full((g.n,), -3, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    plan = lpa.Plan(off, idx, w, mode=mode, k=k, graph=True, prune=prune, modularity=want_q,
                    stream=side)
    try:
        ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode], k=k, tol=0.05,
                         max_iter=20, prune=prune, threads=4)
        st = plan.run(out, tol=0.05, max_iter=20)  # records, then launches
        check_run(g, st, out.cpu().numpy(), ref, want_q)
        before = lpa.lpa_launch_count()
        out.fill_(-4)
        torch.cuda.synchronize()
        st = plan.run(out, tol=0.05, max_iter=20)  # the same arguments: replays
        assert lpa.lpa_launch_count() > before
        check_run(g, st, out.cpu().numpy(), ref, want_q)
        # another max_iter records a new graph
        ref5 = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode], k=k, tol=0.05,
                          max_iter=5, prune=prune, threads=4)
        st = plan.run(out, tol=0.05, max_iter=5)
        check_run(g, st, out.cpu().numpy(), ref5, want_q)
    finally:
        plan.close()


def test_replay_reads_the_current_warm_start_labels(lpa):
    g = graph()
    off, idx, w = to_dev(g)
    rng = np.random.default_rng(3)
    lab_in = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    plan = lpa.Plan(off, idx, w, mode="mg", graph=True, labels_in=lab_in)
    try:
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for r in range(3):  # the first run records; the others replay with new labels_in
            start = rng.integers(0, g.n // (3 + 5 * r), size=g.n).astype(np.int32)
            lab_in.copy_(torch.from_numpy(start))
            torch.cuda.synchronize()
            st = plan.run(out, tol=0.05, max_iter=20)
            ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, tol=0.05,
                             max_iter=20, labels_in=start, threads=4)
            check_run(g, st, out.cpu().numpy(), ref)
    finally:
        plan.close()


def test_detect_and_batch_with_graph_equal_the_oracle(lpa):
    g = graph()
    off, idx, w = to_dev(g)
    labels, st = lpa.detect(off, idx, w, mode="mg", graph=True, modularity=True)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, threads=4)
    check_run(g, st, labels.cpu().numpy(), ref, want_q=True)
    gs = [synth.cliques(4, 6), synth.planted_partition(n=1000, ncomm=10, p_in=0.1, p_out=0.005,
                                                      seed=0), g]
    gs += [synth.sbm_member(i, seed=1, nmin=100, nmax=3000) for i in range(6)]
    tensors = [(*to_dev(h), torch.full((h.n,), -5, dtype=torch.int32, device="cuda"))
               for h in gs]
    stats, changed = lpa.lpa_batch_detect(tensors, mode="mg", opt=lpa.make_options(graph=True))
    for i, h in enumerate(gs):
        ref = oracle.lpa(h.offsets, h.indices, h.weights, mode=oracle.MG, threads=4)
        assert np.array_equal(tensors[i][3].cpu().numpy(), ref["labels"]), i
        assert stats[i]["iterations"] == ref["iterations"], i
        assert changed[i, :ref["iterations"]].tolist() == ref["changed"].tolist(), i
