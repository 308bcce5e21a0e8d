"""Parity of the served form (lpa_server_*) with the oracle: requests join at different
sweeps, share the resident set with others, and each must end exactly as an independent
oracle run of its graph (labels, iteration count, convergence)."""
import numpy as np
import pytest

import oracle
import synth

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


def tensors(g):
    w = None if g.weights is None else dev(g.weights, np.float32)
    idx = dev(g.indices if g.m else np.zeros(0, np.int32), np.int32)
    return (dev(g.offsets, np.int64), idx, w,
            torch.full((max(g.n, 1),), -3, dtype=torch.int32, device="cuda")[:g.n])


def pool():
    return [
        synth.planted_partition(n=1000, ncomm=10, p_in=0.1, p_out=0.005, seed=0),
        synth.random_graph(3000, 10, seed=5, wmax=6, power=2.2, hubs=[(3, 4500), (9, 700)]),
        synth.cliques(5, 7),
        synth.random_graph(2000, 20, seed=7, wmax=3, self_loops=0.05, zero_weights=0.02),
    ] + [synth.sbm_member(g, seed=3, nmin=100, nmax=4000) for g in range(6)]


def drive(lpa, srv, gs, arrivals, max_steps=200):
    """Submit graph i at step arrivals[i]; step until every request is done."""
    pending = {}
    outs, stats = {}, {}
    for step in range(max_steps):
        for i, at in enumerate(arrivals):
            if at == step:
                t = tensors(gs[i])
                pending[srv.submit(*t)] = (i, t)
        srv.step()
        for tk in list(pending):
            st = srv.poll(tk)
            if st is not None:
                i, t = pending.pop(tk)
                outs[i] = t[3].cpu().numpy()
                stats[i] = st
        if not pending and step >= max(arrivals):
            return outs, stats
    raise AssertionError("requests did not finish")


@pytest.mark.parametrize("mode,k,extra", [("mg", 8, {}), ("bm", 1, {}), ("exact", 1, {}),
                                          ("mg", 4, {"rescan": True, "leaf_e0": 1})])
def test_staggered_requests_match_oracle(lpa, mode, k, extra):
    gs = pool()
    arrivals = [0, 0, 1, 2, 2, 5, 7, 7, 11, 12]
    with lpa.Server(mode=mode, k=k, **extra) as srv:
        outs, stats = drive(lpa, srv, gs, arrivals)
    for i, g in enumerate(gs):
        ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode], k=k,
                         e0=extra.get("leaf_e0", 64), rescan=extra.get("rescan", False),
                         tol=0.05, max_iter=20, threads=4)
        assert np.array_equal(outs[i], ref["labels"]), i
        assert stats[i]["iterations"] == ref["iterations"], i
        assert stats[i]["converged"] == ref["converged"], i


def test_budget_queues_requests_and_results_do_not_depend_on_the_mix(lpa):
    gs = pool()
    # about two of the larger graphs fit at a time
    with lpa.Server(mode="mg", hbm_budget_bytes=6_000_000) as srv:
        outs, stats = drive(lpa, srv, gs + gs[:3], list(range(0, 13)))
    for i, g in enumerate(gs + gs[:3]):
        ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, threads=4)
        assert np.array_equal(outs[i], ref["labels"]), i
        assert stats[i]["iterations"] == ref["iterations"], i


def test_server_edge_cases(lpa):
    with lpa.Server(mode="mg", max_iter=20, hbm_budget_bytes=100_000) as srv:
        empty = synth.from_edges(0, np.zeros((0, 2), np.int64))
        t = srv.submit(*tensors(empty))
        assert srv.poll(t) == {"iterations": 0, "converged": True, "edges_scanned": 0}
        with pytest.raises(lpa.LpaError, match="unknown ticket"):
            srv.poll(t)
        big = synth.random_graph(20000, 20, seed=1)
        with pytest.raises(lpa.LpaError, match="budget"):
            srv.submit(*tensors(big))
        assert srv.step() == 0
    with lpa.Server(mode="mg", max_iter=0) as srv:
        g = synth.cliques(2, 4)
        tt = tensors(g)
        t = srv.submit(*tt)
        assert srv.poll(t)["iterations"] == 0
        assert np.array_equal(tt[3].cpu().numpy(), np.arange(g.n))
    with pytest.raises(lpa.LpaError, match="LPA_PRUNE"):
        lpa.Server(mode="mg", prune=True)


@pytest.mark.parametrize("window", [0, 2048])
def test_arena_appends_compacts_and_drains(lpa, window):
    """Thirty requests over thirty steps: the arena appends, leaves dead slots, compacts;
    drain lists exactly the finished tickets and every result matches the oracle.  With
    2048-vertex binning windows most appends keep the windows before the new graph (only
    the rest is re-binned), so the kept and the redone parts must fit together."""
    gs = [synth.sbm_member(g, seed=4, nmin=100, nmax=2500) for g in range(30)]
    gs[7] = synth.random_graph(3000, 10, seed=5, wmax=6, power=2.2, hubs=[(3, 4500), (9, 700)])
    refs = [oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, threads=4) for g in gs]
    outs = {}
    with lpa.Server(mode="mg", tuning={"window": window}) as srv:
        inflight = {}
        for step in range(400):
            if step < 30:
                t = tensors(gs[step])
                inflight[srv.submit(*t)] = (step, t)
            srv.step()
            for tk in srv.drain():
                i, t = inflight.pop(tk)
                st = srv.poll(tk)
                assert st is not None and st["iterations"] == refs[i]["iterations"]
                outs[i] = t[3].cpu().numpy()
            if step >= 30 and not inflight:
                break
        assert not inflight and srv.drain() == []
    for i in range(30):
        assert np.array_equal(outs[i], refs[i]["labels"]), i
