"""The autotuner's candidates (lpa_tuning: binning window, lane CTA size, weight format,
hub stream) never change a result: every candidate must give the oracle's labels and
per-iteration change counts bit for bit, on graphs that reach hubs, mid rows and short
rows, weighted and not.  Also the tuner end to end (JSON cache) and the tuning checks."""
import json

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OMODE = {"mg": oracle.MG, "bm": oracle.BM}


@pytest.fixture(scope="module")
def lpa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_19901_gb300 import build

    build.build()
    import paper_2411_19901_gb300 as mod

    return mod


def _dev(g):
    d = torch.device("cuda:0")
    return (torch.from_numpy(g.offsets).to(d), torch.from_numpy(g.indices).to(d),
            None if g.weights is None else torch.from_numpy(g.weights).to(d))


GRAPHS = {
    "weighted": lambda: synth.random_graph(40000, 14, seed=61, wmax=8, power=2.1,
                                           hubs=[(5, 9000), (77, 5000), (901, 300)],
                                           self_loops=0.02, zero_weights=0.01),
    "unit": lambda: synth.random_graph(30000, 10, seed=62, power=2.3, hubs=[(1, 6000)]),
}


@pytest.mark.parametrize("graph", ["weighted", "unit"])
@pytest.mark.parametrize("mode,k", [("mg", 8), ("bm", 1), ("mg", 4)])
def test_every_candidate_matches_oracle(lpa, graph, mode, k):
    from paper_2411_19901_gb300 import tune

    g = GRAPHS[graph]()
    off, idx, w = _dev(g)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode], k=k, threads=8)
    cands = tune.candidates(g.weights is not None, mode, k)
    assert len(cands) == (18 if k != 4 else 6)
    for c in cands:
        labels, st = lpa.detect(off, idx, w, mode=mode, k=k, tuning=c)
        assert np.array_equal(labels.cpu().numpy(), ref["labels"]), c
        assert st["changed"] == ref["changed"].tolist(), c


def test_tuner_picks_a_candidate_and_caches_it(lpa, tmp_path):
    from paper_2411_19901_gb300 import tune

    g = GRAPHS["weighted"]()
    off, idx, w = _dev(g)
    cache = str(tmp_path / "tuning.json")
    best, table = tune.tune_graph(off, idx, w, reps=1, cache=cache)
    assert best in tune.candidates(True) and len(table) == 18
    assert min(r["ms"] for r in table) == next(r["ms"] for r in table if r["tuning"] == best)
    data = json.load(open(cache))
    assert list(data.values())[0]["best"] == best
    again, _ = tune.tune_graph(off, idx, w, cache=cache)  # served from the cache
    assert again == best
    labels, _ = lpa.detect(off, idx, w, tuning=best)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, threads=8)
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])


def test_batch_tuning_keeps_results(lpa):
    from paper_2411_19901_gb300 import tune

    gs = [synth.sbm_member(i, seed=0) for i in range(6)]
    dev = torch.device("cuda:0")
    graphs = [(torch.from_numpy(g.offsets).to(dev), torch.from_numpy(g.indices).to(dev), None,
               torch.empty(g.n, dtype=torch.int32, device=dev)) for g in gs]
    best, table = tune.tune_batch(graphs, reps=1)
    assert len(table) == 18
    lpa.lpa_batch_detect(graphs, opt=lpa.make_options(tuning=best))
    for g, (_, _, _, out) in zip(gs, graphs):
        ref = oracle.lpa(g.offsets, g.indices, None, threads=8)
        assert np.array_equal(out.cpu().numpy(), ref["labels"])


@pytest.mark.parametrize("bad", [{"window": 1000}, {"window": 32768}, {"lane_threads": 96},
                                 {"serial_hubs": -1}])
def test_tuning_out_of_range_is_refused(lpa, bad):
    g = synth.random_graph(100, 4, seed=1)
    off, idx, w = _dev(g)
    with pytest.raises(lpa.LpaError, match="tuning"):
        lpa.detect(off, idx, w, tuning=bad)
