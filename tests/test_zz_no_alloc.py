"""The allocation-free modularity entry point (lpa_modularity_noalloc).

It is for callers that cannot allocate device memory when they ask for a result (their
own allocator holds the GPU's memory, or a cudaMalloc would stall a latency-critical
loop); its scratch is a fixed array inside the library.  The tests call it through the
C ABI twice in a row with different labels -- the shared array keeps the first call's
contents, so the second result shows the call clears what it needs -- and compare each
result with lpa_modularity_ex and with the CPU oracle (Eq. 1) within the tolerance the
parity tests use.  They also check that a call changes neither the device's free memory
nor PyTorch's reserved memory, on a caller's stream with validation off, and the empty
graph.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import synth
from tolerance import q_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lpa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_19901_gb300 import build

    build.build()
    import paper_2411_19901_gb300.lpa as mod

    mod.load()
    return mod


@pytest.fixture(scope="module")
def graph():
    g = synth.random_graph(200_000, 12, seed=31, wmax=8, power=2.1, self_loops=0.01)
    dev = torch.device("cuda:0")
    return g, (torch.from_numpy(g.offsets).to(dev), torch.from_numpy(g.indices).to(dev),
               torch.from_numpy(g.weights).to(dev))


def _label_sets(n):
    rng = np.random.default_rng(5)
    return [rng.integers(0, 3000, n).astype(np.int32), (np.arange(n) // 7).astype(np.int32)]


def test_noalloc_matches_existing_entry_point_and_oracle_twice(lpa, graph):
    g, (off, idx, w) = graph
    opt = lpa.make_options()
    for labels in _label_sets(g.n):
        d_lab = torch.from_numpy(labels).to(off.device)
        q_new = lpa.lpa_modularity_noalloc(off, idx, w, g.n, g.m, d_lab, opt)
        q_ex = lpa.lpa_modularity_ex(off, idx, w, g.n, g.m, d_lab, opt)
        q_ref = oracle.modularity(g.offsets, g.indices, g.weights, labels)
        assert q_close(q_new, q_ref), (q_new, q_ref)
        assert q_close(q_new, q_ex), (q_new, q_ex)
    torch.cuda.synchronize()


def test_noalloc_allocates_nothing_on_a_callers_stream(lpa, graph):
    g, (off, idx, w) = graph
    labels = _label_sets(g.n)[1]
    d_lab = torch.from_numpy(labels).to(off.device)
    side = torch.cuda.Stream()
    opt = lpa.make_options(validate=False, stream=side)
    side.wait_stream(torch.cuda.current_stream())
    # the first call on a device may look up the scratch array (module loading); measure
    # around the calls after it
    lpa.lpa_modularity_noalloc(off, idx, w, g.n, g.m, d_lab, opt)
    lpa.lpa_release_memory()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    qs = [lpa.lpa_modularity_noalloc(off, idx, w, g.n, g.m, d_lab, opt) for _ in range(2)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    q_ref = oracle.modularity(g.offsets, g.indices, g.weights, labels)
    assert all(q_close(q, q_ref) for q in qs), (qs, q_ref)


def test_noalloc_empty_graph_is_zero(lpa):
    dev = torch.device("cuda:0")
    off = torch.zeros(1, dtype=torch.int64, device=dev)
    idx = torch.zeros(4, dtype=torch.int32, device=dev)
    lab = torch.zeros(4, dtype=torch.int32, device=dev)
    assert lpa.lpa_modularity_noalloc(off, idx, None, 0, 0, lab, lpa.make_options()) == 0.0


def test_noalloc_rejects_graphs_over_the_limit(lpa):
    n = lpa.LPA_NOALLOC_MAX_N + 1
    dev = torch.device("cuda:0")
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    idx = torch.zeros(1, dtype=torch.int32, device=dev)
    labels = torch.zeros(n, dtype=torch.int32, device=dev)
    with pytest.raises(lpa.LpaError, match="static scratch limit"):
        lpa.lpa_modularity_noalloc(off, idx, None, n, 0, labels, lpa.make_options())
