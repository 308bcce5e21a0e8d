"""The allocation-free modularity entry point (lpa_modularity_noalloc).

It is for callers that cannot allocate device memory when they ask for a result (their
own allocator holds the GPU's memory, or a cudaMalloc would stall a latency-critical
loop); its scratch is a fixed array inside the library.  The test calls it through the
C ABI twice in a row with different labels -- the shared array keeps the first call's
contents, so the second result shows the call clears what it needs -- and compares each
result with lpa_modularity_ex within the 1e-9 relative tolerance the parity tests use.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q_RTOL = 1e-9


@pytest.fixture(scope="module")
def lpa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_19901_gb300 import build

    build.build()
    import paper_2411_19901_gb300.lpa as mod

    mod.load()
    return mod


def test_noalloc_matches_existing_entry_point_twice(lpa):
    g = synth.random_graph(200_000, 12, seed=31, wmax=8, power=2.1, self_loops=0.01)
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    idx = torch.from_numpy(g.indices).to(dev)
    w = torch.from_numpy(g.weights).to(dev)
    rng = np.random.default_rng(5)
    first = torch.from_numpy(rng.integers(0, 3000, g.n).astype(np.int32)).to(dev)
    second = torch.from_numpy((np.arange(g.n) // 7).astype(np.int32)).to(dev)
    opt = lpa.make_options()
    for labels in (first, second):
        q_new = lpa.lpa_modularity_noalloc(off, idx, w, g.n, g.m, labels, opt)
        q_ref = lpa.lpa_modularity_ex(off, idx, w, g.n, g.m, labels, opt)
        assert abs(q_new - q_ref) <= Q_RTOL * max(abs(q_ref), 1e-3), (q_new, q_ref)
    torch.cuda.synchronize()


def test_noalloc_rejects_graphs_over_the_limit(lpa):
    n = lpa.LPA_NOALLOC_MAX_N + 1
    dev = torch.device("cuda:0")
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    idx = torch.zeros(1, dtype=torch.int32, device=dev)
    labels = torch.zeros(n, dtype=torch.int32, device=dev)
    with pytest.raises(lpa.LpaError, match="static scratch limit"):
        lpa.lpa_modularity_noalloc(off, idx, None, n, 0, labels, lpa.make_options())
