"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The 2^26-vertex LFR-style graph (1.45e9 CSR entries) and the R-MAT scale-22 graph are
built exactly as bench.py builds them and planned with its options (MG, k = 8, e0 = 64,
Lmax = 256).  The oracle is plain C with OpenMP over vertices, so a full sweep of either
graph takes seconds on the host cores: the first two sweeps are compared label by label
and dN by dN, then a whole run (every iteration's dN and the final labels) and the
modularity of the result (1e-9 relative)."""
import os

import numpy as np
import pytest

import oracle
from tolerance import q_close

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def lpa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_19901_gb300 import build

    build.build()
    import paper_2411_19901_gb300 as mod

    return mod


def bench_graph(name):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    return bench.make_graph(name)


@pytest.mark.parametrize("name", ["rmat22", "lfr26"])
def test_full_size_sweeps_and_run(lpa, name):
    g = bench_graph(name)
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    idx = torch.from_numpy(g.indices).to(dev)
    w = None if g.weights is None else torch.from_numpy(g.weights).to(dev)
    # two sweeps from the identity labels: iteration 0 (pick-less) and iteration 1
    c_prev = np.arange(g.n, dtype=np.int32)
    with lpa.Plan(off, idx, w, mode="mg", k=8, validate=False) as plan:
        cp = torch.from_numpy(c_prev).to(dev)
        cn = torch.empty_like(cp)
        for pick_less in (True, False):
            dn = plan.sweep(cp, cn, pick_less)
            want, want_dn = oracle.move(g.offsets, g.indices, g.weights, c_prev, mode=oracle.MG,
                                        k=8, pick_less=pick_less, threads=THREADS)
            got = cn.cpu().numpy()
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, (name, pick_less, bad[:10], got[bad[:10]], want[bad[:10]])
            assert dn == want_dn
            c_prev = want
            cp, cn = cn, cp
    del cp, cn
    # the whole run as bench.py runs it, with the in-run modularity
    labels, st = lpa.detect(off, idx, w, mode="mg", k=8, tol=0.05, max_iter=20, validate=False,
                            modularity=True)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, k=8, tol=0.05,
                     max_iter=20, threads=THREADS)
    assert st["changed"] == ref["changed"].tolist()
    assert st["iterations"] == ref["iterations"] and st["converged"] == ref["converged"]
    got = labels.cpu().numpy()
    assert np.array_equal(got, ref["labels"]), np.nonzero(got != ref["labels"])[0][:10]
    q = oracle.modularity(g.offsets, g.indices, g.weights, ref["labels"])
    assert q_close(st["modularity"], q), (st["modularity"], q)


def banded_graph(n, half):
    """Vertex i joined to i +- 1 .. i +- half (mod n): every row has 2 * half entries, so
    m = 2 * half * n; unit weights; symmetric."""
    import synth

    delta = np.concatenate([np.arange(-half, 0), np.arange(1, half + 1)]).astype(np.int64)
    d = delta.size
    idx = np.empty(n * d, dtype=np.int32)
    step = 1 << 14
    for lo in range(0, n, step):
        hi = min(n, lo + step)
        rows = np.arange(lo, hi, dtype=np.int64)[:, None]
        idx[lo * d:hi * d] = ((rows + delta[None, :]) % n).astype(np.int32).ravel()
    off = np.arange(n + 1, dtype=np.int64) * d
    return synth.Graph(off, idx, None, f"banded_{n}_{half}")


def test_more_than_2_31_entries(lpa):
    """m = 2^31: CSR positions past the int32 range in every kernel (lane and hub
    descriptors, the pipelined fold, the binning), compared sweep by sweep."""
    g = banded_graph(1 << 20, 1024)
    assert g.m == 1 << 31
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    idx = torch.from_numpy(g.indices).to(dev)
    rng = np.random.default_rng(7)
    c_prev = rng.integers(0, 1 << 12, g.n).astype(np.int32)  # few labels: hits and decrements
    with lpa.Plan(off, idx, None, mode="mg", k=8, validate=True) as plan:
        cp = torch.from_numpy(c_prev).to(dev)
        cn = torch.empty_like(cp)
        for pick_less in (True, False):
            dn = plan.sweep(cp, cn, pick_less)
            want, want_dn = oracle.move(g.offsets, g.indices, None, c_prev, mode=oracle.MG, k=8,
                                        pick_less=pick_less, threads=THREADS)
            got = cn.cpu().numpy()
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, (pick_less, bad[:10], got[bad[:10]], want[bad[:10]])
            assert dn == want_dn
            c_prev = want
            cp, cn = cn, cp
