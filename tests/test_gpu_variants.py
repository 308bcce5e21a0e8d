"""Parity of the CUDA variants with the oracle: pruning by unprocessed flags (Alg. 1),
the paper-literal MG accumulate (Alg. 2) and the double scan (Sec. 4.4).

Labels, per-sweep change counts and (for pruning) the CSR positions swept per
iteration must match the oracle bit for bit.
"""
import zlib

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


def to_dev(g):
    dev = torch.device("cuda:0")
    off = torch.from_numpy(g.offsets).to(dev)
    idx = torch.from_numpy(g.indices if g.m else np.zeros(0, np.int32)).to(dev)
    w = None if g.weights is None else torch.from_numpy(g.weights).to(dev)
    return off, idx, w


def zoo():
    return {
        # hubs above 4096 entries and above 32 leaves, self-loops, zero weights
        "powerlaw_w": synth.random_graph(6000, 14, seed=1, wmax=8, power=2.1,
                                         hubs=[(5, 5000), (77, 300), (901, 4097), (3000, 129)],
                                         self_loops=0.05, zero_weights=0.02),
        "powerlaw_unit": synth.random_graph(5000, 10, seed=2, power=2.3,
                                            hubs=[(1, 4200), (2, 2000), (4999, 128)]),
        "pp": synth.planted_partition(n=1000, ncomm=10, p_in=0.1, p_out=0.005, seed=0),
        # non-integer weights: every fp32 operation must still match
        "fractional": _fractional(synth.random_graph(3000, 16, seed=9, wmax=8, power=2.2,
                                                     hubs=[(11, 4500)])),
    }


def _fractional(g):
    """The same graph with non-integer weights (an elementwise map keeps w_ij = w_ji)."""
    w = (g.weights * np.float32(0.3711) + np.float32(0.0137)).astype(np.float32)
    return synth.Graph(g.offsets, g.indices, w, g.name + "_frac")


@pytest.mark.parametrize("name", ["powerlaw_w", "powerlaw_unit", "pp"])
@pytest.mark.parametrize("mode", ["mg", "bm", "exact"])
@pytest.mark.parametrize("rho", [8, 0])
def test_pruned_run_matches_oracle(lpa, name, mode, rho):
    g = zoo()[name]
    off, idx, w = to_dev(g)
    labels, st = lpa.detect(off, idx, w, mode=mode, k=8, tol=0.05, max_iter=20, pl_period=rho,
                            prune=True)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=OMODE[mode], k=8, tol=0.05,
                     max_iter=20, rho=rho, prune=True, threads=4)
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    assert st["changed"] == ref["changed"].tolist()
    assert st["scanned"] == ref["scanned"].tolist()
    assert st["edges_scanned"] == int(ref["scanned"].sum())
    assert st["iterations"] == ref["iterations"] and st["converged"] == ref["converged"]


def test_unpruned_run_reports_every_position(lpa):
    g = zoo()["pp"]
    off, idx, w = to_dev(g)
    _, st = lpa.detect(off, idx, w, mode="mg")
    assert st["scanned"] == [g.m] * st["iterations"]


VARIANTS = [(True, False), (False, True), (True, True)]  # (unclamped, rescan)


@pytest.mark.parametrize("name", ["powerlaw_w", "powerlaw_unit", "fractional"])
@pytest.mark.parametrize("unclamped,rescan", VARIANTS)
@pytest.mark.parametrize("k,e0,lmax", [(8, 64, 256), (8, 1, 256), (1, 64, 256), (32, 16, 32),
                                       (4, 3, 4)])
def test_variant_sweep_matches_oracle(lpa, name, unclamped, rescan, k, e0, lmax):
    g = zoo()[name]
    off, idx, w = to_dev(g)
    rng = np.random.default_rng(zlib.crc32(f"{name}/{unclamped}/{rescan}/{k}/{e0}".encode()))
    with lpa.Plan(off, idx, w, mode="mg", k=k, leaf_e0=e0, leaf_max=lmax, unclamped=unclamped,
                  rescan=rescan) as plan:
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
                                            mode=oracle.MG, k=k, e0=e0, lmax=lmax,
                                            pick_less=pick_less, threads=4,
                                            unclamped=unclamped, rescan=rescan)
                got = cn.cpu().numpy()
                bad = np.nonzero(got != want)[0]
                assert bad.size == 0, (labeling, pick_less, bad[:10], got[bad[:10]], want[bad[:10]])
                assert dn == want_dn


@pytest.mark.parametrize("unclamped,rescan,prune", [(True, False, False), (False, True, False),
                                                    (False, True, True), (True, True, True)])
def test_variant_full_run_matches_oracle(lpa, unclamped, rescan, prune):
    g = synth.random_graph(20000, 12, seed=11, wmax=8, power=2.1, hubs=[(7, 9000), (8, 600)])
    off, idx, w = to_dev(g)
    labels, st = lpa.detect(off, idx, w, mode="mg", k=8, unclamped=unclamped, rescan=rescan,
                            prune=prune)
    ref = oracle.lpa(g.offsets, g.indices, g.weights, mode=oracle.MG, k=8, unclamped=unclamped,
                     rescan=rescan, prune=prune, threads=4)
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])
    assert st["changed"] == ref["changed"].tolist()
    assert st["scanned"] == ref["scanned"].tolist()


@pytest.mark.parametrize("mode", ["bm", "exact"])
def test_mg_variant_flags_refused_for_other_modes(lpa, mode):
    g = zoo()["pp"]
    off, idx, w = to_dev(g)
    for kw in ({"unclamped": True}, {"rescan": True}):
        with pytest.raises(lpa.LpaError, match="LPA_MG only"):
            lpa.detect(off, idx, w, mode=mode, **kw)
