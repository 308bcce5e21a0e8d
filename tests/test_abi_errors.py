"""Argument checks of the C ABI that happen on the host before any device work, so they
run without a GPU: each bad call returns the status the header documents and leaves a
message in lpa_last_error."""
import ctypes
import math

import pytest


@pytest.fixture(scope="module")
def lpa():
    from paper_2411_19901_gb300 import build, lpa as mod

    try:
        build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    mod.load()
    return mod


def status_of(call):
    from paper_2411_19901_gb300 import lpa as mod

    try:
        call()
    except mod.LpaError as e:
        return e.status, str(e)
    return 0, ""


EINVAL, EUNSUPPORTED = -1, -5


def test_detect_argument_checks(lpa):
    fake = 1 << 20  # never dereferenced: every call below fails before device work
    cases = [
        (dict(n=-1, m=0, offsets=fake), EINVAL, "negative"),
        (dict(n=10, m=-1, offsets=fake), EINVAL, "out of range"),
        (dict(n=10, m=5, offsets=None), EINVAL, "offsets is NULL"),
        (dict(n=10, m=5, offsets=fake, indices=None), EINVAL, "indices is NULL"),
        (dict(n=10, m=5, offsets=fake, mode=7), EINVAL, "unknown mode"),
        (dict(n=10, m=5, offsets=fake, k=0), EINVAL, "k = 0"),
        (dict(n=10, m=5, offsets=fake, k=3), EUNSUPPORTED, "k = 3"),
        (dict(n=10, m=5, offsets=fake, max_iter=-1), EINVAL, "max_iter"),
        (dict(n=10, m=5, offsets=fake, max_iter=100000), EINVAL, "max_iter"),
        (dict(n=10, m=5, offsets=fake, indices=fake + 4), EINVAL, "16-byte"),
    ]
    for kw, want, text in cases:
        args = dict(offsets=fake, indices=fake, weights=None, n=10, m=5, mode="mg", k=8,
                    tol=0.05, max_iter=20)
        args.update(kw)
        st, msg = status_of(lambda: lpa.lpa_detect_ex(
            args["offsets"], args["indices"], args["weights"], args["n"], args["m"],
            args["mode"], args["k"], args["tol"], args["max_iter"], fake))
        assert st == want and text in msg, (kw, st, msg)


def test_option_checks(lpa):
    fake = 1 << 20
    for field, value, text in [("pl_period", -1, "pl_period"), ("leaf_e0", 0, "leaf_e0"),
                               ("leaf_max", 3, "leaf_max"), ("leaf_max", 512, "leaf_max")]:
        o = lpa.lpa_options_init()
        setattr(o, field, value)
        st, msg = status_of(lambda: lpa.lpa_detect_ex(fake, fake, None, 10, 5, "mg", 8, 0.05, 20,
                                                      fake, None, o))
        assert st == EINVAL and text in msg, (field, st, msg)
    for mode in ("bm", "exact"):
        o = lpa.lpa_options_init()
        o.flags |= lpa.LPA_RESCAN
        st, msg = status_of(lambda: lpa.lpa_detect_ex(fake, fake, None, 10, 5, mode, 8, 0.05, 20,
                                                      fake, None, o))
        assert st == EINVAL and "LPA_MG only" in msg
    # a recorded graph cannot carry the per-sweep timing events
    o = lpa.lpa_options_init()
    o.flags |= lpa.LPA_TIMING | lpa.LPA_GRAPH
    st, msg = status_of(lambda: lpa.lpa_detect_ex(fake, fake, None, 10, 5, "mg", 8, 0.05, 20,
                                                  fake, None, o))
    assert st == EINVAL and "LPA_GRAPH" in msg and "LPA_TIMING" in msg


def test_batch_and_server_argument_checks(lpa):
    lib = lpa.load()
    assert lib.lpa_batch_detect(None, -1, 1, 8, 0.05, 20, None, None, None) == EINVAL
    assert lib.lpa_batch_detect(None, 2, 1, 8, 0.05, 20, None, None, None) == EINVAL
    assert lib.lpa_batch_detect(None, 0, 1, 8, 0.05, 20, None, None, None) == 0  # empty batch
    bad = (lpa.lpa_graph * 1)()
    bad[0] = lpa.lpa_graph(None, None, None, 5, 0, None)
    assert lib.lpa_batch_detect(ctypes.cast(bad, ctypes.c_void_p), 1, 1, 8, 0.05, 20, None,
                                None, None) == EINVAL
    assert "graph 0" in lib.lpa_last_error().decode()
    h = ctypes.c_void_p()
    assert lib.lpa_server_create(9, 8, 0.05, 20, 0, None, ctypes.byref(h)) == EINVAL
    assert lib.lpa_server_create(1, 8, math.nan, 20, 0, None, ctypes.byref(h)) == EINVAL
    o = lpa.lpa_options_init()
    o.flags |= lpa.LPA_PRUNE
    assert lib.lpa_server_create(1, 8, 0.05, 20, 0, ctypes.byref(o), ctypes.byref(h)) == EUNSUPPORTED
    assert lib.lpa_server_submit(None, None, None) == EINVAL
    assert lib.lpa_server_destroy(None) == 0


def test_status_strings_and_sizes(lpa):
    lib = lpa.load()
    for code in range(0, -7, -1):
        assert lib.lpa_status_string(code)
    assert lpa.lpa_workspace_size(-1, 0, "mg") == 0
    a = lpa.lpa_workspace_size(10**6, 10**7, "mg")
    b = lpa.lpa_workspace_size(10**6, 10**8, "mg")
    c = lpa.lpa_workspace_size(2 * 10**6, 10**8, "mg")
    assert 0 < a < b < c  # the lane table grows with m / e0, the vertex tables with n
