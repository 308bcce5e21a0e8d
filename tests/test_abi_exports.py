"""The C ABI library loads and exports every function include/lpa.h declares (CPU only:
no compute call is made)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lpa.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s+(lpa_[a-z_0-9]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lpa_detect", "lpa_detect_ex", "lpa_modularity", "lpa_workspace_size",
                     "lpa_plan_create", "lpa_plan_sweep", "lpa_plan_run", "lpa_plan_destroy",
                     "lpa_status_string", "lpa_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2411_19901_gb300 import build, lpa

    try:
        build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    lib = ctypes.CDLL(lpa.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(lpa.EXPORTED)


def test_host_only_calls():
    from paper_2411_19901_gb300 import lpa

    lpa.load()
    o = lpa.lpa_options_init()
    assert (o.pl_period, o.leaf_e0, o.leaf_max, o.flags) == (8, 64, 256, lpa.LPA_VALIDATE)
    assert lpa.lpa_workspace_size(1000, 10000, "mg") > 4 * 1000
    # exact mode's hub tables hold 2 slots per CSR entry; the sketch modes hold none
    assert lpa.lpa_workspace_size(1000, 10**6, "exact") > lpa.lpa_workspace_size(1000, 10**6, "mg")
    # the default options give the plain bound; a smaller leaf_e0 needs a larger lane table
    assert lpa.lpa_workspace_size_ex(1000, 10000, "mg", 8, o) == lpa.lpa_workspace_size(1000, 10000, "mg")
    o1 = lpa.lpa_options_init()
    o1.leaf_e0 = 1
    assert lpa.lpa_workspace_size_ex(1000, 10000, "mg", 8, o1) > lpa.lpa_workspace_size(1000, 10000, "mg")
    o1.leaf_e0 = 0
    assert lpa.lpa_workspace_size_ex(1000, 10000, "mg", 8, o1) == 0
    assert lpa.load().lpa_status_string(-1) == b"invalid argument"
    assert lpa.lpa_version().startswith("lpa-gb300")
