"""The C-ABI library builds, loads and exports every function that
include/panda.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(panda_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_1507_07039_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("panda_create", "panda_step", "panda_run", "panda_get", "panda_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_loads_and_reports_errors_without_a_gpu(lib_path):
    import numpy as np
    from paper_1507_07039_gb300 import panda
    assert panda.default_opts().graph_iters == 8
    with pytest.raises(panda.PandaError):
        panda.panda_create(0, 5, np.zeros((0, 5)), np.zeros((0, 0)), np.eye(5))
