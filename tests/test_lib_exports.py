"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

from paper_2501_17529_b300 import dcflow
from paper_2501_17529_b300.csrc import build as cbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dcflow_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    cbuild.build()
    return ctypes.CDLL(cbuild.LIB)


def test_every_declared_symbol_is_exported(lib):
    decl = _declared()
    assert {"dcflow_setup", "dcflow_base_ptdf", "dcflow_set_study", "dcflow_solve_batch",
            "dcflow_destroy", "dcflow_strerror"} <= decl
    for name in sorted(decl):
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert set(dcflow.EXPORTED) == _declared()


def test_host_only_entry_points_without_gpu():
    lib = dcflow.load_library()
    assert dcflow.dcflow_strerror(0) == "ok"
    assert "not connected" in dcflow.dcflow_strerror(-2)
    o = dcflow.dcflow_default_options()
    assert o.precision == dcflow.FP32 and o.island_tol == 1e-9
    # host-side validation fails before any device work
    with pytest.raises(dcflow.DCFlowError) as e:
        dcflow.dcflow_setup(3, [0, 1], [1, 1], [1.0, 1.0], 0)  # self loop
    assert e.value.code == -1
    with pytest.raises(dcflow.DCFlowError) as e:
        dcflow.dcflow_setup(4, [0, 2], [1, 3], [1.0, 1.0], 0)  # two islands
    assert e.value.code == -2
    assert lib.dcflow_last_launch_count(None) == 0
