"""The C ABI library loads without a GPU and exports every function include/mw.h declares."""
import os
import re

import pytest

from paper_2311_05322_gb300 import mw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    if not os.path.exists(mw.LIB_PATH):
        from paper_2311_05322_gb300 import build
        build.build()


def _declared():
    text = open(os.path.join(ROOT, "include", "mw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(mw_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_functions_are_exported_and_bound():
    lib = mw.load_library()
    declared = _declared()
    assert len(declared) >= 30
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(mw.exported_symbols()), declared ^ set(mw.exported_symbols())


def test_no_device_needed_to_load():
    # loading and querying a pure function must work on a machine without a GPU
    assert mw.load_library().mw_nn_param_count(8192) == 1024 * 8192 + 1024 + 1024 * 1024 + 1024 + \
        16 * 16 * 64 + 16 + 16 * 8 * 64 + 8 + 8 * 2 * 64 + 2
