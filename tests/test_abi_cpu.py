"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/exx.h declares.  No compute calls: this runs without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2011_07209_gb300 import build, exx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "exx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(exx_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return exx.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(exx.EXPORTS) <= set(names)


def test_error_strings_and_version(lib):
    assert b"sm_103a" in lib.exx_version()
    for code in range(10):
        assert lib.exx_error_string(code)
    assert lib.exx_error_string(99) == b"unknown error"


def test_dbox_halfwidth_host_only(lib):
    import numpy as np
    p = exx.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0)
    hw = exx.dbox_halfwidth(np.diag([23.5] * 3), (120, 120, 120), p)
    # ceil((4 + 8) * 120 / 23.5) + 1
    assert list(hw) == [63, 63, 63]


def test_null_arguments_rejected(lib):
    assert lib.exx_ctx_create(None, 0) == exx.ERR_ARG
    assert lib.exx_plan_create(None, None, None, 0, None, None) == exx.ERR_ARG
    assert lib.exx_pairs_solve(None, None, None, None, None, None) == exx.ERR_ARG
    assert lib.exx_plan_query(None, None) == exx.ERR_ARG
