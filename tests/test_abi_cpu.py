"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/bfm.h declares; host-side argument checks."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bfm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bfm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1807_01751_gb300 as bfm
    return bfm.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "bfm_monitor" in names and "bfm_design_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_limits(lib):
    import paper_1807_01751_gb300 as bfm
    assert "sm_103a" in bfm.bfm_version()
    assert bfm.bfm_max_dates() >= 600


def test_design_argument_errors_before_any_cuda_call(lib):
    import paper_1807_01751_gb300 as bfm
    d = np.arange(1, 51, dtype=np.float64)
    for args, code in [((d[::-1].copy(), 3, 23.0), 1), ((d, 0, 23.0), 1), ((d, 3, -1.0), 1),
                       ((d[:1], 3, 23.0), 1), ((np.arange(1, 5000.0), 3, 23.0), 6)]:
        with pytest.raises(bfm.BfmError) as ei:
            bfm.bfm_design_create(*args)
        assert ei.value.code == code


def test_null_handle_is_rejected(lib):
    import paper_1807_01751_gb300 as bfm
    rc = lib.bfm_monitor(None, None, 0, None, 10, 5, 0.25, 1.7, None, None, None, None, None, None)
    assert rc == 1 and "NULL" in bfm.bfm_last_error()
