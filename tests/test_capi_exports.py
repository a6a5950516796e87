"""The C-ABI library builds for sm_103a, loads on a machine without a GPU, and exports every
function that include/sbp_mrab.h declares."""
import ctypes
import os
import re

from conftest import ROOT, build_library


def _declared():
    src = open(os.path.join(ROOT, "include", "sbp_mrab.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sbp[0-9a-z]*_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_header_symbols():
    path = build_library()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_1805_06607_gb300 as sbp
    assert set(_declared()) == set(sbp.exported_symbols())


def test_status_strings_without_gpu():
    import paper_1805_06607_gb300 as sbp
    L = sbp.lib()
    assert L.sbp_status_string(0) == b"ok"
    assert L.sbp_status_string(-6) == b"no donor"
