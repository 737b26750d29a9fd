"""The C-ABI library builds, loads and exports every symbol include/dcrf.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dcrf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dcrf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def library():
    from paper_1608_06192_gb300 import build
    path = build.build()
    return ctypes.CDLL(str(path))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("dcrf_lattice_build", "dcrf_filter", "dcrf_qp_fw", "dcrf_dc_cccp", "dcrf_lp_subgrad",
              "dcrf_lp_solve", "dcrf_filter_adjoint", "dcrf_features"):
        assert n in names


def test_every_declared_symbol_is_exported(library):
    missing = [n for n in _declared() if not hasattr(library, n)]
    assert not missing, missing


def test_binding_covers_the_header(library):
    from paper_1608_06192_gb300 import _abi
    assert set(_declared()) <= set(_abi.exported_symbols())


def test_status_strings_without_gpu(library):
    library.dcrf_status_string.restype = ctypes.c_char_p
    assert library.dcrf_status_string(0) == b"ok"
    assert b"hash" in library.dcrf_status_string(-4)
    # argument errors are caught on the host before any device work
    library.dcrf_lattice_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert library.dcrf_lattice_build(None, 4, 0, None, ctypes.byref(out)) == -1
    assert library.dcrf_lattice_build(None, 4, 9, None, ctypes.byref(out)) == -1
