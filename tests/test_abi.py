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


def test_subtree_masks_marshalling():
    # the binding turns a 0/1 [subtrees][labels] matrix into 64-bit label
    # masks (bit i = label i) and float32 edge lengths; shapes are checked
    import numpy as np
    from paper_1608_06192_gb300 import _abi
    members = np.zeros((3, 64))
    members[0, [0, 63]] = 1
    members[1, :] = 1
    members[2, 5] = 1
    masks, w = _abi._tree(members, [2.0, 4.0, 1.0], 64)
    assert masks.dtype == np.uint64 and w.dtype == np.float32
    assert int(masks[0]) == (1 << 63) | 1 and int(masks[1]) == (1 << 64) - 1 and int(masks[2]) == 1 << 5
    with pytest.raises(ValueError):
        _abi._tree(members[:, :10], [1.0, 1.0, 1.0], 64)
    with pytest.raises(ValueError):
        _abi._tree(members, [1.0, 1.0], 64)


def test_host_buffer_marshalling():
    # host buffers: C-contiguous float32 numpy arrays or CPU tensors of [N, cols]
    import numpy as np
    import torch
    from paper_1608_06192_gb300 import _abi
    a = np.zeros((5, 3), dtype=np.float32)
    arr, ptr = _abi._host(a, "rgb", 3)
    assert arr is a and ptr.value == a.ctypes.data
    t = torch.zeros((5, 21))
    arr, ptr = _abi._host(t, "Y0", 21)
    assert ptr.value == t.data_ptr()
    for bad in (a.astype(np.float64), np.zeros((3, 5), dtype=np.float32).T, np.zeros(5, dtype=np.float32),
                torch.zeros((5, 3), dtype=torch.float64)):
        with pytest.raises(ValueError):
            _abi._host(bad, "x", 3)
    with pytest.raises(ValueError):
        _abi._host(a, "x", 4)
