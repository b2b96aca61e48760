"""The C ABI library loads, exports every entry point of include/csrc.h, and rejects
bad input on the host before anything reaches a GPU (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cs():
    from paper_1003_0952_gb300 import build

    build.build()
    import paper_1003_0952_gb300 as m

    return m


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_][a-z_0-9]*\s*\**\s*(csrc_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("csrc_create_from_csr", "csrc_create_from_coo", "csrc_partition", "csrc_color", "csrc_spmv",
                 "csrc_spmv_t", "csrc_spmm_batched", "csrc_destroy", "csrc_get_last_device_error",
                 "csrc_status_string"):
        assert want in names


def test_library_exports_every_declared_symbol(cs):
    lib = ctypes.CDLL(cs.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in cs.SIGNATURES, f"binding lacks {name}"


def test_status_strings(cs):
    for st in range(0, 19):
        s = cs.csrc_status_string(st)
        assert s and s != "unknown status"
    assert cs.csrc_status_string(99) == "unknown status"


def _create_status(cs, n, rp, col, val, flags=0, storage=0):
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    st = cs.lib().csrc_create_from_csr(ctypes.byref(h), n, rp.ctypes.data, col.ctypes.data, val.ctypes.data, storage,
                                       flags, None)
    return st, h


def test_host_validation_errors(cs):
    # a_01 without a_10
    st, h = _create_status(cs, 2, [0, 2, 3], [0, 1, 1], [1, 2, 3])
    assert st == cs.CSRC_ERR_NOT_STRUCT_SYMMETRIC and not h.value
    # unsorted / duplicate columns
    st, _ = _create_status(cs, 2, [0, 2, 4], [1, 0, 0, 1], np.ones(4))
    assert st == cs.CSRC_ERR_DUPLICATE
    st, _ = _create_status(cs, 2, [0, 2, 3], [0, 0, 1], np.ones(3))
    assert st == cs.CSRC_ERR_DUPLICATE
    # column out of range
    st, _ = _create_status(cs, 2, [0, 1, 2], [0, 7], np.ones(2))
    assert st == cs.CSRC_ERR_INDEX_RANGE
    # bad row pointer, storage and flags
    st, _ = _create_status(cs, 2, [1, 1, 2], [0, 1], np.ones(2))
    assert st == cs.CSRC_ERR_INVALID_ARG
    st, _ = _create_status(cs, 1, [0, 1], [0], [1.0], storage=7)
    assert st == cs.CSRC_ERR_INVALID_ARG
    st, _ = _create_status(cs, 1, [0, 1], [0], [1.0], flags=1 << 10)
    assert st == cs.CSRC_ERR_INVALID_ARG
    # symmetric-value storage requested for a matrix with a_01 != a_10
    st, h = _create_status(cs, 2, [0, 2, 4], [0, 1, 0, 1], [1.0, 2.0, 3.0, 1.0], flags=cs.CSRC_FLAG_SYMMETRIC_VALUES)
    assert st == cs.CSRC_ERR_NOT_NUM_SYMMETRIC and not h.value
    # rectangular creation: fewer columns than rows, and a column past m
    rp = np.array([0, 1, 3], np.int64)
    col = np.array([0, 1, 2], np.int32)
    val = np.ones(3)
    h = ctypes.c_void_p()
    st = cs.lib().csrc_create_rect_from_csr(ctypes.byref(h), 2, 1, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                            0, 0, None)
    assert st == cs.CSRC_ERR_INVALID_ARG and not h.value
    st = cs.lib().csrc_create_rect_from_csr(ctypes.byref(h), 2, 2, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                            0, 0, None)
    assert st == cs.CSRC_ERR_INDEX_RANGE and not h.value
    # null handles and arguments
    assert cs.lib().csrc_spmv(None, None, None, 0, None) == cs.CSRC_ERR_INVALID_ARG
    assert cs.lib().csrc_partition(None, 4, None) == cs.CSRC_ERR_INVALID_ARG
    assert cs.lib().csrc_color(None, 0, None, None) == cs.CSRC_ERR_INVALID_ARG
    assert cs.lib().csrc_get_info(None, None) == cs.CSRC_ERR_INVALID_ARG
    assert cs.lib().csrc_destroy(None) == cs.CSRC_OK


def test_coo_index_range(cs):
    h = ctypes.c_void_p()
    r = np.array([0, 5], np.int32)
    c = np.array([0, 0], np.int32)
    v = np.ones(2)
    st = cs.lib().csrc_create_from_coo(ctypes.byref(h), 2, 2, r.ctypes.data, c.ctypes.data, v.ctypes.data, 0, 0, None)
    assert st == cs.CSRC_ERR_INDEX_RANGE


def test_product_path_has_no_oracle_dependency():
    # the package must not import or load anything from oracle/
    pkg = os.path.join(ROOT, "paper_1003_0952_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("no oracle", ""), f
