"""The C ABI library loads, exports every symbol include/ccm.h declares, and
rejects host-detectable errors before touching the GPU (no GPU needed)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

ccm = pytest.importorskip("paper_1303_0270_gb300.ccm")


@pytest.fixture(scope="module")
def L():
    from paper_1303_0270_gb300 import build
    build.build()
    return ccm.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "ccm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ccm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
        assert name in ccm.SIGNATURES, f"binding lacks {name}"


def test_struct_layout_matches_header():
    assert ctypes.sizeof(ccm.Header) == 64
    assert ctypes.sizeof(ccm.Matrix) == 40


def test_words_for_and_status(L):
    assert ccm.words_for(1, 8, 10) == 4
    assert ccm.words_for(8192, 8192, 5) == 8192 * 8192 * 5 // 32
    assert ccm.words_for(0, 7, 3) == 0
    assert ccm.words_for(3, 3, 0) == 0 and ccm.words_for(3, 3, 65) == 0
    assert ccm.status_str(ccm.E_OVERFLOW) == "CCM_E_OVERFLOW"
    assert L.ccm_version() >= 100


def _m(rows, cols, cap=64, hdr=0x1000, words=0x2000):
    return ccm.Matrix(hdr, words, cap, rows, cols)


def test_host_side_rejections_launch_nothing(L):
    bp = ctypes.byref
    a, b, c = _m(3, 4), _m(4, 3), _m(3, 4)
    # shape mismatch
    assert L.ccm_add(bp(a), bp(b), bp(c), None, 0, None) == ccm.E_SHAPE
    # NULL header
    bad = _m(3, 4, hdr=0)
    assert L.ccm_add(bp(bad), bp(a), bp(c), None, 0, None) == ccm.E_INVAL
    # misaligned header
    assert L.ccm_scale(bp(_m(3, 4, hdr=0x1004)), 2, bp(c), None, 0, None) == ccm.E_INVAL
    # capacity below the width-1 minimum
    small = _m(30, 40, cap=4)
    assert L.ccm_scale(bp(_m(30, 40)), 2, bp(small), None, 0, None) == ccm.E_CAPACITY
    # pack: bad dtype, NULL dense, shape disagreement
    assert L.ccm_pack(ctypes.c_void_p(0x3000), 7, 3, 4, bp(c), None, 0, None) == ccm.E_INVAL
    assert L.ccm_pack(None, ccm.I64, 3, 4, bp(c), None, 0, None) == ccm.E_INVAL
    assert L.ccm_pack(ctypes.c_void_p(0x3000), ccm.I64, 4, 4, bp(c), None, 0, None) == ccm.E_SHAPE
    assert L.ccm_pack(ctypes.c_void_p(0x3000), ccm.I64, 3, 4, bp(c), ctypes.c_void_p(0x10010),
                      1 << 20, None) == ccm.E_INVAL
    # matvec: x shape, workspace size and alignment
    x, y = _m(4, 1), _m(3, 1)
    ws = ctypes.c_void_p(0x10000)
    need = L.ccm_workspace_bytes(ccm.OP_MATVEC, 3, 4, 1)
    assert L.ccm_matvec(bp(a), bp(_m(5, 1)), bp(y), ws, need, None) == ccm.E_SHAPE
    assert L.ccm_matvec(bp(a), bp(x), bp(y), ws, need - 1, None) == ccm.E_CAPACITY
    assert L.ccm_matvec(bp(a), bp(x), bp(y), ctypes.c_void_p(0x10010), need, None) == ccm.E_INVAL
    # matmul: bad path, inner dimension
    need = L.ccm_workspace_bytes(ccm.OP_MATMUL, 3, 4, 3)
    assert L.ccm_matmul(bp(a), bp(b), bp(_m(3, 3)), 9, ws, need, None) == ccm.E_INVAL
    assert L.ccm_matmul(bp(a), bp(a), bp(_m(3, 4)), 0, ws, need, None) == ccm.E_SHAPE
    # VLB matvec: NULL stream pointers, x / y shapes, workspace size and alignment
    h = ctypes.c_void_p(0x5000)
    need = L.ccm_workspace_bytes(ccm.OP_VLB_MATVEC, 3, 4, 0)
    assert need >= 3 * 8
    assert L.ccm_vlb_matvec(h, None, 8, ctypes.c_void_p(0x6000), 3, 4, bp(x), bp(y), ws, need,
                            None) == ccm.E_INVAL
    assert L.ccm_vlb_matvec(h, ctypes.c_void_p(0x7000), 8, ctypes.c_void_p(0x6000), 3, 4,
                            bp(_m(5, 1)), bp(y), ws, need, None) == ccm.E_SHAPE
    assert L.ccm_vlb_matvec(h, ctypes.c_void_p(0x7000), 8, ctypes.c_void_p(0x6000), 3, 4,
                            bp(x), bp(y), ws, need - 1, None) == ccm.E_CAPACITY
    assert L.ccm_vlb_matvec(h, ctypes.c_void_p(0x7000), 8, ctypes.c_void_p(0x6000), 3, 4,
                            bp(x), bp(y), ctypes.c_void_p(0x10010), need, None) == ccm.E_INVAL
    # generators
    assert L.ccm_gen_uniform(None, 5, 1, 0, 0, 0, 1, None) == ccm.E_INVAL
    assert L.ccm_gen_uniform(ctypes.c_void_p(0x4000), 5, 1, 0, 0, 3, 1, None) == ccm.E_INVAL
    assert L.ccm_gen_poisson(ctypes.c_void_p(0x4000), 5, 1, 0, 0, None, 3, None) == ccm.E_INVAL


def test_product_does_not_touch_the_oracle():
    """The product package never imports, loads or names the oracle."""
    pkg = os.path.join(ROOT, "paper_1303_0270_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "ccm_oracle" not in text and "ccmo_" not in text, f
