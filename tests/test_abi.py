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
    # repack: width range, shape, word alignment of the block, capacity
    y, big = _m(40, 1, cap=64), _m(100, 1, cap=64)
    assert L.ccm_repack(bp(y), 0, 0, bp(big), 0, None) == ccm.E_WIDTH
    assert L.ccm_repack(bp(y), 65, 1, bp(big), 0, None) == ccm.E_WIDTH
    assert L.ccm_repack(bp(y), 8, 2, bp(big), 0, None) == ccm.E_WIDTH
    assert L.ccm_repack(bp(y), 8, 0, bp(big), 61, None) == ccm.E_SHAPE   # 61 + 40 > 100
    assert L.ccm_repack(bp(y), 8, 0, bp(_m(100, 2, cap=64)), 0, None) == ccm.E_SHAPE
    assert L.ccm_repack(bp(y), 9, 0, bp(big), 3, None) == ccm.E_SHAPE    # 27 bits in
    assert L.ccm_repack(bp(y), 8, 0, bp(_m(100, 1, cap=24)), 0, None) == ccm.E_CAPACITY
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


def _range_width(lo, hi):
    """The width rule on an integer range, written out: unsigned
    max(1, bitlen(hi)) when lo >= 0, else the smallest two's complement
    width holding both ends."""
    if lo >= 0:
        return max(1, hi.bit_length())
    b = 1
    while not (-(1 << (b - 1)) <= lo and hi <= (1 << (b - 1)) - 1):
        b += 1
    return b


def _field_values(b, sgn):
    return range(-(1 << (b - 1)), 1 << (b - 1)) if sgn else range(0, 1 << b)


def test_bound_calls_match_brute_force(L):
    """ccm_bound_*: the smallest width holding every result that operands of
    the given widths allow, against enumeration of every operand value."""
    for ba in range(1, 6):
        for sa in (0, 1):
            va = list(_field_values(ba, sa))
            for bb in range(1, 6):
                for sb in (0, 1):
                    vb = list(_field_values(bb, sb))
                    sums = [p + q for p in va for q in vb]
                    assert L.ccm_bound_add(ba, sa, bb, sb) == _range_width(min(sums), max(sums))
                    prods = [p * q for p in va for q in vb]
                    for k in (0, 1, 2, 3, 1000):
                        # sum of k products reaches k*min and k*max (all terms equal)
                        want = 1 if k == 0 else _range_width(k * min(prods), k * max(prods))
                        assert L.ccm_bound_matvec(ba, sa, bb, sb, k) == want
                        assert L.ccm_bound_matmul(ba, sa, bb, sb, k) == want
            for s in (-33, -7, -1, 0, 1, 2, 7, 31, 1 << 20):
                sc = [s * p for p in va]
                assert L.ccm_bound_scale(ba, sa, s) == _range_width(min(sc), max(sc))


def test_bound_calls_small_exhaustive_sums(L):
    """For k = 2 the bound is attained: enumerate every pair of products."""
    for ba, sa, bb, sb in ((2, 1, 2, 0), (3, 0, 2, 1), (2, 1, 3, 1)):
        va, vb = list(_field_values(ba, sa)), list(_field_values(bb, sb))
        dots = [a0 * x0 + a1 * x1 for a0 in va for a1 in va for x0 in vb for x1 in vb]
        assert L.ccm_bound_matvec(ba, sa, bb, sb, 2) == _range_width(min(dots), max(dots))


def test_bound_calls_edges(L):
    assert L.ccm_bound_add(64, 1, 64, 1) == 64       # beyond int64: capped, overflow is reported
    assert L.ccm_bound_add(63, 1, 63, 1) == 64
    assert L.ccm_bound_add(62, 0, 62, 0) == 63
    assert L.ccm_bound_scale(64, 0, -(1 << 63)) == 64
    assert L.ccm_bound_scale(10, 1, 0) == 1
    assert L.ccm_bound_matvec(32, 1, 31, 1, 1 << 20) == 64
    assert L.ccm_bound_matvec(5, 0, 8, 1, 8192) == 26
    for bad in (0, 65, -3):
        assert L.ccm_bound_add(bad, 0, 3, 0) == ccm.E_WIDTH
        assert L.ccm_bound_scale(bad, 1, 3) == ccm.E_WIDTH
        assert L.ccm_bound_matvec(3, 0, bad, 1, 5) == ccm.E_WIDTH
        assert L.ccm_bound_matmul(bad, 0, 3, 0, 5) == ccm.E_WIDTH


def test_workspace_sizes_saturate_instead_of_wrapping(L):
    """Sizes whose byte counts would wrap uint64 come back as SIZE_MAX."""
    size_max = (1 << (8 * ctypes.sizeof(ctypes.c_size_t))) - 1
    assert L.ccm_workspace_bytes(ccm.OP_MATVEC, 1 << 61, 1, 0) == size_max
    assert L.ccm_workspace_bytes(ccm.OP_MATVEC, 1, 1 << 61, 0) == size_max
    assert L.ccm_workspace_bytes(ccm.OP_MATMUL, 1 << 40, 1 << 40, 1 << 40) == size_max
    assert L.ccm_workspace_bytes(ccm.OP_PACK, 1 << 40, 1 << 40, 16) == size_max
    assert L.ccm_workspace_bytes(ccm.OP_VLB, 1 << 40, 1 << 40, 0) == size_max
    assert L.ccm_workspace_bytes(ccm.OP_MATVEC, 1000, 1000, 1) < 1 << 20
    # shapes whose field count wraps are rejected before any launch
    bp = ctypes.byref
    huge = _m(1 << 33, 1 << 31)
    assert L.ccm_scale(bp(huge), 2, bp(_m(1 << 33, 1 << 31)), None, 0, None) == ccm.E_INVAL


STATIC_BYTES = (1 << 20) + 4096


def _static_need(rows, cols):
    up = lambda v: (v + 255) // 256 * 256  # noqa: E731
    return up(8 * cols) + up(8 * rows) + 256


def test_static_matvec_size_limit_boundary(L):
    """ccm_matvec_static: the largest A that fits the fixed scratch passes the
    size check (and then fails on a misaligned y, so nothing launches); one
    column more returns CCM_E_CAPACITY; a size that would wrap the size
    arithmetic is rejected too."""
    bp = ctypes.byref
    rows = 4
    cols = max(c for c in range(131000, 132000) if _static_need(rows, c) <= STATIC_BYTES)
    assert cols == 131520 and _static_need(rows, cols + 1) > STATIC_BYTES
    assert L.ccm_workspace_bytes(ccm.OP_MATVEC, rows, cols, 1) == _static_need(rows, cols)
    for c, want in ((cols, ccm.E_INVAL), (cols + 1, ccm.E_CAPACITY)):
        a, x = _m(rows, c, cap=1 << 20), _m(c, 1, cap=1 << 16)
        y_misaligned = _m(rows, 1, cap=16, words=0x2004)
        assert L.ccm_matvec_static(bp(a), bp(x), bp(y_misaligned), None) == want
    wrap = 1 << 61
    a, x, y = _m(wrap, 1), _m(1, 1), _m(wrap, 1)
    assert L.ccm_matvec_static(bp(a), bp(x), bp(y), None) == ccm.E_CAPACITY
