"""Pins of the oracle's SM format against the paper and against brute force.

The oracle is not compared with itself here: the expected values come from the
paper's printed worked example (Eq. 3, Table 1), from the definition of the
width as "the smallest b whose range holds every entry" searched by brute
force, and from an independent construction of the bit stream as a string of
binary digits written right to left, as the paper draws it.
"""
import itertools

import numpy as np
import pytest

import oracle
from conftest import golden_lines


def _golden(name):
    d = {}
    for ln in golden_lines(name):
        k, *v = ln.split()
        d[k] = v
    return d


def _words64(p):
    w = p.words.astype(np.uint64)
    if w.size % 2:
        w = np.append(w, np.uint64(0))
    return [int(w[2 * i]) | (int(w[2 * i + 1]) << 32) for i in range(w.size // 2)]


def test_eq3_worked_example_words():
    g = _golden("sm_example_eq3.txt")
    entries = [int(v) for v in g["entries"]]
    b = int(g["width"][0])
    p = oracle.pack(np.array(entries, dtype=np.int64).reshape(1, -1))
    assert (p.width, p.is_signed) == (b, 0)
    words = _words64(p)
    # bitstring_1: the printed six fields, topped by segment a of element 700
    six = g["bitstring1_six"][0]
    assert six.startswith("0000") and len(six) == 64
    bitstring1 = int(g["segment_a"][0] + six[4:], 2)
    bitstring2 = int(g["field_20"][0] + g["segment_b"][0], 2)
    assert words[0] == bitstring1
    assert words[1] == bitstring2
    assert all(w == 0 for w in words[2:])
    # 80 bits used: three 32-bit data words, padded to four
    assert p.words.size == 4 and int(p.words[3]) == 0


def test_eq3_intermediate_bitstring_after_six_fields():
    g = _golden("sm_example_eq3.txt")
    entries = [int(v) for v in g["entries"]][:6]
    p = oracle.pack_at(np.array(entries), 1, 6, 10, 0)
    assert _words64(p)[0] == int(g["bitstring1_six"][0], 2)


def test_table1_bit_lengths():
    for ln in golden_lines("table1_bitlengths.txt"):
        value, binary, length = ln.split()
        assert int(binary, 2) == int(value)
        assert oracle.bitlen(int(value)) == int(length)


def test_eq1_special_cases():
    # b = 1 when sup M is 0 or 1 (Eq. 1, first case)
    assert oracle.width([0]) == (1, 0)
    assert oracle.width([0, 1, 1, 0]) == (1, 0)
    assert oracle.width([1]) == (1, 0)
    # floor(log2 sup M) + 1 otherwise
    assert oracle.width([2]) == (2, 0)
    assert oracle.width([1023, 5]) == (10, 0)
    assert oracle.width([1024]) == (11, 0)
    assert oracle.width([(1 << 63) - 1]) == (63, 0)


def _brute_width(values):
    """Smallest b (1..64) whose unsigned or two's complement range holds every entry."""
    signed = any(v < 0 for v in values)
    for b in range(1, 65):
        lo, hi = (-(1 << (b - 1)), (1 << (b - 1)) - 1) if signed else (0, (1 << b) - 1)
        if all(lo <= v <= hi for v in values):
            return b, int(signed)
    raise AssertionError


@pytest.mark.parametrize("b", range(1, 65))
def test_width_signed_endpoints(b):
    lo, hi = -(1 << (b - 1)), (1 << (b - 1)) - 1
    assert oracle.width([lo, hi]) == (b, 1)
    assert oracle.width([lo]) == (b, 1)
    if b < 64:
        assert oracle.width([lo - 1]) == (b + 1, 1)
        assert oracle.width([hi + 1, -1]) == (b + 1, 1)


@pytest.mark.parametrize("b", range(1, 64))
def test_width_unsigned_endpoints(b):
    assert oracle.width([(1 << b) - 1]) == (b, 0)
    if b < 63:
        assert oracle.width([1 << b]) == (b + 1, 0)


def test_width_matches_brute_force_random():
    rng = np.random.default_rng(7)
    for _ in range(400):
        b = int(rng.integers(1, 64))
        n = int(rng.integers(1, 9))
        vals = [int(v) for v in rng.integers(-(1 << (b - 1)), 1 << (b - 1), size=n)]
        if rng.random() < 0.5:
            vals = [abs(v) for v in vals]
        assert oracle.width(vals) == _brute_width(vals)


def _string_stream(values, b):
    """The stream as the paper draws it: each field's b binary digits, written
    right to left, element 0 at the right end; then cut into 32-bit words."""
    s = ""
    for v in values:
        s = format(v & ((1 << b) - 1), f"0{b}b") + s
    total = int(s, 2) if s else 0
    nbits = len(values) * b
    nwords = oracle.words_for(len(values), b)
    assert nbits <= nwords * 32
    return [(total >> (32 * i)) & 0xFFFFFFFF for i in range(nwords)]


@pytest.mark.parametrize("b", range(1, 13))
def test_pack_unpack_brute_force_small(b):
    """All matrices of tiny size whose b*n <= 12, both sign modes."""
    n_max = max(1, 12 // b)
    for n in range(1, n_max + 1):
        for signed in (0, 1):
            lo, hi = (-(1 << (b - 1)), (1 << (b - 1)) - 1) if signed else (0, (1 << b) - 1)
            span = hi - lo + 1
            for combo in itertools.product(range(span), repeat=n):
                vals = [lo + c for c in combo]
                p = oracle.pack_at(np.array(vals), 1, n, b, signed)
                assert [int(w) for w in p.words] == _string_stream(vals, b)
                assert oracle.unpack(p).ravel().tolist() == vals


@pytest.mark.parametrize("shape", [(1, 1), (1, 31), (3, 33), (7, 13), (32, 32), (33, 65)])
@pytest.mark.parametrize("b", [1, 2, 3, 5, 7, 8, 9, 13, 16, 17, 24, 31, 32, 33, 40, 47, 63, 64])
def test_round_trip_random_shapes(shape, b):
    rng = np.random.default_rng(b * 1000 + shape[0] * 37 + shape[1])
    rows, cols = shape
    for signed in (0, 1):
        if not signed and b == 64:
            continue
        lo, hi = (-(1 << (b - 1)), (1 << (b - 1)) - 1) if signed else (0, (1 << b) - 1)
        vals = rng.integers(lo, hi, size=rows * cols, dtype=np.int64, endpoint=True)
        vals[0] = lo
        vals[-1] = hi
        p = oracle.pack_at(vals, rows, cols, b, signed)
        assert [int(w) for w in p.words] == _string_stream([int(v) for v in vals], b)
        assert np.array_equal(oracle.unpack(p).ravel(), vals)
        # padding words beyond ceil(n*b/32) are zero, and so are the bits above the last field
        nbits = rows * cols * b
        tail = [int(w) for w in p.words]
        full = sum(w << (32 * i) for i, w in enumerate(tail))
        assert full >> nbits == 0


def test_pack_exact_width_and_padding():
    p = oracle.pack(np.zeros((5, 7), dtype=np.int64))
    assert (p.width, p.is_signed) == (1, 0)
    assert np.all(p.words == 0) and p.words.size == 4
    p = oracle.pack(-np.ones((3, 3), dtype=np.int64))
    assert (p.width, p.is_signed) == (1, 1)
    assert int(p.words[0]) == (1 << 9) - 1


def test_get_by_row_and_column():
    rng = np.random.default_rng(3)
    a = rng.integers(-500, 500, size=(9, 11))
    p = oracle.pack(a)
    for i in range(9):
        for j in range(11):
            assert oracle.get(p, i, j) == a[i, j]
    with pytest.raises(IndexError):
        oracle.get(p, 9, 0)
    with pytest.raises(IndexError):
        oracle.get(p, 0, 11)


def test_words_for_rule():
    # ceil(n*b/32) data words padded to a multiple of 4
    assert oracle.words_for(8, 10) == 4
    assert oracle.words_for(32, 1) == 4
    assert oracle.words_for(129, 1) == 8
    assert oracle.words_for(0, 5) == 0
    assert oracle.words_for(64 * 8192, 64) == 64 * 8192 * 2
