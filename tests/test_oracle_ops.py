"""Pins of the oracle's operations on the compressed form.

Expected values come from Python's arbitrary-precision integers written as
textbook loops (sum over j of a_ij x_j, and so on), from special cases with a
known answer (scale by 0, 1 and -1, A + (-A), identity and one-hot operands)
and from the mathematical invariant that an operation on the compressed form
equals the operation on the uncompressed integers (Introduction), i.e.
unpack(op(pack A)) == op(A).  Shapes are non-square so that a transposed
operand or a swapped index fails.
"""
import numpy as np
import pytest

import oracle


def _rand(rng, shape, b):
    lo, hi = -(1 << (b - 1)), (1 << (b - 1)) - 1
    return rng.integers(lo, hi, size=shape, dtype=np.int64, endpoint=True)


def _py_matmul(a, b):
    a, b = a.tolist(), b.tolist()
    m, k, n = len(a), len(b), len(b[0])
    return [[sum(a[i][l] * b[l][j] for l in range(k)) for j in range(n)] for i in range(m)]


def _expect_packed(p, values):
    values = np.asarray(values, dtype=object)
    flat = [int(v) for v in values.ravel()]
    assert np.array_equal(oracle.unpack(p).ravel(), np.array(flat, dtype=np.int64))
    # canonical width: the smallest that holds every entry of the result
    signed = any(v < 0 for v in flat)
    b = 1
    while not all(((-(1 << (b - 1)) <= v < (1 << (b - 1))) if signed else (0 <= v < (1 << b)))
                  for v in flat):
        b += 1
    assert (p.width, p.is_signed) == (b, int(signed))


@pytest.mark.parametrize("shape", [(1, 1), (3, 7), (17, 33), (64, 5)])
@pytest.mark.parametrize("ba,bb", [(1, 1), (5, 8), (8, 8), (13, 3), (31, 32), (62, 62)])
def test_add(shape, ba, bb):
    rng = np.random.default_rng(ba * 100 + bb + shape[0])
    a, b = _rand(rng, shape, ba), _rand(rng, shape, bb)
    c = oracle.add(oracle.pack(a), oracle.pack(b))
    _expect_packed(c, [[int(x) + int(y) for x, y in zip(ra, rb)] for ra, rb in zip(a, b)])


def test_add_inverse_is_zero():
    rng = np.random.default_rng(1)
    a = _rand(rng, (9, 10), 12)
    c = oracle.add(oracle.pack(a), oracle.pack(-a))
    assert (c.width, c.is_signed) == (1, 0) and not c.words.any()


def test_add_overflow():
    a = np.array([[(1 << 63) - 1]], dtype=np.int64)
    with pytest.raises(OverflowError):
        oracle.add(oracle.pack(a), oracle.pack(np.array([[1]])))


@pytest.mark.parametrize("s", [0, 1, -1, 7, -3, 1 << 20, -(1 << 30) + 5])
@pytest.mark.parametrize("b", [1, 4, 8, 20])
def test_scale(s, b):
    rng = np.random.default_rng(b + 11)
    a = _rand(rng, (11, 6), b)
    pa = oracle.pack(a)
    c = oracle.scale(pa, s)
    _expect_packed(c, [[int(v) * s for v in row] for row in a])
    if s == 0:
        assert (c.width, c.is_signed) == (1, 0) and not c.words.any()
    if s == 1:
        assert c.width == pa.width and np.array_equal(c.words, pa.words)


def test_scale_overflow():
    with pytest.raises(OverflowError):
        oracle.scale(oracle.pack(np.array([[1 << 40]])), 1 << 23)
    # exactly at the int64 limits is fine
    c = oracle.scale(oracle.pack(np.array([[-(1 << 62)]])), 2)
    assert oracle.unpack(c)[0, 0] == -(1 << 63) and c.width == 64


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (3, 5), (31, 33), (64, 130)])
@pytest.mark.parametrize("ba,bx", [(1, 1), (5, 8), (8, 8), (16, 8), (32, 8), (24, 24)])
def test_matvec(m, n, ba, bx):
    rng = np.random.default_rng(m * 7 + n + ba)
    a, x = _rand(rng, (m, n), ba), _rand(rng, n, bx)
    y = oracle.matvec(oracle.pack(a), oracle.pack(x.reshape(n, 1)))
    assert (y.rows, y.cols) == (m, 1)
    _expect_packed(y, [sum(int(a[i, j]) * int(x[j]) for j in range(n)) for i in range(m)])


def test_matvec_one_hot_selects_column():
    rng = np.random.default_rng(5)
    a = _rand(rng, (13, 9), 10)
    for j in range(9):
        x = np.zeros(9, dtype=np.int64)
        x[j] = 1
        y = oracle.matvec(oracle.pack(a), oracle.pack(x.reshape(9, 1)))
        assert np.array_equal(oracle.unpack(y).ravel(), a[:, j])


def test_matvec_rows_subset_and_overflow():
    rng = np.random.default_rng(9)
    a, x = _rand(rng, (20, 30), 30), _rand(rng, 30, 30)
    rows = [19, 0, 7]
    ys = oracle.matvec_dense(a, x, rows=rows)
    assert [int(v) for v in ys] == [sum(int(a[i, j]) * int(x[j]) for j in range(30)) for i in rows]
    big = np.full((1, 4), (1 << 62), dtype=np.int64)
    with pytest.raises(OverflowError):
        oracle.matvec_dense(big, np.array([1, 1, 0, 0]))


@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (2, 3, 4), (5, 1, 3), (9, 17, 6), (33, 40, 31)])
@pytest.mark.parametrize("b", [1, 4, 8, 12, 16])
def test_matmul(m, k, n, b):
    rng = np.random.default_rng(m * 100 + k * 10 + n + b)
    a, bm = _rand(rng, (m, k), b), _rand(rng, (k, n), b)
    c = oracle.matmul(oracle.pack(a), oracle.pack(bm))
    assert (c.rows, c.cols) == (m, n)
    _expect_packed(c, _py_matmul(a, bm))


def test_matmul_identity_and_rows():
    rng = np.random.default_rng(2)
    a = _rand(rng, (7, 7), 9)
    eye = np.eye(7, dtype=np.int64)
    pe = oracle.pack(eye)
    assert (pe.width, pe.is_signed) == (1, 0)
    assert np.array_equal(oracle.unpack(oracle.matmul(pe, oracle.pack(a))), a)
    assert np.array_equal(oracle.unpack(oracle.matmul(oracle.pack(a), pe)), a)
    b = _rand(rng, (7, 5), 9)
    full = np.array(_py_matmul(a, b), dtype=np.int64)
    assert np.array_equal(oracle.matmul_dense(a, b, rows=[6, 2]), full[[6, 2]])


def test_get_flat_matches_unpack():
    rng = np.random.default_rng(4)
    a = _rand(rng, (6, 9), 7)
    p = oracle.pack(a)
    idx = [0, 53, 17, 8, 9]
    assert oracle.get_flat(p, idx).tolist() == [int(a.ravel()[e]) for e in idx]


@pytest.mark.parametrize("m,n1,n2", [(1, 1, 1), (3, 5, 2), (7, 4, 9), (5, 0, 3)])
def test_matvec2_textbook(m, n1, n2):
    """y_i = sum_j a_ij x_j + sum_j b_ij z_j with Python integers."""
    rng = np.random.default_rng(m * 100 + n1 * 10 + n2)
    a, b = _rand(rng, (m, n1), 9), _rand(rng, (m, n2), 13)
    x, z = _rand(rng, (n1, 1), 7), _rand(rng, (n2, 1), 5)
    want = [sum(int(a[i, j]) * int(x[j, 0]) for j in range(n1)) +
            sum(int(b[i, j]) * int(z[j, 0]) for j in range(n2)) for i in range(m)]
    got = oracle.matvec2(oracle.pack(a, m, n1), oracle.pack(x, n1, 1), oracle.pack(b, m, n2),
                         oracle.pack(z, n2, 1))
    _expect_packed(got, np.array(want).reshape(m, 1))


def test_matvec2_overflow_of_the_sum():
    """Each product fits int64, their sum does not."""
    a = np.array([[1 << 62]], dtype=np.int64)
    x = np.array([[1]], dtype=np.int64)
    with pytest.raises(OverflowError):
        oracle.matvec2(oracle.pack(a), oracle.pack(x), oracle.pack(a), oracle.pack(x))
    neg = oracle.matvec2(oracle.pack(a), oracle.pack(x), oracle.pack(-a), oracle.pack(x))
    _expect_packed(neg, np.zeros((1, 1), dtype=np.int64))


def test_matvec_chain_associates():
    """A (B x) == (A B) x exactly, and both equal the textbook loops."""
    rng = np.random.default_rng(11)
    a, b, x = _rand(rng, (4, 6), 8), _rand(rng, (6, 3), 8), _rand(rng, (3, 1), 8)
    want = np.array(_py_matmul(a, np.array(_py_matmul(b, x), dtype=object)), dtype=object)
    chain = oracle.matvec_chain(oracle.pack(a), oracle.pack(b), oracle.pack(x))
    _expect_packed(chain, want)
    ab_x = oracle.matvec(oracle.matmul(oracle.pack(a), oracle.pack(b)), oracle.pack(x))
    assert (ab_x.width, ab_x.is_signed) == (chain.width, chain.is_signed)
    assert np.array_equal(ab_x.words, chain.words)


@pytest.mark.parametrize("m,k,n,b", [(1, 1, 1, 1), (9, 17, 6, 8), (33, 40, 31, 16), (5, 300, 7, 20)])
def test_matmul_f64_textbook(m, k, n, b):
    """The float64-BLAS product equals textbook Python-integer loops."""
    rng = np.random.default_rng(7 * m + k + n + b)
    a, bm = _rand(rng, (m, k), b), _rand(rng, (k, n), b)
    assert np.array_equal(oracle.matmul_dense_f64(a, bm),
                          np.array(_py_matmul(a, bm), dtype=np.int64))


def test_matmul_f64_near_its_exactness_limit():
    """Sums just below 2^53 in magnitude, reached through partial sums of
    both signs, stay exact; at the limit the function refuses."""
    k = 8
    big = (1 << 22) - 1  # |a| * |b| * k = (2^22-1)^2 * 8 < 2^47
    a = np.full((3, k), big, dtype=np.int64)
    a[1, ::2] = -big
    b = np.full((k, 2), big, dtype=np.int64)
    assert np.array_equal(oracle.matmul_dense_f64(a, b), np.array(_py_matmul(a, b), dtype=np.int64))
    x = (1 << 24) + 1  # odd, so products need every bit
    a2 = np.array([[x, -x, x]], dtype=np.int64)
    b2 = np.array([[x], [x], [x + 2]], dtype=np.int64)
    assert int(oracle.matmul_dense_f64(a2, b2)[0, 0]) == x * x - x * x + x * (x + 2)
    with pytest.raises(ValueError):
        oracle.matmul_dense_f64(np.full((1, 2), 1 << 26, dtype=np.int64),
                                np.full((2, 1), 1 << 26, dtype=np.int64))
