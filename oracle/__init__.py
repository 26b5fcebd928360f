"""CPU oracle for SM-compressed integer matrices -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package imports nothing from the product package: the two share no code.

The arithmetic lives in ``ccm_oracle.c`` (plain C, bit by bit, compiled with
gcc by :func:`build`).  This wrapper only moves numpy arrays in and out and
composes the documented steps: an operation on compressed matrices is the same
operation on the unpacked integers (Introduction), re-packed with the width
rule of Eq. 1 (Methods, Method 1) extended to two's complement.

Every function below is pinned by ``tests/test_oracle_*.py`` against the
paper's worked example (Eq. 3, Table 1), closed forms, brute force over small
inputs and textbook Python-integer arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libccm_oracle.so")

OK = 0
OVERFLOW = -4
RANGE = -6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no machine-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u64, i64, i32, sz = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        vp = ctypes.c_void_p
        L.ccmo_bitlen_u64.argtypes = [u64]
        L.ccmo_bitlen_u64.restype = i32
        L.ccmo_width.argtypes = [vp, sz, ctypes.POINTER(ctypes.c_int)]
        L.ccmo_width.restype = i32
        L.ccmo_words_for.argtypes = [u64, i32]
        L.ccmo_words_for.restype = sz
        L.ccmo_pack.argtypes = [vp, sz, i32, vp, sz]
        L.ccmo_pack.restype = None
        L.ccmo_field.argtypes = [vp, u64, i32, i32]
        L.ccmo_field.restype = i64
        L.ccmo_unpack.argtypes = [vp, sz, i32, i32, vp]
        L.ccmo_unpack.restype = None
        L.ccmo_get.argtypes = [vp, u64, u64, i32, i32, u64, u64, ctypes.POINTER(ctypes.c_int64)]
        L.ccmo_get.restype = i32
        L.ccmo_add.argtypes = [vp, vp, sz, vp]
        L.ccmo_add.restype = i32
        L.ccmo_scale.argtypes = [vp, sz, i64, vp]
        L.ccmo_scale.restype = i32
        L.ccmo_matvec_rows.argtypes = [vp, u64, u64, vp, vp, sz, vp]
        L.ccmo_matvec_rows.restype = i32
        L.ccmo_matmul_rows.argtypes = [vp, vp, u64, u64, u64, vp, sz, vp]
        L.ccmo_matmul_rows.restype = i32
        L.ccmo_vlb_prefix_width.argtypes = [vp, sz]
        L.ccmo_vlb_prefix_width.restype = i32
        L.ccmo_vlb_bits.argtypes = [vp, sz, i32]
        L.ccmo_vlb_bits.restype = u64
        L.ccmo_vlb_pack.argtypes = [vp, sz, i32, vp, sz]
        L.ccmo_vlb_pack.restype = u64
        L.ccmo_vlb_unpack.argtypes = [vp, sz, i32, vp]
        L.ccmo_vlb_unpack.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.int64)


@dataclass
class Packed:
    """A matrix in SM form: shape, field width, sign mode and the word stream."""

    rows: int
    cols: int
    width: int
    is_signed: int
    words: np.ndarray  # uint32, zero padded to a multiple of 4 words

    @property
    def n(self) -> int:
        return self.rows * self.cols


def bitlen(v: int) -> int:
    return lib().ccmo_bitlen_u64(int(v))


def width(values) -> tuple[int, int]:
    """(b, is_signed) of a set of integers (Eq. 1, two's complement when negative)."""
    a = _i64(values).ravel()
    s = ctypes.c_int(0)
    b = lib().ccmo_width(_ptr(a), a.size, ctypes.byref(s))
    return b, s.value


def words_for(n: int, b: int) -> int:
    return lib().ccmo_words_for(int(n), int(b))


def pack_at(values, rows: int, cols: int, b: int, is_signed: int) -> Packed:
    """Pack at a given width (the caller guarantees every entry fits)."""
    a = _i64(values).ravel()
    assert a.size == rows * cols
    nw = words_for(a.size, b)
    words = np.zeros(nw, dtype=np.uint32)
    lib().ccmo_pack(_ptr(a), a.size, b, _ptr(words), nw)
    return Packed(rows, cols, b, is_signed, words)


def pack(values, rows: int | None = None, cols: int | None = None) -> Packed:
    """SM compression of an integer matrix (Methods, Method 1)."""
    arr = np.asarray(values)
    if rows is None:
        if arr.ndim == 1:
            rows, cols = arr.shape[0], 1
        else:
            rows, cols = arr.shape
    b, s = width(arr)
    return pack_at(arr, rows, cols, b, s)


def unpack(p: Packed) -> np.ndarray:
    out = np.empty(p.n, dtype=np.int64)
    lib().ccmo_unpack(_ptr(p.words), p.n, p.width, p.is_signed, _ptr(out))
    return out.reshape(p.rows, p.cols)


def field(p: Packed, e: int) -> int:
    return int(lib().ccmo_field(_ptr(p.words), int(e), p.width, p.is_signed))


def get(p: Packed, i: int, j: int) -> int:
    out = ctypes.c_int64(0)
    st = lib().ccmo_get(_ptr(p.words), p.rows, p.cols, p.width, p.is_signed, int(i), int(j),
                        ctypes.byref(out))
    if st != OK:
        raise IndexError((i, j))
    return int(out.value)


def get_flat(p: Packed, idx) -> np.ndarray:
    """Entries at flat row-major indices i*cols + j."""
    idx = np.asarray(idx, dtype=np.uint64).ravel()
    return np.array([get(p, int(e) // p.cols, int(e) % p.cols) for e in idx], dtype=np.int64)


def _check(status: int):
    if status == OVERFLOW:
        raise OverflowError("result does not fit int64")
    if status != OK:
        raise RuntimeError(f"oracle status {status}")


def add_dense(a, b) -> np.ndarray:
    a, b = _i64(a), _i64(b)
    assert a.shape == b.shape
    c = np.empty_like(a)
    _check(lib().ccmo_add(_ptr(a), _ptr(b), a.size, _ptr(c)))
    return c


def scale_dense(a, s: int) -> np.ndarray:
    a = _i64(a)
    c = np.empty_like(a)
    _check(lib().ccmo_scale(_ptr(a), a.size, int(s), _ptr(c)))
    return c


def matvec_dense(a, x, rows=None) -> np.ndarray:
    a, x = _i64(a), _i64(x).ravel()
    m, n = a.shape
    assert x.size == n
    if rows is None:
        y = np.empty(m, dtype=np.int64)
        _check(lib().ccmo_matvec_rows(_ptr(a), m, n, _ptr(x), None, 0, _ptr(y)))
    else:
        rl = np.ascontiguousarray(rows, dtype=np.uint64)
        y = np.empty(rl.size, dtype=np.int64)
        _check(lib().ccmo_matvec_rows(_ptr(a), m, n, _ptr(x), _ptr(rl), rl.size, _ptr(y)))
    return y


def matmul_dense(a, b, rows=None) -> np.ndarray:
    a, b = _i64(a), _i64(b)
    m, k = a.shape
    k2, n = b.shape
    assert k == k2
    if rows is None:
        c = np.empty((m, n), dtype=np.int64)
        _check(lib().ccmo_matmul_rows(_ptr(a), _ptr(b), m, k, n, None, 0, _ptr(c)))
    else:
        rl = np.ascontiguousarray(rows, dtype=np.uint64)
        c = np.empty((rl.size, n), dtype=np.int64)
        _check(lib().ccmo_matmul_rows(_ptr(a), _ptr(b), m, k, n, _ptr(rl), rl.size, _ptr(c)))
    return c


def matmul_dense_f64(a, b) -> np.ndarray:
    """The same integer product C = A B (Introduction: the compressed form
    supports the same mathematics), with a float64 BLAS matrix product as the
    one library step.  Exact when max|a| * max|b| * k < 2^53: every product
    and every partial sum, in whatever order the library adds them, is then
    an integer that float64 represents exactly.  Raises ValueError outside
    that range (use matmul_dense there)."""
    a, b = _i64(a), _i64(b)
    m, k = a.shape
    k2, n = b.shape
    assert k == k2
    ma = int(np.abs(a).max()) if a.size else 0
    mb = int(np.abs(b).max()) if b.size else 0
    if ma * mb * max(k, 1) >= 1 << 53:
        raise ValueError("float64 product not exact for these magnitudes")
    c = np.matmul(a.astype(np.float64), b.astype(np.float64))
    return c.astype(np.int64)


# Operations on the compressed form: unpack, operate, re-pack at the new width.
def add(pa: Packed, pb: Packed) -> Packed:
    assert (pa.rows, pa.cols) == (pb.rows, pb.cols)
    return pack(add_dense(unpack(pa), unpack(pb)))


def scale(pa: Packed, s: int) -> Packed:
    return pack(scale_dense(unpack(pa), s))


def matvec(pa: Packed, px: Packed) -> Packed:
    assert px.n == pa.cols
    y = matvec_dense(unpack(pa), unpack(px).ravel())
    return pack(y.reshape(pa.rows, 1))


def matmul(pa: Packed, pb: Packed) -> Packed:
    assert pa.cols == pb.rows
    return pack(matmul_dense(unpack(pa), unpack(pb)))


# Chains that stay compressed: the same integers as the chain on the
# uncompressed operands (Introduction), re-packed once at the end.
def matvec2(pa: Packed, px: Packed, pb: Packed, pz: Packed) -> Packed:
    """y = A x + B z (int64 overflow of the sum raises, as in add_dense)."""
    assert pa.rows == pb.rows and px.n == pa.cols and pz.n == pb.cols
    ya = matvec_dense(unpack(pa), unpack(px).ravel())
    yb = matvec_dense(unpack(pb), unpack(pz).ravel())
    return pack(add_dense(ya, yb).reshape(pa.rows, 1))


def matvec_chain(pa: Packed, pb: Packed, px: Packed) -> Packed:
    """y = A (B x), the intermediate B x packed at its own width."""
    return matvec(pa, matvec(pb, px))


# VLB, Method 2: a k-bit length prefix then the entry in its own bit length.
@dataclass
class Vlb:
    n: int
    k: int
    nbits: int
    words: np.ndarray  # uint32, zero padded to a multiple of 4 words


def vlb_pack(values) -> Vlb:
    a = _i64(values).ravel()
    k = lib().ccmo_vlb_prefix_width(_ptr(a), a.size)
    if k < 0:
        raise ValueError("VLB takes non-negative entries")
    nbits = int(lib().ccmo_vlb_bits(_ptr(a), a.size, k))
    nw = ((nbits + 31) // 32 + 3) // 4 * 4
    words = np.zeros(nw, dtype=np.uint32)
    used = int(lib().ccmo_vlb_pack(_ptr(a), a.size, k, _ptr(words), nw))
    assert used == nbits
    return Vlb(a.size, k, nbits, words)


def vlb_unpack(v: Vlb) -> np.ndarray:
    out = np.empty(v.n, dtype=np.int64)
    lib().ccmo_vlb_unpack(_ptr(v.words), v.n, v.k, _ptr(out))
    return out
