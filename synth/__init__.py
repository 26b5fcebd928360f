"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the compression method itself: it only draws
the integer matrices, vectors and shapes that the workloads are made of.  Every
draw is counter-based, so element ``i`` of stream ``s`` under seed ``seed`` is a
pure function of ``(seed, s, i)`` and any subset of a large input can be
regenerated on its own.

Generator (published definitions, written out here):

* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): the generator seeded with ``x`` returns, as its
  ``k``-th output (k = 1, 2, ...), ``mix(x + k * GAMMA)`` with
  ``GAMMA = 0x9E3779B97F4A7C15`` and the finaliser ``mix`` below.
* Stream key: ``key(seed, s) = mix(seed + (s + 1) * GAMMA)``, i.e. output
  ``s + 1`` of SplitMix64 seeded with ``seed``.
* Element ``i`` of stream ``s``: ``u64(seed, s, i) = mix(key(seed, s) + (i + 1) * GAMMA)``.
* Integers uniform in ``[lo, hi]``: Lemire's multiply-high map
  ``lo + floor(u * r / 2**64)`` with ``r = hi - lo + 1`` (no rejection step, so
  the bias is at most ``r / 2**64``).
* Poisson(lambda): inversion of a float64 CDF table built on the host,
  ``u53 = (u >> 11) * 2**-53``, value = number of table entries ``<= u53``.
  The last table entry is forced to +inf, so draws never exceed the table.
* Log-uniform sizes in ``[lo, hi)``: ``floor(lo * (hi / lo) ** u53)`` (host only).

The CUDA library carries its own implementation of the same definitions for
bench-scale inputs; the GPU tests check it against this one element by element.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream ids used by the workloads (one per role, so that A, B and x differ).
STREAM_A = 0
STREAM_B = 1
STREAM_X = 2
STREAM_SHAPES = 3
STREAM_WIDTHS = 4
STREAM_ARRIVALS = 5
STREAM_KINDS = 6
STREAM_INDEX = 7


def mix_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (reference form for tests)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    return mix_int((seed + (stream + 1) * GAMMA) & MASK64)


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Elements ``start .. start+count-1`` of stream ``stream`` as uint64."""
    key = np.uint64(stream_key(seed, stream))
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key + idx * np.uint64(GAMMA)
    return _mix(z)


def u64_at(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Elements at arbitrary indices (uint64 array) of a stream."""
    key = np.uint64(stream_key(seed, stream))
    idx = np.asarray(index, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        z = key + idx * np.uint64(GAMMA)
    return _mix(z)


def mulhi64(u: np.ndarray, r: int) -> np.ndarray:
    """floor(u * r / 2**64) for uint64 ``u`` and an integer ``0 <= r < 2**64``."""
    u = np.asarray(u, dtype=np.uint64)
    m32 = np.uint64(0xFFFFFFFF)
    a, b = u >> np.uint64(32), u & m32
    c, d = np.uint64(r >> 32), np.uint64(r & 0xFFFFFFFF)
    with np.errstate(over="ignore"):
        ad, bc, bd, ac = a * d, b * c, b * d, a * c
        mid = (bd >> np.uint64(32)) + (ad & m32) + (bc & m32)
        return ac + (ad >> np.uint64(32)) + (bc >> np.uint64(32)) + (mid >> np.uint64(32))


def map_uniform(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Lemire map of uint64 draws onto the integers ``[lo, hi]`` (int64)."""
    if not (-(1 << 63) <= lo <= hi <= (1 << 63) - 1):
        raise ValueError("bounds must fit int64")
    r = hi - lo + 1
    with np.errstate(over="ignore"):
        if r == 1 << 64:
            off = u
        else:
            off = mulhi64(u, r)
        return (off + np.uint64(lo & MASK64)).view(np.int64)


def uniform_int(seed: int, stream: int, count: int, lo: int, hi: int, start: int = 0) -> np.ndarray:
    return map_uniform(u64(seed, stream, start, count), lo, hi)


def signed_range(b: int) -> tuple[int, int]:
    """The two's complement range of a ``b``-bit field."""
    return -(1 << (b - 1)), (1 << (b - 1)) - 1


def uniform_signed(seed: int, stream: int, count: int, b: int, start: int = 0) -> np.ndarray:
    lo, hi = signed_range(b)
    return uniform_int(seed, stream, count, lo, hi, start)


def poisson_cdf_table(lam: float, max_len: int = 256) -> np.ndarray:
    """float64 CDF table of Poisson(lam), terms summed in order; last entry +inf."""
    p = math.exp(-lam)
    acc = 0.0
    cdf = []
    for k in range(max_len):
        acc += p
        cdf.append(acc)
        p = p * lam / (k + 1)
        if acc >= 1.0 or (k > lam and p < 1e-300):
            break
    cdf[-1] = math.inf
    return np.asarray(cdf, dtype=np.float64)


def u53(u: np.ndarray) -> np.ndarray:
    return (np.asarray(u, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def poisson(seed: int, stream: int, count: int, lam: float, start: int = 0) -> np.ndarray:
    table = poisson_cdf_table(lam)
    x = u53(u64(seed, stream, start, count))
    return np.searchsorted(table, x, side="right").astype(np.int64)


def log_uniform_sizes(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    x = u53(u64(seed, stream, 0, count))
    return np.floor(lo * (hi / lo) ** x).astype(np.int64)


# ---------------------------------------------------------------------------
# Workload recipes (shapes, distributions and seeds of each configuration).
# ---------------------------------------------------------------------------
SEED_A = 1303
SEED_B = 1304


def pr1_inputs(seed: int = SEED_A):
    """256x256 A and B uniform in [-100, 100], x of length 256 in [-100, 100], s = 7."""
    n = 256
    a = uniform_int(seed, STREAM_A, n * n, -100, 100).reshape(n, n)
    b = uniform_int(seed, STREAM_B, n * n, -100, 100).reshape(n, n)
    x = uniform_int(seed, STREAM_X, n, -100, 100)
    return a, b, x, 7


def count_matrix(seed: int, stream: int, rows: int, cols: int, lam: float = 5.0, start: int = 0):
    """Poisson(lam) count matrix, rows x cols, int64."""
    return poisson(seed, stream, rows * cols, lam, start).reshape(rows, cols)


def sweep_matrix(seed: int, stream: int, rows: int, cols: int, b: int):
    """Entries uniform over the signed b-bit range."""
    return uniform_signed(seed, stream, rows * cols, b).reshape(rows, cols)


def x_vector(seed: int, n: int, b: int = 8):
    """Matvec operand: uniform over the signed 8-bit range unless told otherwise."""
    return uniform_signed(seed, STREAM_X, n, b)


def batch_shapes(seed: int, count: int, lo: int = 16, hi: int = 2048, wlo: int = 1, whi: int = 24):
    """Shapes (rows, cols) log-uniform in [lo, hi) and widths uniform in [wlo, whi]."""
    rc = log_uniform_sizes(seed, STREAM_SHAPES, 2 * count, lo, hi).reshape(count, 2)
    w = uniform_int(seed, STREAM_WIDTHS, count, wlo, whi)
    return rc[:, 0].copy(), rc[:, 1].copy(), w


def batch_matrix_seed(seed: int, index: int) -> int:
    """Per-matrix seed of a batch (matrix ``index``), derived counter-style."""
    return mix_int((seed * 0x100000001B3 + index * GAMMA + 0x632BE59BD9B4E019) & MASK64)
