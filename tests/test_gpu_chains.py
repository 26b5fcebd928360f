"""Chains that stay compressed on the GPU against the oracle, word for word:
y = A x + B z (both products summed in one scratch, y packed once) through
the row-streaming, column-slab and generic kernels, its overflow and error
propagation, and y = A (B x) with the intermediate packed on the GPU."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_packed, device, lib_ccm, to_dev, words_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccm():
    device()
    return lib_ccm()


def _signed(seed, shape, b):
    return synth.uniform_signed(seed, synth.STREAM_A, int(np.prod(shape)), b).reshape(shape)


@pytest.mark.parametrize("m,n1,n2,ba,bb", [
    (257, 1280, 4096, 5, 3),     # row-streaming kernel for both terms (byte lanes)
    (300, 1024, 768, 12, 20),    # row-streaming, int32 path
    (3, 262144, 128, 5, 8),      # the first term on the column-slab kernel
    (33, 100, 77, 9, 9),         # generic kernel (cols not a multiple of 128)
    (64, 128, 130, 40, 6),       # wide fields: generic 128-bit sums
    (5, 0, 128, 4, 4),           # an empty first product
])
def test_matvec2_matches_oracle(ccm, m, n1, n2, ba, bb):
    a, b = _signed(m + ba, (m, n1), ba), _signed(m + bb + 1, (m, n2), bb)
    x = synth.uniform_int(n1 + 3, synth.STREAM_X, n1, -128, 127).reshape(n1, 1)
    z = synth.uniform_int(n2 + 5, synth.STREAM_X, n2, 0, 100).reshape(n2, 1)
    expect = oracle.matvec2(oracle.pack(a, m, n1), oracle.pack(x, n1, 1), oracle.pack(b, m, n2),
                            oracle.pack(z, n2, 1))
    pa, pb = ccm.pack(to_dev(a)), ccm.pack(to_dev(b))
    px, pz = ccm.pack(to_dev(x)), ccm.pack(to_dev(z))
    y = ccm.matvec2(pa, px, pb, pz)
    assert_same_packed(y, expect, f"matvec2 {m}x{n1} + {m}x{n2}")
    # the same as two separate products and an add (each packed on the way)
    if n1:
        y2 = ccm.add(ccm.matvec(pa, px), ccm.matvec(pb, pz), capacity=y.capacity)
        assert np.array_equal(words_np(y2), words_np(y))


def test_matvec2_overflow_and_errors(ccm):
    big = np.full((2, 128), 3 << 47, dtype=np.int64)
    x = np.full((128, 1), 127, dtype=np.int64)  # each product ~1.49 * 2^62, the sum ~1.49 * 2^63
    pa, px = ccm.pack(to_dev(big)), ccm.pack(to_dev(x))
    assert ccm.matvec2(pa, px, pa, px).status == ccm.E_OVERFLOW
    assert ccm.matvec2(pa, px, ccm.pack(to_dev(-big)), px).check().width == 1
    # an invalid second operand's status reaches y
    bad = ccm.scale(pa, 1 << 20, capacity=ccm.words_for(2, 128, 64))  # overflows: status set
    assert bad.status == ccm.E_OVERFLOW
    assert ccm.matvec2(pa, px, bad, px).status == ccm.E_OVERFLOW


@pytest.mark.parametrize("m,k,n,b", [(200, 384, 256, 6), (64, 1000, 37, 11)])
def test_matvec_chain(ccm, m, k, n, b):
    """y = A (B x): the intermediate stays packed on the GPU."""
    a, bm = _signed(m + b, (m, k), b), _signed(k + b, (k, n), b)
    x = synth.uniform_int(n, synth.STREAM_X, n, -128, 127).reshape(n, 1)
    expect = oracle.matvec_chain(oracle.pack(a), oracle.pack(bm), oracle.pack(x))
    y = ccm.matvec_chain(ccm.pack(to_dev(a)), ccm.pack(to_dev(bm)), ccm.pack(to_dev(x)))
    assert_same_packed(y, expect, f"chain {m}x{k}x{n}")
