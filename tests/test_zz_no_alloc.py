"""ccm_matvec_static: the matvec entry point for callers that must not
allocate device memory (their memory is reserved up front by another
allocator, or they cannot afford the device-wide synchronisation of a
cudaMalloc).  Its scratch is a fixed array inside libccm; this test calls it
through the C ABI and checks that three calls in a row give exactly the words
ccm_matvec gives with a caller-provided workspace (integer results: the
tolerance is zero), including when the second call must not see what the
earlier ones left in the shared scratch."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import device, lib_ccm, to_dev, words_np

pytestmark = pytest.mark.gpu


def _case(ccm, seed, m, n, b):
    a = synth.uniform_signed(seed, synth.STREAM_A, m * n, b).reshape(m, n)
    x = synth.uniform_signed(seed, synth.STREAM_X, n, 8).reshape(n, 1)
    return ccm.pack(to_dev(a)), ccm.pack(to_dev(x))


def test_static_scratch_matvec_matches_workspace_matvec():
    ccm = lib_ccm()
    L = ccm.lib()
    dev = device()
    # calls in a row: row-aligned (streaming kernel), ragged (row kernel), then
    # a smaller row-aligned one that finds the larger call's y sums and x
    # still in the shared scratch beyond its own rows and columns
    for seed, (m, n, b) in ((11, (1000, 1024, 7)), (12, (333, 777, 19)),
                            (13, (96, 256, 12))):
        pa, px = _case(ccm, seed, m, n, b)
        ref = ccm.matvec(pa, px, capacity=ccm.words_for(m, 1, 64))
        out = ccm.PackedMatrix(m, 1, ccm.words_for(m, 1, 64), dev)
        ma, mx, my = pa.c(), px.c(), out.c()
        st = L.ccm_matvec_static(ctypes.byref(ma), ctypes.byref(mx), ctypes.byref(my),
                                 ccm._stream(None))
        assert st == ccm.OK
        out._written()
        assert out.header().status == 0 and ref.header().status == 0
        assert out.header().width == ref.header().width
        assert np.array_equal(words_np(out), words_np(ref))


def test_static_scratch_rejects_oversized_problems():
    ccm = lib_ccm()
    L = ccm.lib()
    big = ccm.Matrix(0x1000, 0x2000, 1 << 20, 4, 200000)
    x = ccm.Matrix(0x3000, 0x4000, 1 << 20, 200000, 1)
    y = ccm.Matrix(0x5000, 0x6000, 16, 4, 1)
    assert L.ccm_matvec_static(ctypes.byref(big), ctypes.byref(x), ctypes.byref(y),
                               None) == ccm.E_CAPACITY
