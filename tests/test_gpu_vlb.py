"""VLB (Method 2) on the GPU against the oracle: the stream word for word, the
offset index, the round trip, and the SM/VLB size comparison."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_packed, device, lib_ccm, to_dev, torch, words_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccm():
    device()
    return lib_ccm()


def _cases():
    n = 70000  # 69 encoder blocks, a ragged last block and index chunk
    yield "zeros", np.zeros((7, 9), dtype=np.int64)
    yield "one", np.array([[5]], dtype=np.int64)
    yield "worked", np.array([[900, 1023, 721, 256, 1, 10, 700, 20]], dtype=np.int64)
    yield "poisson5", synth.poisson(1303, 0, n, 5.0).reshape(100, 700)
    u = synth.u53(synth.u64(7, 0, 0, n))
    heavy = np.floor(2.0 ** (u * 40)).astype(np.int64)  # bit lengths spread over 1..40
    yield "heavy", heavy.reshape(700, 100)
    big = synth.uniform_int(9, 0, 3000, 0, (1 << 62) - 1)
    yield "big", big.reshape(3, 1000)
    # prefix + value of at most 16 bits (two entries per refill of the fast
    # decoder) and of 17..32 bits (one), on whole index chunks only
    yield "len12", synth.uniform_int(11, 0, 64 * 700, 0, (1 << 12) - 1).reshape(64, 700)
    yield "len20", synth.uniform_int(12, 0, 64 * 700, 0, (1 << 20) - 1).reshape(700, 64)
    yield "pr1abs", np.abs(synth.pr1_inputs()[0])


@pytest.mark.parametrize("name,arr", list(_cases()), ids=[c[0] for c in _cases()])
def test_vlb_matches_oracle(ccm, name, arr):
    o = oracle.vlb_pack(arr)
    v = ccm.vlb_pack(to_dev(arr))
    h = v.header()
    assert h.status == 0 and h.magic == ccm.VLB_MAGIC
    assert (h.width, int(h.stat_or)) == (o.k, o.nbits), name
    words = v.words().cpu().numpy().view(np.uint32)
    assert words.size == o.words.size
    assert np.array_equal(words, o.words), name
    # the index: bit offset of every 64th entry, then the total
    flat = arr.ravel()
    lens = np.array([max(1, int(x).bit_length()) for x in flat], dtype=np.int64) + o.k
    offs = np.concatenate([[0], np.cumsum(lens)])
    expect = np.concatenate([offs[:-1][::64], [offs[-1]]])
    assert np.array_equal(v.index.cpu().numpy(), expect), name
    assert np.array_equal(ccm.vlb_unpack(v).cpu().numpy(), arr), name
    if int(flat.max()).bit_length() <= 31:
        assert np.array_equal(ccm.vlb_unpack(v, dtype=torch.int32).cpu().numpy(), arr)


def test_vlb_negative_is_rejected(ccm):
    h = ccm.vlb_measure(to_dev(np.array([[3, -1, 4]])))
    assert h.status == ccm.E_RANGE


def test_choose_matches_the_two_sizes(ccm):
    for name, arr in _cases():
        c = ccm.choose(to_dev(arr))
        assert c["sm_bits"] == arr.size * oracle.pack(arr).width
        assert c["vlb_bits"] == oracle.vlb_pack(arr).nbits
        assert c["choice"] == ("sm" if c["sm_bits"] <= c["vlb_bits"] else "vlb")


# cols a multiple of 64 and at most 16384 take the fast kernel (x staged in
# shared memory); the others, and x wider than 32 bits, the general one.
@pytest.mark.parametrize("rows,cols,kind", [(1, 1, "poisson"), (7, 64, "poisson"), (13, 100, "poisson"),
                                            (257, 1280, "poisson"), (33, 4096, "wide"),
                                            (64, 63, "wide"), (5, 3000, "zeros"),
                                            (24, 16384, "poisson"), (3, 16448, "poisson"),
                                            (50, 640, "len12"), (40, 704, "len20"),
                                            (9, 192, "widex")])
def test_vlb_matvec_matches_oracle(ccm, rows, cols, kind):
    """y = A x with A in VLB form against the oracle (A decoded by the oracle's
    VLB unpack, multiplied, y re-packed): word for word."""
    n = rows * cols
    if kind == "poisson":
        a = synth.count_matrix(rows + cols, synth.STREAM_A, rows, cols)
    elif kind == "wide":  # bit lengths spread over 1..40 (the prefix needs 6 bits)
        u = synth.u53(synth.u64(rows, synth.STREAM_A, 0, n))
        a = np.floor(2.0 ** (u * 40)).astype(np.int64).reshape(rows, cols)
    elif kind in ("len12", "len20"):
        a = synth.uniform_int(rows, synth.STREAM_A, n, 0, (1 << int(kind[3:])) - 1)
        a = a.reshape(rows, cols)
    elif kind == "widex":
        a = synth.count_matrix(rows + cols, synth.STREAM_A, rows, cols)
    else:
        a = np.zeros((rows, cols), dtype=np.int64)
    lo, hi = (-(1 << 40), 1 << 40) if kind == "widex" else (-128, 127)
    x = synth.uniform_int(cols, synth.STREAM_X, cols, lo, hi).reshape(cols, 1)
    ov = oracle.vlb_pack(a.ravel())
    expect = oracle.matvec(oracle.pack(oracle.vlb_unpack(ov).reshape(rows, cols)), oracle.pack(x))
    v = ccm.vlb_pack(to_dev(a))
    y = ccm.vlb_matvec(v, ccm.pack(to_dev(x)))
    assert_same_packed(y, expect, f"vlb matvec {rows}x{cols} {kind}")
    # the SM route gives the same y
    ys = ccm.matvec(ccm.pack(to_dev(a)), ccm.pack(to_dev(x)), capacity=y.capacity)
    assert np.array_equal(words_np(ys), words_np(y))


def test_vlb_matvec_overflow_is_reported(ccm):
    a = np.full((2, 8), (1 << 62) - 1, dtype=np.int64)
    x = np.full((8, 1), 3, dtype=np.int64)
    y = ccm.vlb_matvec(ccm.vlb_pack(to_dev(a)), ccm.pack(to_dev(x)))
    assert y.status == ccm.E_OVERFLOW


def test_vlb_matvec_overflow_fast_shape_is_reported(ccm):
    # cols a multiple of 64: the fast kernel declines (partial sums may leave
    # int64) and the general one reports the overflow
    a = np.full((2, 64), (1 << 62) - 1, dtype=np.int64)
    x = np.full((64, 1), 3, dtype=np.int64)
    y = ccm.vlb_matvec(ccm.vlb_pack(to_dev(a)), ccm.pack(to_dev(x)))
    assert y.status == ccm.E_OVERFLOW


def _unpack_at(ccm, v, words_dev, dtype=torch.int64):
    import ctypes
    out = torch.empty((v.rows, v.cols), dtype=dtype, device=v.device)
    err = torch.full((1,), -7, dtype=torch.int32, device=v.device)
    rc = ccm.lib().ccm_vlb_unpack(ctypes.c_void_p(v.buf.data_ptr()), ctypes.c_void_p(words_dev),
                                  v.capacity, ctypes.c_void_p(v.index.data_ptr()), v.rows, v.cols,
                                  ctypes.c_void_p(out.data_ptr()),
                                  ccm.I64 if dtype == torch.int64 else ccm.I32,
                                  ctypes.c_void_p(err.data_ptr()), None)
    assert rc == 0
    torch.cuda.synchronize()
    return out, int(err.item())


def test_vlb_unpack_words_not_16_byte_aligned(ccm):
    """The stream at a 4-byte offset takes the one-thread-per-chunk decoder:
    same entries."""
    arr = synth.poisson(77, 0, 64 * 500 + 17, 5.0).reshape(1, -1)
    v = ccm.vlb_pack(to_dev(arr))
    w = v.words()
    moved = torch.zeros(w.numel() + 4, dtype=torch.int32, device=w.device)
    moved[1:1 + w.numel()] = w
    out, err = _unpack_at(ccm, v, moved.data_ptr() + 4)
    assert err == 0
    assert np.array_equal(out.cpu().numpy(), arr)


def test_vlb_unpack_reports_a_damaged_stream(ccm):
    """A zeroed stream word puts a prefix of 0 (L = 0, never written by the
    encoder) in some chunk: CCM_E_INPUT in *err."""
    arr = synth.poisson(78, 0, 64 * 4000, 5.0).reshape(64, 4000)
    v = ccm.vlb_pack(to_dev(arr))
    base = v.buf.data_ptr() + 4 * ccm.HEADER_WORDS
    ok, err = _unpack_at(ccm, v, base)
    assert err == 0 and np.array_equal(ok.cpu().numpy(), arr)
    w = v.buf.view(torch.int32)
    w[ccm.HEADER_WORDS + int(v.header().nwords) // 2] = 0
    _, err = _unpack_at(ccm, v, base)
    assert err == ccm.E_INPUT
    # the same stream at a 4-byte offset (the one-thread-per-chunk decoder)
    words = v.words()
    moved = torch.zeros(words.numel() + 4, dtype=torch.int32, device=words.device)
    moved[1:1 + words.numel()] = words
    _, err = _unpack_at(ccm, v, moved.data_ptr() + 4)
    assert err == ccm.E_INPUT
