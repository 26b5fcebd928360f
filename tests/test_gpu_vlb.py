"""VLB (Method 2) on the GPU against the oracle: the stream word for word, the
offset index, the round trip, and the SM/VLB size comparison."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import device, lib_ccm, to_dev, torch

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
