"""Row-sharded matvec on the GPU: ccm_repack against the oracle (re-pack at a
wider width and another sign mode, at a row offset, every other word zero),
and the sharded schedule of paper_1303_0270_gb300.shard with two ranks
emulated in one process (the per-rank steps through libccm; the MAX and SUM
reductions done here on the host, no kernel waits on another), compared word
for word with the oracle's matvec of the whole matrix."""
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


@pytest.mark.parametrize("rows,cols,b,signed,width,to_signed,offset,out_rows",
                         [(32, 1, 5, 0, 5, 0, 0, 32), (32, 1, 5, 0, 9, 1, 64, 100),
                          (37, 1, 7, 1, 7, 1, 32, 69), (64, 3, 12, 1, 20, 1, 32, 96),
                          (5, 1, 1, 0, 64, 1, 0, 5), (96, 1, 31, 1, 33, 1, 0, 200)])
def test_repack_at_width_and_offset(ccm, rows, cols, b, signed, width, to_signed, offset,
                                    out_rows):
    v = synth.uniform_signed(rows + b, 0, rows * cols, b) if signed else \
        synth.uniform_int(rows + b, 0, rows * cols, 0, (1 << b) - 1)
    v = v.reshape(rows, cols)
    pa = ccm.pack(to_dev(v))
    out = ccm.PackedMatrix(out_rows, cols, ccm.words_for(out_rows, cols, width))
    ccm.repack_into(pa, width, to_signed, out, offset)
    h = out.check().header()
    assert (h.width, h.is_signed, h.rows, h.cols) == (width, to_signed, out_rows, cols)
    full = np.zeros((out_rows, cols), dtype=np.int64)
    full[offset:offset + rows] = v
    expect = oracle.pack_at(full.ravel(), out_rows, cols, width, to_signed)
    assert h.nwords == expect.words.size
    assert np.array_equal(words_np(out), expect.words)


def test_repack_rejects_widths_that_do_not_fit(ccm):
    v = synth.uniform_signed(3, 0, 64, 9).reshape(64, 1)
    v[0, 0], v[1, 0] = -256, 255  # width exactly 9, signed
    pa = ccm.pack(to_dev(v))
    assert (pa.width, pa.is_signed) == (9, 1)
    for width, sgn in ((8, 1), (9, 0), (12, 0)):  # too narrow, or unsigned for signed data
        out = ccm.PackedMatrix(64, 1, ccm.words_for(64, 1, 12))
        ccm.repack_into(pa, width, sgn, out)
        assert out.header().status == ccm.E_WIDTH
    with pytest.raises(ccm.CCMError):  # the block would not start on a word boundary
        ccm.repack_into(pa, 9, 1, ccm.PackedMatrix(80, 1, ccm.words_for(80, 1, 9)), 3)


@pytest.mark.parametrize("seed,m,n,b,world", [(1, 100, 384, 5, 2), (2, 8192, 1024, 8, 2),
                                              (3, 257, 130, 12, 3), (4, 40, 64, 2, 4)])
def test_sharded_schedule_two_ranks_on_one_gpu(ccm, seed, m, n, b, world):
    from paper_1303_0270_gb300 import shard
    a = synth.uniform_signed(seed, synth.STREAM_A, m * n, b).reshape(m, n)
    x = synth.uniform_int(seed, synth.STREAM_X, n, -128, 127).reshape(n, 1)
    px = ccm.pack(to_dev(x))
    be = shard.CcmBackend()
    blocks = shard.row_blocks(m, world)
    ys = [be.matvec(ccm.pack(to_dev(a[r0:r1])), px) for r0, r1 in blocks]
    stats = [be.stats(y) for y in ys]
    assert all(s[2] == 0 for s in stats)
    width, sgn = shard.width_from_stats(max(s[0] for s in stats), max(s[1] for s in stats))
    outs = [be.repack(y, width, sgn, m, r0) for y, (r0, _) in zip(ys, blocks)]
    total = sum(be.words(o) for o in outs)          # the SUM all-reduce
    be.words(outs[0]).copy_(total)
    expect = oracle.matvec(oracle.pack(a), oracle.pack(x))
    assert_same_packed(be.finish(outs[0]), expect, f"sharded matvec seed={seed}")


def test_sharded_matvec_single_rank(ccm):
    from paper_1303_0270_gb300 import shard
    a = synth.uniform_signed(9, synth.STREAM_A, 300 * 256, 6).reshape(300, 256)
    x = synth.uniform_int(9, synth.STREAM_X, 256, -128, 127).reshape(256, 1)
    y = shard.sharded_matvec(ccm.pack(to_dev(a)), ccm.pack(to_dev(x)), 300, 0)
    assert_same_packed(y, oracle.matvec(oracle.pack(a), oracle.pack(x)), "one rank")
