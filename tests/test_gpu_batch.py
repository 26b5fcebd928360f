"""Batched matvec (one persistent launch over many packed matrices of uneven
shapes and widths) against the oracle and against one call per matrix."""
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


def _batch_inputs(seed, count, lo=1, hi=300, wlo=1, whi=24):
    rows, cols, widths = synth.batch_shapes(seed, count, lo, hi, wlo, whi)
    mats, xs = [], []
    for i in range(count):
        s = synth.batch_matrix_seed(seed, i)
        b = int(widths[i])
        a = synth.uniform_signed(s, synth.STREAM_A, int(rows[i] * cols[i]), b)
        if i % 3 == 0:
            a = np.abs(a)  # unsigned fields too
        # x kinds: signed 8-bit (byte lanes for b <= 8), unsigned 7-bit (byte
        # lanes), unsigned 8-bit and signed 12-bit (the int32 path at any b)
        xk = i % 4
        if xk == 0:
            x = synth.uniform_signed(s, synth.STREAM_X, int(cols[i]), 8)
        elif xk == 1:
            x = synth.uniform_int(s, synth.STREAM_X, int(cols[i]), 0, 127)
        elif xk == 2:
            x = synth.uniform_int(s, synth.STREAM_X, int(cols[i]), 0, 255)
        else:
            x = synth.uniform_signed(s, synth.STREAM_X, int(cols[i]), 12)
        mats.append(a.reshape(int(rows[i]), int(cols[i])))
        xs.append(x.reshape(-1, 1))
    return mats, xs


def _pack_exact(ccm, arr):
    return ccm.pack(to_dev(arr))


@pytest.mark.parametrize("slots,unit_segments,stage_bytes",
                         [(2, 64, 0), (4, 64, 128), (3, 4096, 6144), (0, 1024, 1536)])
def test_batch_matches_oracle(ccm, slots, unit_segments, stage_bytes):
    from paper_1303_0270_gb300.batch import BatchMatvec
    mats, xs = _batch_inputs(77, 160)
    # degenerate shapes: short rows, a single field, rows of exactly 32 and 33 fields
    extra = [(1, 1), (5, 16), (3, 31), (2, 32), (4, 33), (1, 2048), (300, 1)]
    for k, (r, c) in enumerate(extra):
        mats.append(synth.uniform_signed(900 + k, 0, r * c, 11).reshape(r, c))
        xs.append(synth.uniform_signed(950 + k, 0, c, 8).reshape(-1, 1))
    pa = [_pack_exact(ccm, a) for a in mats]
    px = [_pack_exact(ccm, x) for x in xs]
    bm = BatchMatvec(pa, px, unit_segments=unit_segments)
    bm.slots = slots  # ring depth: 1 to 3 stages in flight per warp (0: the default)
    bm.stage_bytes = stage_bytes  # 128: one segment per lane per stage; 6144: up to 8
    bm.launch()
    torch.cuda.synchronize()
    for i, (a, x) in enumerate(zip(mats, xs)):
        o = oracle.matvec(oracle.pack(a), oracle.pack(x))
        assert_same_packed(bm.ys[i], o, f"batch entry {i} {a.shape}")


def test_batch_equals_single_calls_and_graph_replay(ccm):
    from paper_1303_0270_gb300.batch import BatchMatvec
    mats, xs = _batch_inputs(78, 120, lo=16, hi=700)
    pa = [_pack_exact(ccm, a) for a in mats]
    px = [_pack_exact(ccm, x) for x in xs]
    singles = [ccm.matvec(a, x) for a, x in zip(pa, px)]
    bm = BatchMatvec(pa, px, unit_segments=256)
    bm.run()  # captured graph
    torch.cuda.synchronize()
    for i in range(len(mats)):
        assert np.array_equal(words_np(bm.ys[i]), words_np(singles[i]))
        assert bm.ys[i].header().width == singles[i].header().width
    # replay twice more: same words (the scratch is re-initialised every run)
    first = [words_np(y).copy() for y in bm.ys]
    bm.run()
    bm.run()
    torch.cuda.synchronize()
    for i in range(len(mats)):
        assert np.array_equal(words_np(bm.ys[i]), first[i])


def test_batch_autotune_keeps_results(ccm, tmp_path):
    from paper_1303_0270_gb300.batch import BatchMatvec
    mats, xs = _batch_inputs(79, 60, lo=16, hi=500)
    pa = [_pack_exact(ccm, a) for a in mats]
    px = [_pack_exact(ccm, x) for x in xs]
    bm = BatchMatvec(pa, px)
    best = bm.autotune(candidates=[(64, 152), (256, 304), (1024, 608)], reps=2,
                       cache=str(tmp_path / "tune.json"))
    assert best["unit_segments"] in (64, 256, 1024)
    bm.launch()
    torch.cuda.synchronize()
    for i, (a, x) in enumerate(zip(mats, xs)):
        assert_same_packed(bm.ys[i], oracle.matvec(oracle.pack(a), oracle.pack(x)), f"tuned {i}")
    # a second tuner on the same batch reads the cache
    bm2 = BatchMatvec(pa, px)
    again = bm2.autotune(cache=str(tmp_path / "tune.json"))
    assert again["unit_segments"] == best["unit_segments"]


def test_batch_errors(ccm):
    from paper_1303_0270_gb300.batch import BatchMatvec
    a = _pack_exact(ccm, synth.uniform_signed(1, 0, 12, 5).reshape(3, 4))
    x_wrong = _pack_exact(ccm, synth.uniform_signed(2, 0, 5, 5).reshape(5, 1))
    with pytest.raises(ccm.CCMError) as ei:
        BatchMatvec([a], [x_wrong])
    assert ei.value.status == ccm.E_SHAPE
    # a 41-bit A is outside the kernel's widths: that entry alone reports it
    wide = _pack_exact(ccm, np.full((3, 4), 1 << 40, dtype=np.int64))
    x = _pack_exact(ccm, np.ones((4, 1), dtype=np.int64))
    bm = BatchMatvec([wide, a], [x, x], ys=None)
    bm.launch()
    torch.cuda.synchronize()
    assert bm.ys[0].status == ccm.E_WIDTH
    assert np.array_equal(ccm.unpack(bm.ys[1].check()).cpu().numpy().ravel(),
                          ccm.unpack(a).cpu().numpy() @ np.ones(4, dtype=np.int64))


def test_batch_wide_widths_and_loose_capacity(ccm):
    """Widths 25..32 (the staging slots sized for the widest A the capacities
    admit) and entries packed into buffers much larger than their width needs
    (bound clamped at 32): every y against the oracle."""
    from paper_1303_0270_gb300.batch import BatchMatvec
    mats, xs, pa = [], [], []
    shapes = [(33, 70), (7, 2048), (130, 33), (64, 64), (1, 500), (257, 96)]
    for k, (r, c) in enumerate(shapes):
        for b in (25, 28, 31, 32, 3):
            a = synth.uniform_signed(1000 + 7 * k + b, synth.STREAM_A, r * c, b).reshape(r, c)
            if (k + b) % 2:
                a = np.abs(a) if b < 32 else a
            x = synth.uniform_signed(2000 + k + b, synth.STREAM_X, c, 8).reshape(-1, 1)
            mats.append(a)
            xs.append(x)
            loose = (k + b) % 3 == 0
            pa.append(ccm.pack(to_dev(a), capacity=ccm.words_for(r, c, 64)) if loose
                      else _pack_exact(ccm, a))
    px = [_pack_exact(ccm, x) for x in xs]
    for us in (32, 512):
        bm = BatchMatvec(pa, px, unit_segments=us)
        bm.launch()
        torch.cuda.synchronize()
        for i, (a, x) in enumerate(zip(mats, xs)):
            o = oracle.matvec(oracle.pack(a), oracle.pack(x))
            assert_same_packed(bm.ys[i], o, f"wide batch entry {i} {a.shape} us={us}")


@pytest.mark.parametrize("whi", [12, 16, 20, 24])
def test_batch_bounded_widths(ccm, whi):
    """Batches of widths up to 12, 16, 20, 24 (shapes of at least 16 x 16, so
    the capacity bound is the width itself and the staging slots are sized to
    it): every y against the oracle."""
    from paper_1303_0270_gb300.batch import BatchMatvec
    mats, xs = _batch_inputs(80 + whi, 40, lo=16, hi=400, wlo=1, whi=whi)
    pa = [_pack_exact(ccm, a) for a in mats]
    px = [_pack_exact(ccm, x) for x in xs]
    bm = BatchMatvec(pa, px, unit_segments=128)
    bm.launch()
    torch.cuda.synchronize()
    for i, (a, x) in enumerate(zip(mats, xs)):
        assert_same_packed(bm.ys[i], oracle.matvec(oracle.pack(a), oracle.pack(x)),
                           f"class batch whi={whi} entry {i} {a.shape}")
