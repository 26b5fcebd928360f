"""GPU parity: every hot-path step through the C ABI against the oracle,
word for word (integer work: tolerance 0), on seeded inputs that span several
1024-field tiles with ragged tails, every width 1..64 in both sign modes, and
the degenerate cases (empty, 1x1, all-zero, all-minus-one, exact word ends)."""
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


def _rand(seed, shape, b, signed=True):
    n = int(np.prod(shape))
    if signed:
        v = synth.uniform_signed(seed, 0, n, b)
    else:
        v = synth.uniform_int(seed, 0, n, 0, (1 << b) - 1 if b < 63 else (1 << 63) - 1)
    v = v.reshape(shape)
    lo, hi = synth.signed_range(b) if signed else (0, (1 << min(b, 63)) - 1)
    if n >= 2:
        v.flat[0] = lo
        v.flat[-1] = hi
    elif n == 1:
        v.flat[0] = lo if signed else hi  # the one entry alone fixes the width at b
    return v


SHAPES = [(1, 1), (1, 31), (7, 13), (33, 65), (3, 1000), (5, 2048)]


@pytest.mark.parametrize("b", list(range(1, 65)))
@pytest.mark.parametrize("signed", [0, 1])
def test_pack_unpack_every_width(ccm, b, signed):
    if not signed and b == 64:
        pytest.skip("int64 holds unsigned values up to 63 bits")
    for shape in SHAPES:
        a = _rand(b * 7 + signed, shape, b, bool(signed))
        o = oracle.pack(a)
        assert o.width == b
        p = ccm.pack(to_dev(a))
        assert_same_packed(p, o, f"pack b={b} s={signed} {shape}")
        assert np.array_equal(ccm.unpack(p).cpu().numpy(), a)
        if (signed and b <= 32) or (not signed and b <= 31):
            assert np.array_equal(ccm.unpack(p, dtype=torch.int32).cpu().numpy(), a)
        else:
            with pytest.raises(ccm.CCMError):
                ccm.unpack(p, dtype=torch.int32)


def test_pack_int32_input_and_degenerate(ccm):
    a, _, _, _ = synth.pr1_inputs()
    p = ccm.pack(to_dev(a, np.int32))
    assert_same_packed(p, oracle.pack(a), "pack int32 PR1")
    assert p.width == 8 and p.is_signed == 1
    for arr in (np.zeros((9, 70)), -np.ones((9, 70)), np.ones((1, 1)), np.zeros((1, 1))):
        arr = arr.astype(np.int64)
        assert_same_packed(ccm.pack(to_dev(arr)), oracle.pack(arr), "degenerate")
    # fields that end exactly on word ends: 32 fields of width 4 -> 4 words
    arr = np.arange(32, dtype=np.int64).reshape(4, 8) % 16
    assert_same_packed(ccm.pack(to_dev(arr)), oracle.pack(arr), "word end")


@pytest.mark.parametrize("dtype", [np.int64, np.int32])
def test_pack_unaligned_dense_input(ccm, dtype):
    """A dense input aligned only to its element size (a view one element into
    a buffer): the single-pass pack stages 16-byte copies, so such an input
    takes the element-wise path; the packed words are the same."""
    rows, cols = 37, 1003  # 37111 fields: 37 tiles, a ragged last one
    a = synth.uniform_signed(4242, 0, rows * cols, 9).reshape(rows, cols).astype(dtype)
    flat = torch.empty(rows * cols + 1, dtype=torch.int64 if dtype == np.int64 else torch.int32,
                       device=device())
    flat[1:] = torch.from_numpy(a.ravel()).to(flat.device)
    view = flat[1:].view(rows, cols)
    assert view.data_ptr() % 16 != 0
    o = oracle.pack(a.astype(np.int64))
    p = ccm.pack_into(view, ccm.PackedMatrix(rows, cols, ccm.words_for(rows, cols, o.width),
                                             device()))
    assert_same_packed(p, o, f"unaligned {np.dtype(dtype).name} pack")


def test_empty_matrix(ccm):
    dev = device()
    p = ccm.pack(torch.empty((0, 5), dtype=torch.int64, device=dev))
    h = p.header()
    assert (h.status, h.width, h.nwords, h.rows, h.cols) == (0, 1, 0, 0, 5)
    assert ccm.unpack(p).shape == (0, 5)


def test_get(ccm):
    a = _rand(11, (37, 91), 13)
    p = ccm.pack(to_dev(a))
    idx = synth.uniform_int(5, synth.STREAM_INDEX, 5000, 0, a.size - 1)
    idx[:2] = [0, a.size - 1]
    got = ccm.get(p, torch.from_numpy(idx)).cpu().numpy()
    assert np.array_equal(got, a.ravel()[idx])
    o = oracle.pack(a)
    assert [oracle.get(o, int(e) // 91, int(e) % 91) for e in idx[:50]] == got[:50].tolist()
    with pytest.raises(ccm.CCMError) as ei:
        ccm.get(p, torch.tensor([3, a.size], dtype=torch.int64))
    assert ei.value.status == ccm.E_RANGE


@pytest.mark.parametrize("ba,bb,sa,sb", [(1, 1, 0, 0), (5, 5, 0, 0), (8, 8, 1, 1), (13, 3, 1, 0),
                                         (32, 32, 1, 1), (33, 20, 1, 1), (62, 62, 1, 1),
                                         (63, 63, 1, 1), (64, 10, 1, 1)])
def test_add(ccm, ba, bb, sa, sb):
    for shape in [(1, 1), (17, 33), (3, 1000)]:
        a, b = _rand(ba, shape, ba, sa), _rand(bb + 100, shape, bb, sb)
        if ba == 64:
            b = np.where(a > 0, -np.abs(b), np.abs(b))  # keep the sum inside int64
        o = oracle.add(oracle.pack(a), oracle.pack(b))
        assert_same_packed(ccm.add(ccm.pack(to_dev(a)), ccm.pack(to_dev(b))), o,
                           f"add {ba}/{bb} {shape}")


def test_add_overflow_and_inverse(ccm):
    a = np.array([[(1 << 63) - 1, 5]], dtype=np.int64)
    b = np.array([[1, 5]], dtype=np.int64)
    c = ccm.add(ccm.pack(to_dev(a)), ccm.pack(to_dev(b)), capacity=16)
    assert c.status == ccm.E_OVERFLOW
    x = _rand(3, (40, 50), 20)
    z = ccm.add(ccm.pack(to_dev(x)), ccm.pack(to_dev(-x)))
    assert (z.width, z.is_signed) == (1, 0) and not words_np(z).any()


@pytest.mark.parametrize("s", [0, 1, -1, 7, -3, 1 << 20, -(1 << 30) + 5, (1 << 40) + 1])
@pytest.mark.parametrize("b", [1, 5, 8, 20])
def test_scale(ccm, s, b):
    for shape in [(1, 1), (11, 6), (3, 1000)]:
        a = _rand(b + 5, shape, b)
        pa = ccm.pack(to_dev(a))
        c = ccm.scale(pa, s)
        assert_same_packed(c, oracle.scale(oracle.pack(a), s), f"scale {s} b={b}")
        if s == 1:
            assert np.array_equal(words_np(c), words_np(pa))


def test_scale_overflow_and_capacity(ccm):
    pa = ccm.pack(to_dev(np.array([[1 << 40, 3]])))
    assert ccm.scale(pa, 1 << 23, capacity=16).status == ccm.E_OVERFLOW
    c = ccm.scale(pa, 2, capacity=4)  # needs 42-bit fields: 3 words, padded to 4 -> fits
    assert c.status == 0
    big = ccm.pack(to_dev(_rand(1, (100, 100), 30)))
    c = ccm.scale(big, 1 << 20, capacity=ccm.words_for(100, 100, 1))
    assert c.status == ccm.E_CAPACITY


def test_error_propagates_through_a_chain(ccm):
    pa = ccm.pack(to_dev(np.array([[1 << 62, 1]])))
    bad = ccm.scale(pa, 4, capacity=16)  # overflow
    c = ccm.add(bad, pa, capacity=16)
    assert c.status == ccm.E_OVERFLOW
    d = ccm.scale(c, 1, capacity=16)
    assert d.status == ccm.E_OVERFLOW


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (3, 5), (31, 33), (64, 130), (256, 256),
                                 (100, 1000), (1000, 100)])
@pytest.mark.parametrize("ba,bx", [(1, 1), (5, 8), (8, 8), (16, 8), (32, 8), (24, 24),
                                   (40, 30)])
def test_matvec(ccm, m, n, ba, bx):
    a, x = _rand(m * 3 + ba, (m, n), ba), _rand(n + bx, (n, 1), bx)
    oa, ox = oracle.pack(a), oracle.pack(x)
    try:
        o = oracle.matvec(oa, ox)
    except OverflowError:
        o = None
    y = ccm.matvec(ccm.pack(to_dev(a)), ccm.pack(to_dev(x)), capacity=ccm.words_for(m, 1, 64))
    if o is None:
        assert y.status == ccm.E_OVERFLOW
    else:
        assert_same_packed(y, o, f"matvec {m}x{n} b={ba}/{bx}")


def test_matvec_one_hot_and_empty_inner(ccm):
    a = _rand(2, (13, 9), 10)
    pa = ccm.pack(to_dev(a))
    for j in (0, 4, 8):
        x = np.zeros((9, 1), dtype=np.int64)
        x[j] = 1
        y = ccm.matvec(pa, ccm.pack(to_dev(x)))
        assert np.array_equal(ccm.unpack(y).cpu().numpy().ravel(), a[:, j])
    dev = device()
    e = ccm.pack(torch.empty((4, 0), dtype=torch.int64, device=dev))
    x0 = ccm.pack(torch.empty((0, 1), dtype=torch.int64, device=dev))
    y = ccm.matvec(e, x0, capacity=4)
    assert y.status == 0 and y.width == 1 and not ccm.unpack(y).any()


def test_matvec_pr1(ccm):
    a, _, x, _ = synth.pr1_inputs()
    o = oracle.matvec(oracle.pack(a), oracle.pack(x.reshape(-1, 1)))
    y = ccm.matvec(ccm.pack(to_dev(a, np.int32)), ccm.pack(to_dev(x.reshape(-1, 1), np.int32)))
    assert_same_packed(y, o, "matvec PR1")


@pytest.mark.parametrize("path", ["cuda", "auto"])
@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (2, 3, 4), (9, 17, 6), (33, 40, 31),
                                   (64, 64, 64), (130, 70, 90)])
@pytest.mark.parametrize("b", [1, 4, 8, 12, 16, 31])
def test_matmul(ccm, path, m, k, n, b):
    a, bm = _rand(m + k + b, (m, k), b), _rand(n + b, (k, n), b)
    try:
        o = oracle.matmul(oracle.pack(a), oracle.pack(bm))
    except OverflowError:
        o = None
    p = ccm.MATMUL_CUDACORE if path == "cuda" else ccm.MATMUL_AUTO
    c = ccm.matmul(ccm.pack(to_dev(a)), ccm.pack(to_dev(bm)), path=p,
                   capacity=ccm.words_for(m, n, 64))
    if o is None:
        assert c.status == ccm.E_OVERFLOW
    else:
        assert_same_packed(c, o, f"matmul {path} {m}x{k}x{n} b={b}")


def test_matmul_identity_and_overflow(ccm):
    a = _rand(4, (7, 7), 9)
    eye = ccm.pack(to_dev(np.eye(7, dtype=np.int64)))
    pa = ccm.pack(to_dev(a))
    assert np.array_equal(ccm.unpack(ccm.matmul(eye, pa)).cpu().numpy(), a)
    big = np.full((2, 3), 1 << 61, dtype=np.int64)
    c = ccm.matmul(ccm.pack(to_dev(big)), ccm.pack(to_dev(big.T.copy())), capacity=16,
                   path=ccm.MATMUL_CUDACORE)
    assert c.status == ccm.E_OVERFLOW


def test_pr1_full_chain(ccm):
    """PR1: 256x256 int32 A, B in [-100, 100], x, s = 7 -- every op, bit-exact."""
    a, b, x, s = synth.pr1_inputs()
    oa, ob, ox = oracle.pack(a), oracle.pack(b), oracle.pack(x.reshape(-1, 1))
    pa, pb = ccm.pack(to_dev(a, np.int32)), ccm.pack(to_dev(b, np.int32))
    px = ccm.pack(to_dev(x.reshape(-1, 1), np.int32))
    assert_same_packed(pa, oa, "PR1 pack A")
    assert pa.width == 8
    assert np.array_equal(ccm.unpack(pa, dtype=torch.int32).cpu().numpy(), a)
    assert_same_packed(ccm.add(pa, pb), oracle.add(oa, ob), "PR1 add")
    assert_same_packed(ccm.scale(pa, s), oracle.scale(oa, s), "PR1 scale")
    assert_same_packed(ccm.matvec(pa, px), oracle.matvec(oa, ox), "PR1 matvec")
    for path in (ccm.MATMUL_CUDACORE, ccm.MATMUL_AUTO):
        assert_same_packed(ccm.matmul(pa, pb, path=path), oracle.matmul(oa, ob), "PR1 matmul")


def test_device_generator_matches_synth(ccm):
    for lo, hi in [(-100, 100), (-(1 << 31), (1 << 31) - 1), (0, 1), (-(1 << 63), (1 << 63) - 1)]:
        g = ccm.gen_uniform(10000, 1303, 2, lo, hi, start=77).cpu().numpy()
        assert np.array_equal(g, synth.uniform_int(1303, 2, 10000, lo, hi, start=77))
    table = torch.from_numpy(synth.poisson_cdf_table(5.0))
    g = ccm.gen_poisson(200000, 1303, 0, table).cpu().numpy()
    assert np.array_equal(g, synth.poisson(1303, 0, 200000, 5.0))


# ---------------------------------------------------------------------------
# Both kernel families agree: the width-class kernels (chosen when the buffer
# capacities bound the widths) and the run-time-width kernels (chosen when a
# capacity allows any width up to 64).
# ---------------------------------------------------------------------------
def _pack_cap(ccm, a, cap_width):
    rows, cols = a.shape
    cap = ccm.words_for(rows, cols, cap_width)
    return ccm.pack_into(to_dev(a), ccm.PackedMatrix(rows, cols, cap, device()))


@pytest.mark.parametrize("b", [1, 2, 3, 5, 7, 8, 9, 12, 16, 17, 24, 31, 32])
def test_width_class_and_runtime_kernels_agree(ccm, b):
    shape = (13, 1111)  # 14443 fields: 15 tiles, a ragged last tile
    a = _rand(b + 1000, shape, b)
    c = _rand(b + 2000, shape, max(1, b - 1))
    oa, oc = oracle.pack(a), oracle.pack(c)
    pa_fast, pa_rt = _pack_cap(ccm, a, b), _pack_cap(ccm, a, 64)
    pc_fast = _pack_cap(ccm, c, max(1, b - 1))
    assert_same_packed(pa_fast, oa, f"class pack b={b}")
    two_pass = ccm.pack_into(to_dev(a), ccm.PackedMatrix(*shape, ccm.words_for(*shape, b), device()),
                             single_pass=False)
    assert_same_packed(two_pass, oa, f"two-pass class pack b={b}")
    assert_same_packed(pa_rt, oa, f"runtime pack b={b}")
    assert np.array_equal(ccm.unpack(pa_fast).cpu().numpy(), a)
    assert np.array_equal(ccm.unpack(pa_fast, dtype=torch.int32).cpu().numpy(), a)
    # output capacities: the exact width (the speculative width may not fit:
    # statistics then pack), a few bits more, and 64 bits (the run-time kernels)
    s_exp = oracle.add(oa, oc)
    for cap in (s_exp.width, s_exp.width + 3, 64):
        out = ccm.PackedMatrix(*shape, ccm.words_for(*shape, cap), device())
        assert_same_packed(ccm.add_into(pa_fast, pc_fast, out), s_exp, f"add b={b} cap={cap}")
    for s in (-3, 1 << 20):
        d_exp = oracle.scale(oa, s)
        for cap in (d_exp.width, 64):
            out = ccm.PackedMatrix(*shape, ccm.words_for(*shape, cap), device())
            assert_same_packed(ccm.scale_into(pa_fast, s, out), d_exp,
                               f"scale {s} b={b} cap={cap}")


@pytest.mark.parametrize("b", [1, 3, 5, 8, 11, 16, 23, 30, 32])
@pytest.mark.parametrize("case", ["first", "last", "over"])
def test_pack_speculative_width(ccm, b, case):
    """Single-pass pack when the output capacity bounds the width by exactly
    the matrix width (the speculative width): the one entry that needs all b
    bits sits in the first tile or in the last, every other tile is narrower,
    so most tiles are packed before any has reached the speculative width.
    'over': the capacity allows two bits more than the data needs, the
    speculation misses and every tile is re-coded from its local-width slot.
    Against the oracle word for word (padding included)."""
    shape = (40, 1500)  # 60000 fields: 59 tiles, a ragged last one
    signed = b % 2 == 1
    v = _rand(31 * b + 7, shape, max(1, b - 1), signed)
    extreme = synth.signed_range(b)[0] if signed else (1 << b) - 1
    if case == "last":
        v.flat[-3] = extreme
    else:
        v.flat[5] = extreme
    cap_width = b + 2 if case == "over" else b
    if cap_width > 32:
        pytest.skip("a capacity above 32 bits takes the run-time-width kernels")
    o = oracle.pack(v)
    assert o.width == b
    p = _pack_cap(ccm, v, cap_width)
    assert_same_packed(p, o, f"speculative pack b={b} {case}")
    assert np.array_equal(ccm.unpack(p).cpu().numpy(), v)


@pytest.mark.parametrize("ba,sa,bb,sb", [(5, 0, 5, 0), (1, 0, 1, 0), (3, 0, 4, 0), (7, 0, 7, 0),
                                         (2, 0, 6, 0), (8, 0, 1, 0), (7, 1, 3, 0), (3, 0, 7, 1),
                                         (8, 1, 8, 1), (16, 1, 1, 0), (13, 0, 13, 0),
                                         (31, 1, 31, 1)])
@pytest.mark.parametrize("hit", [True, False])
def test_add_speculative_width(ccm, ba, sa, bb, sb, hit):
    """The one-pass add writes C at the width the input ranges bound the sum
    to; that bound is reached (hit: entries at the range extremes, one pass)
    or not (miss: extremes avoided, the exact width is smaller and the second
    pass re-packs).  Both against the oracle word for word."""
    shape = (9, 3001)
    a = _rand(ba * 7 + sa, shape, ba, bool(sa))
    b = _rand(bb * 11 + sb, shape, bb, bool(sb))
    lo_a, hi_a = synth.signed_range(ba) if sa else (0, (1 << ba) - 1)
    lo_b, hi_b = synth.signed_range(bb) if sb else (0, (1 << bb) - 1)
    if hit:  # one pair at the top of both ranges and one at the bottom
        a.flat[5], b.flat[5], a.flat[9], b.flat[9] = hi_a, hi_b, lo_a, lo_b
    else:    # a still needs ba bits and b bb bits, but no extreme meets another
        a[:] = np.clip(a, lo_a // 2, hi_a // 2)
        b[:] = np.clip(b, lo_b // 2, hi_b // 2)
        a.flat[0], b.flat[0], a.flat[1], b.flat[1] = hi_a, 0, 0, hi_b
        a.flat[2], b.flat[2], a.flat[3], b.flat[3] = lo_a, 0, 0, lo_b
    oa, ob = oracle.pack(a), oracle.pack(b)
    assert (oa.width, ob.width) == (ba, bb)
    expect = oracle.add(oa, ob)
    got = ccm.add(ccm.pack(to_dev(a)), ccm.pack(to_dev(b)))
    assert_same_packed(got, expect, f"add spec {ba}/{sa} + {bb}/{sb} hit={hit}")


@pytest.mark.parametrize("b,sgn", [(29, 1), (30, 0), (31, 1), (31, 0), (32, 1), (32, 0)])
@pytest.mark.parametrize("cap", [None, 64])
@pytest.mark.parametrize("hit", [True, False])
def test_add_lanes_wide(ccm, b, sgn, cap, hit):
    """Same-width add of 29..32-bit operands with an output capacity of
    b + 1 bits (a width class when that is at most 32) or of 64 bits (no
    width class): the lane pass writes the sum (64-bit lanes for a 33-bit
    sum) and the remaining passes return at once or re-pack; word-identical
    to the oracle, and the lane pass ran."""
    shape = (3, 2011)
    lo, hi = synth.signed_range(b) if sgn else (0, (1 << b) - 1)
    a = _rand(b * 13 + sgn, shape, b, bool(sgn))
    c = _rand(b * 17 + sgn, shape, b, bool(sgn))
    if hit:
        a.flat[0], c.flat[0] = hi, hi
        a.flat[1], c.flat[1] = lo, lo
    else:  # both operands keep width b and sign; every sum fits b bits
        a, c = np.clip(a, lo // 2, hi // 2), np.clip(c, lo // 2, hi // 2)
        ext = lo if sgn else hi
        a.flat[0], c.flat[0] = ext, 0
        a.flat[1], c.flat[1] = 0, ext
    oa, oc = oracle.pack(a), oracle.pack(c)
    expect = oracle.add(oa, oc)
    pa = ccm.pack(to_dev(a), capacity=ccm.words_for(*shape, b))
    pc = ccm.pack(to_dev(c), capacity=ccm.words_for(*shape, b))
    out = ccm.PackedMatrix(*shape, ccm.words_for(*shape, cap or b + 1), device())
    ccm.add_into(pa, pc, out)
    assert_same_packed(out, expect, f"add lanes wide b={b} sgn={sgn} cap={cap} hit={hit}")
    same = (oa.width, oa.is_signed) == (oc.width, oc.is_signed)
    assert out.header().reserved1 == int(same), f"lane pass use b={b} sgn={sgn}"


@pytest.mark.parametrize("b,sgn", [(5, 0), (1, 0), (3, 0), (8, 0), (4, 1), (12, 1), (20, 0)])
@pytest.mark.parametrize("s", [7, -7, 8, 1, 0, 2, -1, 3000, -40000])
def test_scale_speculative_width(ccm, b, sgn, s):
    """One-pass scale: s times the range of A's width; the maximum entry at the
    range top (hit) and below it (the exact width may be smaller: second pass).
    For 1 <= |s| < 32 the lane pass writes C (see test_scale_lanes for the
    cases it takes); larger |s| and s = 0 take the general passes."""
    shape = (7, 2049)
    a = _rand(b * 3 + sgn, shape, b, bool(sgn))
    for top in (True, False):
        lo, hi = synth.signed_range(b) if sgn else (0, (1 << b) - 1)
        v = a.copy()
        if not top:
            v = np.clip(v, lo // 2 if sgn else 0, (hi // 2) + 1)
            v.flat[0] = (hi // 2) + 1
        oa = oracle.pack(v)
        expect = oracle.scale(oa, s)
        assert_same_packed(ccm.scale(ccm.pack(to_dev(v)), s), expect,
                           f"scale spec b={b} s={sgn} by {s} top={top}")


def _range_width(lo, hi):
    """Eq. 1 width of the values [lo, hi] (two's complement when lo < 0)."""
    h = max(hi, 0).bit_length()
    return max(h, 1) if lo >= 0 else 1 + max(h, (~lo).bit_length())


def _scale_lanes_expected(b, sgn, s, bs):
    """Whether the scale lane pass applies: 1 <= |s| < 32, A of at most 32
    bits, 1 <= bs - b <= 4 (every result then fits its bs-bit slot, or its
    64-bit value for 33..36-bit results), and not 1-bit signed A with
    s < 0."""
    t = abs(s)
    return 1 <= t < 32 and b <= 32 and 1 <= bs - b <= 4 and \
        not (sgn and b == 1 and s < 0)


@pytest.mark.parametrize("b,sgn", [(1, 0), (1, 1), (3, 0), (5, 0), (7, 1), (8, 1), (12, 1),
                                   (13, 0), (16, 1), (20, 1), (27, 1), (28, 0), (29, 1), (31, 1),
                                   (31, 0), (32, 1), (32, 0)])
@pytest.mark.parametrize("s", [2, -1, -2, 3, 7, -7, 8, -8, 15, -16, 31, -31])
def test_scale_lanes(ccm, b, sgn, s):
    """Scale through the lane pass (offset binary for signed A or negative s),
    output capacity at the speculative width so that the width class allows
    it: word-identical to the oracle with the range extremes present (one
    pass) and absent (the exact width is smaller: second pass), and the lane
    pass ran exactly where its conditions hold."""
    shape = (5, 3001)
    lo, hi = synth.signed_range(b) if sgn else (0, (1 << b) - 1)
    bs = _range_width(*sorted((s * lo, s * hi)))
    a = _rand(b * 5 + sgn + 3 * abs(s), shape, b, bool(sgn))
    for top in (True, False):
        v = a.copy()
        if top:
            v.flat[0], v.flat[-1] = lo, hi
        else:
            v = np.clip(v, lo // 2 if sgn else 0, hi // 2)
        oa = oracle.pack(v)
        expect = oracle.scale(oa, s)
        pa = ccm.pack(to_dev(v), capacity=ccm.words_for(*shape, b))
        out = ccm.PackedMatrix(*shape, ccm.words_for(*shape, min(bs, 64)), device())
        ccm.scale_into(pa, s, out)
        assert_same_packed(out, expect, f"scale lanes b={b} sgn={sgn} by {s} top={top}")
        # the speculative width follows A's packed width and sign
        alo, ahi = synth.signed_range(oa.width) if oa.is_signed else (0, (1 << oa.width) - 1)
        spec = _range_width(*sorted((s * alo, s * ahi)))
        n = shape[0] * shape[1]
        a_ok = min(pa.capacity * 32 // n, 64) <= 32  # the input's capacity bound
        lanes = a_ok and \
            _scale_lanes_expected(oa.width, oa.is_signed, s, spec)
        assert out.header().reserved1 == int(lanes), \
            f"lane pass use b={oa.width} sgn={oa.is_signed} s={s} spec={spec}"


@pytest.mark.parametrize("m,n", [(1, 128), (31, 256), (300, 384), (257, 1280), (1000, 128)])
@pytest.mark.parametrize("ba,bx,sa", [(1, 1, 0), (3, 8, 1), (5, 8, 0), (8, 8, 1), (12, 7, 1),
                                      (16, 8, 0), (17, 8, 1), (24, 16, 1), (31, 8, 0), (32, 8, 1),
                                      (32, 8, 0)])
def test_matvec_row_aligned(ccm, m, n, ba, bx, sa):
    """Row-aligned A (cols % 128 == 0): the streaming kernel vs the oracle."""
    a = _rand(m + n + ba, (m, n), ba, bool(sa))
    x = _rand(bx + n, (n, 1), bx)
    o = oracle.matvec(oracle.pack(a), oracle.pack(x))
    pa, px = _pack_cap(ccm, a, ba), _pack_cap(ccm, x, bx)
    y = ccm.matvec(pa, px, capacity=ccm.words_for(m, 1, 64))
    assert_same_packed(y, o, f"matvec aligned {m}x{n} b={ba}/{bx}")


def _x_kind(seed, n, kind):
    if kind == "s8":
        return _rand(seed, (n, 1), 8)
    if kind == "u7":
        return _rand(seed, (n, 1), 7, False)
    if kind == "u8":  # does not fit int8: the int32 path
        return _rand(seed, (n, 1), 8, False)
    return _rand(seed, (n, 1), 9)  # "s9", likewise


@pytest.mark.parametrize("ba", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("sa", [0, 1])
@pytest.mark.parametrize("xk", ["s8", "u7", "u8", "s9"])
def test_matvec_byte_lanes(ccm, ba, sa, xk):
    """Widths <= 8 with x in int8: the dp4a byte-lane path (offset binary for
    signed fields, x permuted for the widths 1, 2, 4), against the oracle; x
    that does not fit int8 takes the int32 path of the same kernel.  257 rows
    (a ragged last row block) by 1280 columns (several column slabs)."""
    m, n = 257, 1280
    a = _rand(ba * 31 + sa, (m, n), ba, bool(sa))
    x = _x_kind(ba + 7 * sa, n, xk)
    o = oracle.matvec(oracle.pack(a), oracle.pack(x))
    px = ccm.pack(to_dev(x))
    for cap in (ba, 16, 32):  # the width-class kernels for 8, 16 and 32 bits
        pa = _pack_cap(ccm, a, cap)
        y = ccm.matvec(pa, px, capacity=ccm.words_for(m, 1, 64))
        assert_same_packed(y, o, f"matvec byte lanes b={ba} s={sa} x={xk} cap={cap}")


@pytest.mark.parametrize("ba,sa", [(5, 0), (4, 1), (8, 1), (3, 1)])
def test_matvec_byte_lanes_large(ccm, ba, sa):
    """2048 x 8192 (64 stages per row, long slabs): byte-lane path."""
    m, n = 2048, 8192
    a = _rand(ba * 131 + sa, (m, n), ba, bool(sa))
    x = _rand(n, (n, 1), 8)
    o = oracle.matvec(oracle.pack(a), oracle.pack(x))
    y = ccm.matvec(ccm.pack(to_dev(a)), ccm.pack(to_dev(x)))
    assert_same_packed(y, o, f"matvec byte lanes {m}x{n} b={ba} s={sa}")


@pytest.mark.parametrize("m,n,ba,sa,xk", [(3, 262144, 5, 0, "s8"), (3, 262144, 3, 1, "s8"),
                                         (2, 262144, 4, 1, "u7"), (5, 65536, 12, 1, "s9"),
                                         (33, 131072, 8, 0, "u8")])
def test_matvec_long_rows(ccm, m, n, ba, sa, xk):
    """Rows too long for x to sit in shared memory whole: the column-slab
    kernel (x staged per slab, partial sums added per slab)."""
    a = _rand(n + ba, (m, n), ba, bool(sa))
    x = _x_kind(n + 1, n, xk)
    o = oracle.matvec(oracle.pack(a), oracle.pack(x))
    y = ccm.matvec(ccm.pack(to_dev(a)), ccm.pack(to_dev(x)), capacity=ccm.words_for(m, 1, 64))
    assert_same_packed(y, o, f"matvec long rows {m}x{n} b={ba} s={sa} x={xk}")


# ---------------------------------------------------------------------------
# Tensor-core matmul (exact 4-bit digit decomposition, e4m3 x e4m3 -> f32)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("b", [1, 4, 5, 8, 12, 16])
@pytest.mark.parametrize("m,k,n", [(128, 128, 128), (300, 520, 200), (129, 1, 257)])
def test_matmul_tensor_path(ccm, m, k, n, b):
    a, bm = _rand(m * 7 + b, (m, k), b), _rand(n * 5 + b, (k, n), b)
    o = oracle.matmul(oracle.pack(a), oracle.pack(bm))
    pa, pb = _pack_cap(ccm, a, b), _pack_cap(ccm, bm, b)
    c = ccm.matmul(pa, pb, path=ccm.MATMUL_TENSOR, capacity=ccm.words_for(m, n, 64))
    assert_same_packed(c, o, f"tensor matmul {m}x{k}x{n} b={b}")


def test_matmul_tensor_worst_case_sums(ccm):
    """Largest digit products in every class: all entries at the extremes of
    the signed 16-bit range, k = 4096, plus a half-large / half-small row
    that a narrow accumulator would round."""
    k = 4096
    a = np.full((128, k), 32767, dtype=np.int64)
    a[1::2] = -32768
    a[2, k // 2:] = 1
    bm = np.full((k, 64), 32767, dtype=np.int64)
    bm[:, 1::3] = -32768
    bm[k // 2:, 2] = 1
    rows = [0, 1, 2, 3, 127]
    expect = oracle.matmul_dense(a, bm, rows=rows)
    pa, pb = _pack_cap(ccm, a, 16), _pack_cap(ccm, bm, 16)
    c = ccm.matmul(pa, pb, path=ccm.MATMUL_TENSOR, capacity=ccm.words_for(128, 64, 64))
    got = ccm.unpack(c.check()).cpu().numpy()
    assert np.array_equal(got[rows], expect)


@pytest.mark.parametrize("b", [4, 8, 12, 16])
@pytest.mark.parametrize("m,k,n", [(130, 264, 72), (64, 512, 136)])
def test_matmul_tensor_unsigned_nibble_fields(ccm, m, k, n, b):
    """Unsigned fields of exactly 4L bits (the digit planes read straight
    from the stream's nibbles, the top digit unsigned), with the range ends
    present, and a signed B against an unsigned A."""
    a = _rand(m * 3 + b, (m, k), b, signed=False)
    bm = _rand(n * 5 + b, (k, n), b, signed=b != 8)
    o = oracle.matmul(oracle.pack(a), oracle.pack(bm))
    pa, pb = ccm.pack(to_dev(a)), ccm.pack(to_dev(bm))
    assert (pa.width, pa.is_signed) == (b, 0)
    c = ccm.matmul(pa, pb, path=ccm.MATMUL_TENSOR, capacity=ccm.words_for(m, n, 64))
    assert_same_packed(c, o, f"tensor matmul unsigned {m}x{k}x{n} b={b}")


def test_matmul_tensor_class_sums_cross_2_23(ccm):
    """Mixed-sign digits whose class sums rise above 2^23 within K and come
    back down: P = 32767 has digits (15, 15, 15, 7), N = -32753 has digits
    (15, 0, 0, -8).  For an even row times an even column the middle class
    gains 660 per step over the first 13,000 steps (8.58e6 > 2^23) and then
    loses 240 per step over the last 5,000; the fp32 accumulators are exact
    for every integer below 2^24 (k * 4 * 225 < 2^24 at k = 18,000), so the
    products must come out exact.  A sprinkle of random entries breaks the
    symmetry."""
    k1, k2 = 13000, 5000
    k = k1 + k2
    P, N = 32767, -32753
    a = np.empty((128, k), dtype=np.int64)
    a[0::2, :k1], a[0::2, k1:] = P, N
    a[1::2, :k2], a[1::2, k2:] = N, P
    bm = np.empty((k, 64), dtype=np.int64)
    bm[:k1, 0::2], bm[k1:, 0::2] = P, N
    bm[:k2, 1::2], bm[k2:, 1::2] = N, P
    noise_a = _rand(41, (128, k), 16)
    noise_b = _rand(42, (k, 64), 16)
    a[:, ::97] = noise_a[:, ::97]
    bm[::89, :] = noise_b[::89, :]
    expect = oracle.pack(oracle.matmul_dense(a, bm))
    pa, pb = _pack_cap(ccm, a, 16), _pack_cap(ccm, bm, 16)
    c = ccm.matmul(pa, pb, path=ccm.MATMUL_TENSOR, capacity=ccm.words_for(128, 64, 64))
    assert_same_packed(c, expect, "tensor matmul, class sums across 2^23")


def test_matmul_tensor_and_cudacore_agree(ccm):
    m, k, n = 384, 1000, 272
    for b in (4, 8, 13, 16):
        a, bm = _rand(b, (m, k), b), _rand(b + 1, (k, n), b)
        pa, pb = _pack_cap(ccm, a, b), _pack_cap(ccm, bm, b)
        ct = ccm.matmul(pa, pb, path=ccm.MATMUL_TENSOR)
        cc = ccm.matmul(pa, pb, path=ccm.MATMUL_CUDACORE)
        assert ct.check().width == cc.check().width
        assert np.array_equal(words_np(ct), words_np(cc))
        rows = [0, 191, 383]
        assert np.array_equal(ccm.unpack(ct).cpu().numpy()[rows],
                              oracle.matmul_dense(a, bm, rows=rows))
