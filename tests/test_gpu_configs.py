"""Parity at the workload configurations' full sizes, in the launch
configurations the bench uses: whole outputs where the oracle finishes in
seconds, sampled outputs otherwise (integer work: tolerance 0)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_packed, device, lib_ccm, to_dev, torch, words_np

pytestmark = pytest.mark.gpu

N = 8192


@pytest.fixture(scope="module")
def ccm():
    device()
    return lib_ccm()


@pytest.fixture(scope="module")
def count_matrices(ccm):
    """The default bench workload: 8192 x 8192 Poisson(5) A (seed 1303) and B
    (seed 1304), x signed 8-bit -- generated on the GPU exactly as the bench
    does, and on the host by the reference generator."""
    dev = device()
    table = torch.from_numpy(synth.poisson_cdf_table(5.0))
    A = ccm.gen_poisson(N * N, 1303, synth.STREAM_A, table, device=dev).view(N, N)
    B = ccm.gen_poisson(N * N, 1304, synth.STREAM_B, table, device=dev).view(N, N)
    X = ccm.gen_uniform(N, 1303, synth.STREAM_X, -128, 127, device=dev).view(N, 1)
    a = synth.count_matrix(1303, synth.STREAM_A, N, N)
    b = synth.count_matrix(1304, synth.STREAM_B, N, N)
    x = synth.uniform_int(1303, synth.STREAM_X, N, -128, 127).reshape(N, 1)
    assert np.array_equal(A.cpu().numpy(), a) and np.array_equal(X.cpu().numpy(), x)
    return A, B, X, a, b, x


def test_count_matrix_full_size(ccm, count_matrices):
    A, B, X, a, b, x = count_matrices
    oa, ob, ox = oracle.pack(a), oracle.pack(b), oracle.pack(x)
    pa, pb, px = ccm.pack(A), ccm.pack(B), ccm.pack(X)  # single-pass pack (workspace)
    assert_same_packed(pa, oa, "cfg2 pack A")
    assert_same_packed(pb, ob, "cfg2 pack B")
    assert pa.width == 5 and pa.is_signed == 0
    assert torch.equal(ccm.unpack(pa), A)
    idx = synth.uniform_int(1303, synth.STREAM_INDEX, 1 << 16, 0, N * N - 1)
    assert np.array_equal(ccm.get(pa, torch.from_numpy(idx)).cpu().numpy(), a.ravel()[idx])
    assert_same_packed(ccm.add(pa, pb), oracle.add(oa, ob), "cfg2 add")
    assert_same_packed(ccm.scale(pa, 7), oracle.scale(oa, 7), "cfg2 scale")
    assert_same_packed(ccm.matvec(pa, px), oracle.matvec(oa, ox), "cfg2 matvec")


@pytest.mark.parametrize("b", [1, 2, 3, 5, 8, 13, 16, 24, 31, 32])
def test_width_sweep(ccm, b):
    """Entries uniform over the signed b-bit range: pack/unpack, add, scale,
    matvec (rows sampled by the oracle for the larger widths)."""
    rows = N if b in (5, 32) else 1024
    a = synth.sweep_matrix(1303 + b, synth.STREAM_A, rows, N, b)
    bb = synth.sweep_matrix(1304 + b, synth.STREAM_B, rows, N, b)
    x = synth.x_vector(1303, N).reshape(N, 1)
    oa = oracle.pack(a)
    pa, pb, px = ccm.pack(to_dev(a)), ccm.pack(to_dev(bb)), ccm.pack(to_dev(x))
    assert_same_packed(pa, oa, f"sweep pack b={b}")
    assert np.array_equal(ccm.unpack(pa).cpu().numpy(), a)
    ob = oracle.pack(bb)
    # packed words, width, sign mode and padding of C against the oracle
    assert_same_packed(ccm.add(pa, pb), oracle.add(oa, ob), f"sweep add b={b}")
    assert_same_packed(ccm.scale(pa, -7), oracle.scale(oa, -7), f"sweep scale -7 b={b}")
    assert_same_packed(ccm.scale(pa, 7), oracle.scale(oa, 7), f"sweep scale 7 b={b}")
    y = ccm.unpack(ccm.matvec(pa, px).check()).cpu().numpy().ravel()
    sample = np.unique(synth.uniform_int(b, synth.STREAM_INDEX, 64, 0, rows - 1))
    assert np.array_equal(y[sample], oracle.matvec_dense(a, x.ravel(), rows=sample))


@pytest.mark.parametrize("b", [4, 8, 12, 16])
def test_matmul_4096(ccm, b):
    """4096^3 at b in {4, 8, 12, 16}: the tensor path's whole packed C (every
    word, exact width, sign mode, padding) equals the CUDA-core path's and the
    oracle's.  The oracle's product is the float64 BLAS one, exact here since
    |a| |b| k <= 2^15 * 2^15 * 2^12 < 2^53."""
    n = 4096
    dev = device()
    lo, hi = synth.signed_range(b)
    A = ccm.gen_uniform(n * n, 1303 + b, synth.STREAM_A, lo, hi, device=dev).view(n, n)
    B = ccm.gen_uniform(n * n, 1303 + b, synth.STREAM_B, lo, hi, device=dev).view(n, n)
    a = synth.uniform_signed(1303 + b, synth.STREAM_A, n * n, b).reshape(n, n)
    bm = synth.uniform_signed(1303 + b, synth.STREAM_B, n * n, b).reshape(n, n)
    assert np.array_equal(A.cpu().numpy(), a) and np.array_equal(B.cpu().numpy(), bm)
    pa, pb = ccm.pack(A), ccm.pack(B)
    del A, B
    ct = ccm.matmul(pa, pb, path=ccm.MATMUL_TENSOR)
    cc = ccm.matmul(pa, pb, path=ccm.MATMUL_CUDACORE, capacity=ct.capacity)
    expect = oracle.pack(oracle.matmul_dense_f64(a, bm))
    assert_same_packed(ct, expect, f"4096^3 tensor b={b}")
    assert_same_packed(cc, expect, f"4096^3 CUDA-core b={b}")
    # and the int64 product rows by the plain oracle loop
    rows = [0, 2047, 4095]
    assert np.array_equal(oracle.matmul_dense(a[rows], bm), oracle.unpack(expect)[rows])


def test_batch_10000(ccm):
    """The batched workload at full size: 10,000 matrices; sampled entries
    against the oracle, every entry against its own single call."""
    from paper_1303_0270_gb300.batch import BatchMatvec
    dev = device()
    count = 10000
    rows, cols, widths = synth.batch_shapes(1303, count)
    dense = torch.empty(int((rows * cols).max()), dtype=torch.int64, device=dev)
    xd = torch.empty(2048, dtype=torch.int64, device=dev)
    mats, xs = [], []
    for i in range(count):
        r, c_, w = int(rows[i]), int(cols[i]), int(widths[i])
        si = synth.batch_matrix_seed(1303, i)
        lo, hi = synth.signed_range(w)
        ccm.gen_uniform(r * c_, si, synth.STREAM_A, lo, hi, out=dense[: r * c_])
        mats.append(ccm.pack_into(dense[: r * c_].view(r, c_),
                                  ccm.PackedMatrix(r, c_, ccm.words_for(r, c_, w), dev)))
        ccm.gen_uniform(c_, si, synth.STREAM_X, -128, 127, out=xd[:c_])
        xs.append(ccm.pack_into(xd[:c_].view(c_, 1), ccm.PackedMatrix(c_, 1, ccm.words_for(c_, 1, 8), dev)))
    bm = BatchMatvec(mats, xs)
    bm.run()
    torch.cuda.synchronize()
    sample = synth.uniform_int(7, synth.STREAM_INDEX, 40, 0, count - 1)
    for i in sample:
        i = int(i)
        r, c_, w = int(rows[i]), int(cols[i]), int(widths[i])
        si = synth.batch_matrix_seed(1303, i)
        a = synth.uniform_signed(si, synth.STREAM_A, r * c_, w).reshape(r, c_)
        x = synth.uniform_int(si, synth.STREAM_X, c_, -128, 127).reshape(-1, 1)
        assert_same_packed(bm.ys[i], oracle.matvec(oracle.pack(a), oracle.pack(x)), f"batch {i}")
    for i in range(0, count, 97):
        single = ccm.matvec(mats[i], xs[i], capacity=bm.ys[i].capacity)
        assert np.array_equal(words_np(single), words_np(bm.ys[i]))
