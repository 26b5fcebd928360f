"""The seeded input generator against its published definitions."""
import math

import numpy as np

import synth


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 1234567: first five outputs of the published generator
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    got = [synth.mix_int(1234567 + k * synth.GAMMA) for k in range(1, 6)]
    assert got == expect


def test_counter_based_streams():
    a = synth.u64(1303, 0, 0, 1000)
    assert np.array_equal(synth.u64(1303, 0, 500, 500), a[500:])
    assert np.array_equal(synth.u64_at(1303, 0, np.array([3, 999, 0])), a[[3, 999, 0]])
    assert not np.array_equal(synth.u64(1303, 1, 0, 1000), a)
    assert not np.array_equal(synth.u64(1304, 0, 0, 1000), a)


def test_mulhi_matches_python_ints():
    rng = np.random.default_rng(0)
    u = rng.integers(0, 2**63, size=500, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    for r in (1, 7, 201, 2**32, 2**32 + 5, 2**63 + 12345, 2**64 - 1):
        got = synth.mulhi64(u, r)
        assert [int(v) for v in got] == [(int(x) * r) >> 64 for x in u]


def test_uniform_ranges():
    v = synth.uniform_int(1303, 0, 100000, -100, 100)
    assert v.min() == -100 and v.max() == 100
    for b in (1, 2, 8, 24, 32, 63, 64):
        lo, hi = synth.signed_range(b)
        v = synth.uniform_signed(5, 0, 20000, b)
        assert v.min() >= lo and v.max() <= hi


def test_poisson_table_and_moments():
    t = synth.poisson_cdf_table(5.0)
    assert math.isinf(t[-1]) and np.all(np.diff(t[:-1]) >= 0)
    assert abs(t[0] - math.exp(-5)) < 1e-15
    v = synth.poisson(1303, 0, 200000, 5.0)
    assert v.min() >= 0 and abs(v.mean() - 5.0) < 0.05 and abs(v.var() - 5.0) < 0.1


def test_batch_shapes():
    r, c, w = synth.batch_shapes(1303, 10000)
    assert r.min() >= 16 and r.max() < 2048 and c.min() >= 16 and c.max() < 2048
    assert w.min() == 1 and w.max() == 24
    # log-uniform: the median is near the geometric mean of the bounds
    assert 150 < np.median(r) < 210
