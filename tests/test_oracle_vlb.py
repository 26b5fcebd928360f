"""Pins of the VLB oracle (Method 2) against the paper's worked example
(Eq. 12-13), brute force and the efficiency formula Eq. 16/17 evaluated on
the bit-length groups of the data (an independent count)."""
import itertools

import numpy as np
import pytest

import oracle
from conftest import golden_lines
from oracle import efficiency as eff


def _golden():
    d = {}
    for ln in golden_lines("vlb_example_eq12.txt"):
        k, *v = ln.split()
        d[k] = v
    return d


def test_eq12_eq13_worked_example():
    g = _golden()
    entries = [int(v) for v in g["entries"]]
    v = oracle.vlb_pack(np.array(entries))
    assert v.k == int(g["prefix"][0])
    w = v.words.astype(np.uint64)
    word1 = int(w[0]) | (int(w[1]) << 32)
    word2 = int(w[2]) | (int(w[3]) << 32)
    assert word1 == int("".join(g["bitstring1"]), 2)
    assert word2 == int("".join(g["bitstring2"]), 2)
    assert v.nbits == 91  # the layout's own total (the text says 87)
    assert oracle.vlb_unpack(v).tolist() == entries


def test_vlb_round_trip_brute_force():
    for n in range(1, 5):
        for combo in itertools.product(range(0, 9), repeat=n):
            v = oracle.vlb_pack(np.array(combo))
            assert oracle.vlb_unpack(v).tolist() == list(combo)


def _stream_by_strings(values):
    """The VLB stream spelled out as text: for each entry its bit length L in
    k prefix bits, then the entry in L bits, each least significant bit first
    (the stream convention of Method 1, carried over to Method 2)."""
    lens = [max(1, int(v).bit_length()) for v in values]
    k = max(lens).bit_length()
    bits = ""
    for v, L in zip(values, lens):
        bits += format(L, f"0{k}b")[::-1] + format(int(v), f"0{L}b")[::-1]
    return k, bits


def test_vlb_stream_against_string_construction():
    for n in range(1, 5):
        for combo in itertools.product(range(0, 9), repeat=n):
            v = oracle.vlb_pack(np.array(combo))
            k, bits = _stream_by_strings(combo)
            assert (v.k, v.nbits) == (k, len(bits))
            got = "".join(format(int(w), "032b")[::-1] for w in v.words)
            assert got[:len(bits)] == bits and set(got[len(bits):]) <= {"0"}


def test_vlb_size_matches_eq16():
    rng = np.random.default_rng(3)
    for _ in range(50):
        lens = rng.integers(1, 40, size=200)
        vals = np.array([int(rng.integers(1 << (L - 1), 1 << L)) if L > 1 else int(rng.integers(0, 2))
                         for L in lens], dtype=np.int64)
        v = oracle.vlb_pack(vals)
        groups, freqs = np.unique(np.maximum(lens, 1), return_counts=True)
        eta2 = eff.eta2_groups(groups, freqs, v.k)
        assert eff.eta(64 * vals.size, v.nbits) == pytest.approx(eta2, abs=1e-12)
        assert v.k == int(lens.max()).bit_length()


def test_vlb_rejects_negative_and_handles_zero():
    with pytest.raises(ValueError):
        oracle.vlb_pack(np.array([3, -1]))
    v = oracle.vlb_pack(np.zeros(10, dtype=np.int64))
    assert v.k == 1 and v.nbits == 20  # prefix "1" and a 1-bit zero per entry
    assert not oracle.vlb_unpack(v).any()


def test_constant_bit_length_sm_smaller_than_vlb():
    """Figs 19-20: with constant bit lengths SM always needs fewer bits."""
    for b in range(1, 63):
        vals = np.full(100, (1 << b) - 1, dtype=np.int64)
        assert oracle.pack(vals.reshape(10, 10)).width * 100 < oracle.vlb_pack(vals).nbits
