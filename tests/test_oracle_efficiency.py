"""Pins of the efficiency helpers against the paper's printed numbers
(Tables 3-5, the two-group table, the equal-probability groups and Eq. 45,
47 and 50) and against direct bit counting of packed matrices."""
import numpy as np
import pytest

import oracle
from conftest import golden_lines
from oracle import efficiency as eff

TOL = 1e-3  # the paper truncates or rounds to 3-4 decimals


def _rows(kind):
    return [ln.split()[1:] for ln in golden_lines("efficiency_tables.txt") if ln.split()[0] == kind]


def test_table3_uniform():
    for m, printed in _rows("uniform"):
        assert abs(eff.expected_eta2(eff.mean_uniform(int(m)), 7) - float(printed)) < TOL


def test_table4_binomial():
    for n, printed in _rows("binomial"):
        assert abs(eff.expected_eta2(eff.mean_binomial(int(n), 0.5), 7) - float(printed)) < TOL


def test_table5_poisson():
    for lam, printed in _rows("poisson"):
        assert abs(eff.expected_eta2(eff.mean_poisson(float(lam)), 7) - float(printed)) < TOL


def test_two_group_table_eq31():
    for p1, p2, printed in _rows("twogroup"):
        got = eff.eta2_probs([1, 64], [float(p1), float(p2)], k=7)
        assert abs(got - float(printed)) < TOL


def test_equal_probability_groups():
    for lengths, printed in _rows("groups"):
        bl = [int(v) for v in lengths.split(",")]
        got = eff.eta2_groups(bl, [1] * len(bl), k=7)
        assert abs(got - float(printed)) < TOL


def test_half_and_half_and_closed_forms():
    (printed,) = _rows("halfhalf")[0]
    assert abs(eff.eta2_groups([1, 64], [50, 50], 7) - float(printed)) < TOL
    assert abs(eff.expected_eta2(eff.mean_uniform(64)) - float(_rows("eq45")[0][0])) < TOL
    assert abs(eff.expected_eta2(eff.mean_binomial(64, 0.5)) - float(_rows("eq47")[0][0])) < TOL
    assert abs(eff.expected_eta2(eff.mean_poisson(32)) - float(_rows("eq50")[0][0])) < TOL


def test_eta1_eq15_limits_and_worked_example():
    assert eff.eta1(64) == 0.0
    assert eff.eta1(1) == 63 / 64
    # worked example: 8 fields at b = 10 use 80 of 512 bits
    assert eff.eta(512, 80) == eff.eta1(10)
    assert eff.vlb_prefix_width(10) == 4 and eff.vlb_prefix_width(64) == 7


def test_eta1_equals_counted_bits():
    """Eq. 15 against the bits the SM stream actually uses for a packed matrix."""
    rng = np.random.default_rng(0)
    for b in (1, 5, 10, 33):
        a = rng.integers(0, 1 << b, size=(40, 25))
        a[0, 0] = (1 << b) - 1
        p = oracle.pack(a)
        used = p.n * p.width
        assert eff.eta(64 * p.n, used) == pytest.approx(eff.eta1(b), abs=0)


def test_constant_bit_length_sm_beats_vlb():
    """Constant bit length (Figs 19-20): SM is better for every b < 64."""
    for b in range(1, 65):
        e1 = eff.eta1(b)
        e2 = eff.eta2_groups([b], [1], k=eff.vlb_prefix_width(b))
        assert e1 >= e2
        assert (e1 > e2) or b == 64 or eff.vlb_prefix_width(b) == 0
