"""Compression efficiency of the SM and VLB methods -- TEST INFRASTRUCTURE ONLY.

Plain float64 restatements of the paper's efficiency formulas (Compression
Efficiency section and the Discussion):

* Eq. 14: eta = (bits allocated - bits used) / bits allocated.
* Eq. 15: SM against 64-bit storage, eta_1 = (64 - b) / 64.
* Eq. 16 / 17: VLB with g bit-length groups of sizes f_i and prefix width k,
  eta_2 = 1 - sum_i b_i f_i / (64 r c) - k / 64.
* Eq. 29: the same with group probabilities p_i = f_i / (r c).
* Eq. 20 / 21: expected efficiencies from an expected bit length E(b).
* Eq. 44, 47, 49: E(b) of a discrete uniform U(1, m), a binomial B(n, p) and a
  Poisson(lambda) bit-length distribution (k fixed at 7, the bit length of 64).
"""
from __future__ import annotations

import numpy as np


def eta(bits_allocated: float, bits_used: float) -> float:
    """Eq. 14."""
    return (bits_allocated - bits_used) / bits_allocated


def eta1(b: int, word: int = 64) -> float:
    """Eq. 15 (word = 64); word = 32 gives the same ratio against int32 storage."""
    return eta(float(word), float(b))


def eta2_groups(bit_lengths, freqs, k: int) -> float:
    """Eq. 17 from the group bit lengths b_i and their frequencies f_i."""
    b = np.asarray(bit_lengths, dtype=np.float64)
    f = np.asarray(freqs, dtype=np.float64)
    rc = f.sum()
    return 1.0 - float((b * f).sum()) / (64.0 * rc) - k / 64.0


def eta2_probs(bit_lengths, probs, k: int = 7) -> float:
    """Eq. 29 with p_i = f_i / (r c) (Eq. 30)."""
    b = np.asarray(bit_lengths, dtype=np.float64)
    p = np.asarray(probs, dtype=np.float64)
    return 1.0 - float((b * p).sum()) / 64.0 - k / 64.0


def expected_eta1(k: int) -> float:
    """Eq. 20."""
    return 1.0 - k / 64.0


def expected_eta2(mean_bit_length: float, k: int = 7) -> float:
    """Eq. 21 / Eq. 44."""
    return 1.0 - mean_bit_length / 64.0 - k / 64.0


def mean_uniform(m: int) -> float:
    """E(b) for b ~ U(1, m) (Discrete Uniform section)."""
    return (1 + m) / 2.0


def mean_binomial(n: int, p: float) -> float:
    """E(b) = n p (Eq. 47)."""
    return n * p


def mean_poisson(lam: float) -> float:
    """E(b) = lambda (Eq. 49)."""
    return float(lam)


def vlb_prefix_width(max_bit_length: int) -> int:
    """k = bit length of the largest bit length (VLB section; 64 -> 7, 10 -> 4)."""
    return int(max_bit_length).bit_length()
