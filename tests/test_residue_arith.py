"""The binary32 symmetric-residue step of the Scheme II split (bf16 planes)
takes the quotient as floor(RD(t inv + c)) with inv = RN(1/m) and
c = RN((off + 1/2)/m) and applies no correction.  That is exact only if
floor(t inv + c) = floor((t + off)/m) for every integer t the digit sums can
reach, |t| <= 16383 (1 + sum_{j>=1} |c_j|) with c_j the symmetric residue of
2^(14 j) mod m.  Checked here exhaustively, in exact integer arithmetic, for
every modulus of the list (Sec. IV-A: pairwise coprime moduli in the INT8
range) and 2, 4 and 6 digits; and the same check must fail without the half
in the offset (the reason it is there)."""
from fractions import Fraction

import numpy as np
import pytest


def _sym_pows(m, nd):
    hi = (m - 1) // 2
    out, v = [], 1 % m
    for _ in range(nd):
        out.append(v - m if v > hi else v)
        v = (v << 14) % m
    return out


def _mismatches(m, nd, half=True):
    off = m - 1 - (m - 1) // 2
    T = 16383 * (1 + sum(abs(c) for c in _sym_pows(m, nd)[1:]))
    assert T < 2 ** 24  # every partial sum of the FMA chain is an exact binary32 integer
    inv = Fraction(float(np.float32(1) / np.float32(m)))
    c = Fraction(float(np.float32(off + (0.5 if half else 0.0)) / np.float32(m)))
    den = max(inv.denominator, c.denominator)  # powers of two: the exact common denominator
    I, C = int(inv * den), int(c * den)
    assert T * I + C < 2 ** 62  # the int64 products below stay exact
    t = np.arange(-T, T + 1, dtype=np.int64)
    q = np.floor_divide(t * I + C, den)
    return int(np.count_nonzero(q != np.floor_divide(t + off, m)))


@pytest.mark.parametrize("nd", [2, 4, 6])
def test_quotient_exact_over_whole_range(orc, nd):
    for m in orc.moduli(20):
        assert _mismatches(m, nd) == 0, m


def test_offset_half_is_needed(orc):
    # with c = RN(off/m) the exact multiples of m (j = 0) can come out one low
    assert sum(_mismatches(m, 4, half=False) for m in orc.moduli(20)) > 0
