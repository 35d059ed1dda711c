"""Pins of the FP8-slice Scheme I oracle (reading R7: beta = 5, balanced
base-32 digits stored as E4M3): digits reassemble exactly, every digit is an
exact E4M3 value (decoded here from the E4M3 definition), the FP32-exact
chunk bound by brute force, exactness on short integers, exact equality with
the rational triangle sum, and about 5 bits gained per slice."""
from fractions import Fraction

import numpy as np
import pytest

import synth
from test_oracle import exact_trunc, exp_by_definition


def e4m3_value(byte: int) -> float:
    """Value of an E4M3 byte: sign, 4-bit exponent (bias 7), 3-bit mantissa."""
    s = -1.0 if byte & 0x80 else 1.0
    e = (byte >> 3) & 0xF
    m = byte & 7
    if e == 0:
        return s * m / 8.0 * 2.0 ** -6
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


E4M3_INTS = {v for v in (e4m3_value(b) for b in range(256) if (b & 0x7F) != 0x7F) if v == int(v)}


@pytest.mark.parametrize("p", [1, 2, 4, 7, 11, 12])
def test_split_F8_digits(orc, p):
    A = synth.test_matrix(5, 13, 4.0, 40 + p)
    A[1] = 0.0
    E = orc.row_exponents(A)
    D = orc.split_F8_rows(A, p)
    assert D[0].min() >= -16 and D[0].max() <= 16
    if p > 1:
        assert D[1:].min() >= -16 and D[1:].max() <= 15
    assert set(np.unique(D).tolist()) <= E4M3_INTS
    for i in range(5):
        for h in range(13):
            x = exact_trunc(A[i, h], 5 * p - 1 - int(E[i]))
            assert sum(int(D[t, i, h]) * 32 ** (p - 1 - t) for t in range(p)) == x


@pytest.mark.parametrize("p", list(range(1, 13)))
def test_chunk_len_F8(orc, p):
    worst = max(sum(16 * 16 for _ in range(s + 1)) for s in range(p))
    kc = orc.chunk_len_F8(p)
    assert kc % 256 == 0 and kc * worst <= 2 ** 24 and (kc + 256) * worst > 2 ** 24


def test_F8_exact_on_short_integers(orc):
    """Integers |a| < 2^9 with each row/col max in [2^8, 2^9): x = a 2^10 at p = 4,
    so only digits 0 and 1 are nonzero and the p = 4 triangle keeps them all."""
    m, n, k = 6, 5, 40
    A = synth.integer_matrix(m, k, -511, 511, 3)
    B = synth.integer_matrix(k, n, -511, 511, 4)
    A[:, 0] = 300.0
    B[0, :] = -400.0
    C = orc.emu_F8(A, B, 4)
    ref = [[sum(int(A[i, h]) * int(B[h, j]) for h in range(k)) for j in range(n)] for i in range(m)]
    assert all(C[i, j] == ref[i][j] for i in range(m) for j in range(n))


def test_F8_triangle_rational(orc):
    for p, phi, seed in ((3, 1.0, 1), (11, 4.0, 2)):
        m, n, k = 3, 4, 29
        A, B = synth.gemm_pair(m, n, k, phi, seed)
        C = orc.emu_F8(A, B, p)
        DA = orc.split_F8_rows(A, p)
        DB = orc.split_F8_rows(B.T, p)
        for i in range(m):
            for j in range(n):
                S = sum(int(DA[t, i]. astype(np.int64) @ DB[s - t, j].astype(np.int64)) * 32 ** (p - 1 - s)
                        for s in range(p) for t in range(s + 1))
                E, F = exp_by_definition(A[i]), exp_by_definition(B[:, j])
                assert C[i, j] == float(Fraction(S) * Fraction(2) ** (E + F - 8 - 5 * (p - 1)))


def test_F8_error_falls_5_bits_per_slice(orc):
    m = n = k = 40
    A, B = synth.gemm_pair(m, n, k, 0.5, 8)
    ref = orc.dd_gemm(A, B)
    errs = {p: orc.err_metric(orc.emu_F8(A, B, p), ref, A, B) for p in range(2, 13)}
    for p in range(3, 10):
        assert errs[p + 1] <= errs[p] * 2.0 ** -3.5, errs
    assert errs[11] <= 4 * k * 2.0 ** -53 and errs[12] <= 2.0 ** -52
