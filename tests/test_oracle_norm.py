"""Pins for the norm-based Scheme II scaling (reading R9): the exponents bound
the row 2-norms (exactly, by rational arithmetic) and are tight on inputs
whose norm is known in closed form; the scaled operands satisfy the
exactness condition after Eq. (8) (checked with Python big integers); the
product is exact on integer inputs; and it keeps more bits than the
worst-case scaling of R3."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth


def exact_trunc(a: float, shift: int) -> int:
    q = Fraction(a) * (Fraction(2) ** shift)
    return int(q)


def test_norm_exponents_bound_the_norm(orc):
    for phi, seed in ((0.5, 1), (4.0, 2), (8.0, 3)):
        X = synth.test_matrix(12, 300, phi, seed)
        X[4] = 0.0
        E = orc.norm_exponents(X)
        for i in range(12):
            ss = sum(Fraction(v) ** 2 for v in X[i])
            if ss == 0:
                assert E[i] == 0
                continue
            assert ss < Fraction(4) ** int(E[i])
            # at most one above the smallest valid exponent (the integer upper
            # bound adds less than k units of 2^-64 to a scaled sum >= 1/4)
            assert ss >= Fraction(4) ** (int(E[i]) - 2)


def test_norm_exponents_closed_forms(orc):
    # single nonzero entry: the norm is |x|, e is its frexp exponent
    X = np.zeros((5, 7))
    vals = [3.0, -0.75, 1e-300, 2.0 ** 70, -(2.0 ** -1074)]
    for i, v in enumerate(vals):
        X[i, (3 * i) % 7] = v
    E = orc.norm_exponents(X)
    assert [int(e) for e in E] == [math.frexp(v)[1] for v in vals]
    # flat rows of 4^j equal powers of two: ||x|| = 2^(q+j) exactly, e = q + j + 1
    for q, j in ((0, 1), (-5, 3), (40, 5)):
        row = np.full((1, 4 ** j), 2.0 ** q)
        assert int(orc.norm_exponents(row)[0]) == q + j + 1


def test_norm_exponent_rounds_each_square_up(orc):
    # R9 sums ceil(y^2 2^64).  Row (x0, x1): x0 = 1 - 2^-26 gives E = 0 and
    # x0^2 2^64 = 2^64 - 2^39 + 2^12 exactly; x1 = M 2^-65 has x1^2 2^64 =
    # M^2 2^-66 in (T - 1, T], T = 2^39 - 2^12, with a fractional part.  The
    # rounded-up sum is exactly 2^64 (bit length 65, e = 1) although the
    # norm is below 1; squares rounded down would sum to 2^64 - 1 (e = 0).
    T = 2 ** 39 - 2 ** 12
    M = math.isqrt((T - 1) * 2 ** 66) + 1
    while M % 2 == 0:
        M += 1
    assert 2 ** 52 <= M < 2 ** 53 and (T - 1) * 2 ** 66 < M * M <= T * 2 ** 66
    x0, x1 = 1.0 - 2.0 ** -26, M * 2.0 ** -65
    assert Fraction(x0) ** 2 * 2 ** 64 == 2 ** 64 - 2 ** 39 + 2 ** 12
    assert Fraction(x0) ** 2 + Fraction(x1) ** 2 < 1
    assert list(orc.norm_exponents(np.array([[x0, x1], [x1, x0]]))) == [1, 1]


def test_norm_halves(orc):
    for nm in range(2, 21):
        hA, hB = orc.norm_halves_II(nm)
        # equal halves, the largest with 2 (2^hA 2^hB) <= 2^floor(log2 P)
        assert hA == hB and 2 * hA + 1 <= orc.log2P_floor(nm) < 2 * hA + 3


@pytest.mark.parametrize("nm,phi", [(8, 4.0), (14, 8.0), (20, 0.5)])
def test_exactness_condition_holds(orc, nm, phi):
    m, n, k = 6, 5, 257
    A, B = synth.gemm_pair(m, n, k, phi, 40 + nm)
    A[2, :100] = 0.0
    E, F = orc.norm_exponents(A), orc.norm_exponents(B.T)
    hA, hB = orc.norm_halves_II(nm)
    P = math.prod(orc.moduli(nm))
    Ap = [[exact_trunc(A[i, h], hA - int(E[i])) for h in range(k)] for i in range(m)]
    Bp = [[exact_trunc(B[h, j], hB - int(F[j])) for h in range(k)] for j in range(n)]
    for i in range(m):
        for j in range(n):
            assert 2 * sum(abs(x) * abs(y) for x, y in zip(Ap[i], Bp[j])) < P


def test_exact_on_integers(orc):
    rng = np.random.Generator(np.random.PCG64(8))
    A = rng.integers(-1000, 1001, (7, 40)).astype(np.float64)
    B = rng.integers(-1000, 1001, (40, 6)).astype(np.float64)
    C = orc.emu_II(A, B, 12, norm=True)
    exact = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(C, exact.astype(np.float64))


def test_more_bits_than_worst_case_scaling(orc):
    m = n = 24
    k = 2048
    A, B = synth.gemm_pair(m, n, k, 4.0, 12)
    ref = orc.dd_gemm(A, B)
    gains = []
    for nm in (10, 12, 14, 16):
        e3 = orc.err_metric(orc.emu_II(A, B, nm), ref, A, B)
        e9 = orc.err_metric(orc.emu_II(A, B, nm, norm=True), ref, A, B)
        assert e9 <= e3
        gains.append(math.log2(e3 / e9))
    assert np.mean(gains) >= 3.0
    assert orc.err_metric(orc.emu_II(A, B, 20, norm=True), ref, A, B) <= 4 * k * 2.0 ** -53


def test_complex_norm_exponents_bound_the_norm(orc):
    # complex rows use |x|^2 = re^2 + im^2; rows 0-2 have imaginary parts
    # much larger than the real ones, row 3 the reverse, row 4 is zero
    rng = np.random.Generator(np.random.PCG64(21))
    X = rng.uniform(-1, 1, (5, 40)) * 2.0 ** -20 + 1j * rng.uniform(-1, 1, (5, 40)) * 2.0 ** 5
    X[3] = X[3].imag * 2.0 ** -25 + 1j * X[3].real * 2.0 ** 25
    X[4] = 0.0
    E = orc.norm_exponents(X, True)
    for i in range(5):
        ss = sum(Fraction(v.real) ** 2 + Fraction(v.imag) ** 2 for v in X[i])
        if ss == 0:
            assert E[i] == 0
            continue
        assert Fraction(4) ** (int(E[i]) - 2) <= ss < Fraction(4) ** int(E[i])


def test_complex_3m_norm(orc):
    rng = np.random.Generator(np.random.PCG64(13))
    A = rng.integers(-300, 301, (5, 30)) + 1j * rng.integers(-300, 301, (5, 30))
    B = rng.integers(-300, 301, (30, 4)) + 1j * rng.integers(-300, 301, (30, 4))
    assert np.array_equal(orc.emu_Z3M(A, B, 12, norm=True), A @ B)
    # exactness of the real and imaginary sums with the complex norms
    m, n, k, nm = 4, 3, 129, 10
    A, B = synth.gemm_pair_complex(m, n, k, 4.0, 14)
    E, F = orc.norm_exponents(A, True), orc.norm_exponents(np.ascontiguousarray(B.T), True)
    hA, hB = orc.norm_halves_II(nm)
    P = math.prod(orc.moduli(nm))
    for i in range(m):
        for j in range(n):
            ar = [exact_trunc(A[i, h].real, hA - int(E[i])) for h in range(k)]
            ai = [exact_trunc(A[i, h].imag, hA - int(E[i])) for h in range(k)]
            br = [exact_trunc(B[h, j].real, hB - int(F[j])) for h in range(k)]
            bi = [exact_trunc(B[h, j].imag, hB - int(F[j])) for h in range(k)]
            re = sum(x * y - u * v for x, y, u, v in zip(ar, br, ai, bi))
            im = sum(x * v + u * y for x, y, u, v in zip(ar, br, ai, bi))
            assert 2 * abs(re) < P and 2 * abs(im) < P
    ref = orc.dd_zgemm(A, B)
    e3 = orc.err_metric(orc.emu_Z3M(A, B, 14), ref, A, B)
    e9 = orc.err_metric(orc.emu_Z3M(A, B, 14, norm=True), ref, A, B)
    assert e9 <= e3
    # complex64 output is the complex128 result rounded once per part
    Cf = orc.emu_Z3M(A, B, 14, norm=True, out_f32=True)
    Cz = orc.emu_Z3M(A, B, 14, norm=True)
    assert np.array_equal(Cf.real, Cz.real.astype(np.float32)) and np.array_equal(Cf.imag, Cz.imag.astype(np.float32))
