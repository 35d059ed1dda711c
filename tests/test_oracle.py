"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: exact
rationals (fractions.Fraction), Python big integers, textbook integer GEMM
on inputs where the method must be exact, closed-form bounds, invariants, and
the few values the paper prints (tests/golden/paper_facts.txt).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_facts.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, val = line.split(":", 1)
        out[key.strip()] = val.split()
    return out


def fma(a: float, b: float, c: float) -> float:
    """Correctly rounded a*b + c (Fraction -> float rounds to nearest, ties to even)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def exact_trunc(a: float, shift: int) -> int:
    """trunc(a * 2^shift) with exact rational arithmetic."""
    q = Fraction(a) * (Fraction(2) ** shift)
    return int(q)  # int() truncates toward zero


def exp_by_definition(vals) -> int:
    """Smallest integer E with max |v| < 2^E, by search (0 for all zeros)."""
    mx = max((abs(Fraction(v)) for v in vals), default=Fraction(0))
    if mx == 0:
        return 0
    E = -1100
    while not (mx < Fraction(2) ** E):
        E += 1
    return E


# ------------------------------------------------------------ scaling
def test_row_exponents_definition(orc):
    A = synth.test_matrix(9, 13, 4.0, 3)
    A[2, :] = 0.0
    A[3, :5] = 2.0 ** -1070  # subnormal row maximum
    A[3, 5:] = 0.0
    A[4, 0] = 1.0  # exact power of two: 1 < 2^1
    E = orc.row_exponents(A)
    for i in range(A.shape[0]):
        assert E[i] == exp_by_definition(A[i]), i
    F = orc.col_exponents(A)
    for j in range(A.shape[1]):
        assert F[j] == exp_by_definition(A[:, j]), j


def test_row_exponents_nonfinite(orc):
    A = np.ones((3, 4))
    A[1, 2] = np.inf
    with pytest.raises(ValueError):
        orc.row_exponents(A)
    A[1, 2] = np.nan
    with pytest.raises(ValueError):
        orc.row_exponents(A)


# ------------------------------------------------------------ Scheme I split
@pytest.mark.parametrize("p", [1, 2, 3, 5, 7, 8, 10])
def test_split_I_digits_reassemble(orc, p):
    """Eq. (1) with beta = 8: digits are the bytes of x = trunc(a 2^(8p-1-E))."""
    A = synth.test_matrix(6, 11, 4.0, 11 + p)
    A[0, 3] = -A[0, 3]
    A[1, :] = 0.0
    E = orc.row_exponents(A)
    D = orc.split_I_rows(A, p)
    assert D.shape == (p, 6, 11)
    assert D[0].min() >= -128 and D[0].max() <= 127
    if p > 1:
        assert D[1:].min() >= 0 and D[1:].max() <= 255
    for i in range(6):
        for h in range(11):
            x = exact_trunc(A[i, h], 8 * p - 1 - int(E[i]))
            assert abs(x) < 2 ** (8 * p - 1)
            rec = sum(int(D[t, i, h]) * 256 ** (p - 1 - t) for t in range(p))
            assert rec == x, (i, h)
            # a ~= 2^(E-7) sum_t 2^-8t D_t with a truncation residual below one unit
            approx = Fraction(2) ** (int(E[i]) - 7) * sum(Fraction(int(D[t, i, h]), 256 ** t) for t in range(p))
            res = Fraction(A[i, h]) - approx
            assert abs(res) < Fraction(2) ** (int(E[i]) - 8 * p + 1)
            assert res == 0 or (res > 0) == (A[i, h] > 0)


def test_interleave_layout_paper_example(orc):
    """Eq. (11) and its p = 3 example: [A'0|A'1|A'2|A'0|A'1|A'2|...]."""
    g = golden()
    order = [int(v) for v in g["interleave_p3_block_order"]]
    p, rows, k, tk = 3, 2, 64, 32
    D = np.zeros((p, rows, k), dtype=np.int16)
    for t in range(p):
        D[t] = 10 * (t + 1)  # slice t marked by value 10(t+1)
    D[:, :, 32:] += 1  # second K-chunk marked by +1
    hat = orc.interleave(D, tk)
    assert hat.shape == (rows, p * k)
    for blk in range(2 * p):
        vals = hat[:, blk * tk:(blk + 1) * tk]
        t = order[blk]
        chunk = blk // p
        assert np.all(vals == 10 * (t + 1) + chunk), blk


def test_interleave_pads_ragged_k(orc):
    D = np.arange(2 * 3 * 40, dtype=np.int16).reshape(2, 3, 40) % 100
    hat = orc.interleave(D, 32)
    assert hat.shape == (3, 2 * 64)
    # chunk 1 holds k = 32..39 then zeros, for both slices
    assert np.all(hat[:, 2 * 32 + 8:3 * 32] == 0)
    assert np.all(hat[:, 3 * 32 + 8:] == 0)
    assert np.array_equal(hat[:, 2 * 32:2 * 32 + 8], D[0, :, 32:40].astype(np.int8))


# ------------------------------------------------------------ Scheme I chunks
@pytest.mark.parametrize("p", list(range(1, 11)))
def test_chunk_len_is_safe_and_maximal(orc, p):
    """K_c keeps every C_s of Eq. (2) inside int32, by brute force over the digit ranges."""
    lo = {0: -128}
    hi = {0: 127}
    worst = 0
    for s in range(p):
        pos = neg = 0
        for t in range(s + 1):
            ra = (lo.get(t, 0), hi.get(t, 255))
            rb = (lo.get(s - t, 0), hi.get(s - t, 255))
            prods = [x * y for x in ra for y in rb]
            pos += max(prods)
            neg += min(prods)
        worst = max(worst, pos, -neg)
    kc = orc.chunk_len_I(p)
    assert kc % 256 == 0 and kc > 0
    assert kc * worst <= 2 ** 31 - 1
    assert (kc + 256) * worst > 2 ** 31 - 1


# ------------------------------------------------------------ Scheme I partials / full
def test_partials_I_brute_force(orc):
    p, m, n, k, kc = 3, 3, 4, 40, 16
    A, B = synth.gemm_pair(m, n, k, 2.0, 5)
    Cs = orc.partials_I(A, B, p, kc)
    E = [exp_by_definition(A[i]) for i in range(m)]
    F = [exp_by_definition(B[:, j]) for j in range(n)]

    def digits(x, p):
        u = x % (256 ** p)  # two's complement bits of x (Python's % is nonnegative)
        d = [(u >> (8 * (p - 1 - t))) & 0xFF for t in range(p)]
        if d[0] >= 128:
            d[0] -= 256
        return d

    DA = [[digits(exact_trunc(A[i, h], 8 * p - 1 - E[i]), p) for h in range(k)] for i in range(m)]
    DB = [[digits(exact_trunc(B[h, j], 8 * p - 1 - F[j]), p) for h in range(k)] for j in range(n)]
    nch = -(-k // kc)
    assert Cs.shape == (nch, p, m, n)
    for c in range(nch):
        for s in range(p):
            for i in range(m):
                for j in range(n):
                    ref = sum(DA[i][h][t] * DB[j][h][s - t]
                              for t in range(s + 1) for h in range(c * kc, min(k, (c + 1) * kc)))
                    assert Cs[c, s, i, j] == ref


def _int_matmul(A, B):
    m, k = A.shape
    n = B.shape[1]
    return [[sum(int(A[i, h]) * int(B[h, j]) for h in range(k)) for j in range(n)] for i in range(m)]


def test_scheme_I_exact_on_short_integers(orc):
    """Integers |a| < 2^15 with each row/col max in [2^14, 2^15): only slices 0 and 1
    are nonzero, so p = 4 keeps every nonzero pair and Eq. (3) gives A@B exactly."""
    m, n, k = 7, 5, 33
    A = synth.integer_matrix(m, k, -(2 ** 15 - 1), 2 ** 15 - 1, 21)
    B = synth.integer_matrix(k, n, -(2 ** 15 - 1), 2 ** 15 - 1, 22)
    A[:, 0] = 2 ** 15 - 1
    B[0, :] = -(2 ** 15 - 1)
    C = orc.emu_I(A, B, 4)
    ref = _int_matmul(A, B)
    for i in range(m):
        for j in range(n):
            assert C[i, j] == float(ref[i][j])


def test_scheme_I_p1_is_integer_gemm(orc):
    """p = 1 on integers with row/col max in [64, 128): x = a, one INT8 GEMM, exact."""
    m, n, k = 6, 9, 50
    A = synth.integer_matrix(m, k, -127, 127, 1)
    B = synth.integer_matrix(k, n, -127, 127, 2)
    A[:, 3] = 100.0
    B[7, :] = -90.0
    C = orc.emu_I(A, B, 1)
    ref = _int_matmul(A, B)
    assert all(C[i, j] == ref[i][j] for i in range(m) for j in range(n))


def test_scheme_I_triangle_rational(orc):
    """Full Scheme I result == the exact rational triangle sum of Eqs. (2)-(3),
    rounded once to nearest (the shift-reduce adds no error, Sec. III-B)."""
    for p, phi, seed in ((3, 1.0, 9), (5, 4.0, 10), (8, 2.0, 11)):
        m, n, k = 4, 3, 37
        A, B = synth.gemm_pair(m, n, k, phi, seed)
        C = orc.emu_I(A, B, p)
        Cs = orc.partials_I(A, B, p, 16)  # chunking must not matter
        E = orc.row_exponents(A)
        F = orc.col_exponents(B)
        for i in range(m):
            for j in range(n):
                exact = sum(Fraction(int(Cs[c, s, i, j]), 256 ** s) for c in range(Cs.shape[0]) for s in range(p))
                exact *= Fraction(2) ** (int(E[i]) + int(F[j]) - 14)
                assert C[i, j] == float(exact), (p, i, j)


def test_scheme_I_alpha_beta_and_f32(orc):
    m, n, k = 5, 6, 17
    A, B = synth.gemm_pair(m, n, k, 0.5, 3)
    C0 = synth.test_matrix(m, n, 0.5, 99)
    base = orc.emu_I(A, B, 5)
    C = orc.emu_I(A, B, 5, alpha=-1.5, beta=0.25, C=C0)
    assert np.array_equal(C, np.array([[fma(-1.5, base[i, j], 0.25 * C0[i, j]) for j in range(n)]
                                       for i in range(m)]))
    # beta == 0 never reads C: NaN in C is ignored
    Cn = np.full((m, n), np.nan)
    assert np.array_equal(orc.emu_I(A, B, 5, alpha=2.0, beta=0.0, C=Cn), 2.0 * base)
    Cf = orc.emu_I(A.astype(np.float32), B.astype(np.float32), 3, out_f32=True)
    ref = orc.emu_I(A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64), 3)
    assert Cf.dtype == np.float32 and np.array_equal(Cf, ref.astype(np.float32))


def test_scheme_I_chunk_boundary_matches_single_chunk_in_exact_sum(orc):
    """Chunked partials summed over chunks equal the unchunked partials (Eq. 2)."""
    p, m, n, k = 2, 3, 3, 70
    A, B = synth.gemm_pair(m, n, k, 2.0, 17)
    a = orc.partials_I(A, B, p, 16).sum(axis=0)
    b = orc.partials_I(A, B, p, 256)[0]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("phi", [0.5, 4.0])
def test_scheme_I_error_falls_8_bits_per_slice(orc, phi):
    """Table II: each slice adds about beta = 8 bits until the binary64 level.

    The error is measured against |A||B|; row/column scaling costs bits when
    phi is large (wide exponent range inside a row), so the per-slice gain is
    checked from the first p where the leading slices resolve the data."""
    m = n = k = 48
    A, B = synth.gemm_pair(m, n, k, phi, 5)
    ref = orc.dd_gemm(A, B)
    errs = {p: orc.err_metric(orc.emu_I(A, B, p), ref, A, B) for p in range(1, 11)}
    first = 2 if phi < 1 else 4
    for p in range(first, 8):
        assert errs[p + 1] <= errs[p] * 2.0 ** -6, (p, errs)
    if phi < 1:
        assert errs[1] > errs[2] > errs[3]
    if phi < 1:
        assert errs[7] <= 4 * k * 2.0 ** -53  # p = 7 meets the FP64-level bound
    else:
        assert errs[10] <= 4 * k * 2.0 ** -53  # wide exponent range needs more slices
    assert errs[10] <= 2.0 ** -50  # exact shift-reduce: converges to the binary64 level


# ------------------------------------------------------------ Scheme II
def test_moduli_paper_prefix_and_pairwise_coprime(orc):
    g = golden()
    ms = orc.moduli(24)
    assert ms[:3] == [int(v) for v in g["moduli_prefix"]]
    assert all(math.gcd(a, b) == 1 for i, a in enumerate(ms) for b in ms[i + 1:])
    assert ms == sorted(ms, reverse=True) and ms[0] == 256
    # greedy: every skipped integer shares a factor with an earlier chosen modulus
    for x in range(ms[-1], 257):
        if x not in ms:
            assert any(math.gcd(x, y) > 1 for y in ms if y > x), x


def test_log2P_and_scale_bits(orc):
    for nm in range(1, 21):
        P = math.prod(orc.moduli(nm))
        assert orc.log2P_floor(nm) == P.bit_length() - 1
        for k in (1, 2, 3, 255, 256, 257, 4096, 8192, 16384):
            for cplx in (False, True):
                b = orc.scale_bits_II(nm, k, cplx)
                terms = 2 * k if cplx else k
                if b >= 1:
                    # exactness condition after Eq. (8): 2 sum |a'||b'| < P for |a'|,|b'| <= 2^b - 1
                    assert 2 * terms * (2 ** b - 1) ** 2 < P
                # b is the largest with the power-of-two form 2^(2b+1+ceil(log2 terms)) <= 2^floor(log2 P)
                c = (terms - 1).bit_length()
                assert 2 * b + 1 + c <= P.bit_length() - 1
                assert 2 * (b + 1) + 1 + c > P.bit_length() - 1


def test_residues_II_definition(orc):
    nm, k = 6, 9
    A = synth.test_matrix(4, k, 3.0, 8)
    b = orc.scale_bits_II(nm, k)
    E = orc.row_exponents(A)
    R = orc.residues_II_rows(A, nm, b)
    for l, m in enumerate(orc.moduli(nm)):
        for i in range(4):
            for h in range(k):
                x = exact_trunc(A[i, h], b - int(E[i]))
                r = int(R[l, i, h])
                assert -(m // 2) <= r <= (m - 1) // 2
                assert (r - x) % m == 0


def test_crt_matches_python_bigints(orc):
    """Eq. (8) + symmetric lift + round-to-nearest: vs Python int -> float
    (correctly rounded, ties to even)."""
    rng = np.random.Generator(np.random.PCG64(4))
    for nm in (1, 2, 5, 12, 15, 20):
        ms = orc.moduli(nm)
        P = math.prod(ms)
        vals = [int(rng.integers(0, 2 ** 62)) * int(rng.integers(1, 2 ** 62)) * int(rng.integers(1, 2 ** 40))
                for _ in range(200)]
        vals = [v % P for v in vals]
        vals = [v - P if 2 * v > P else v for v in vals]
        vals += [0, 1, -1, (P - 1) // 2, -((P - 1) // 2)]
        if P.bit_length() > 63:  # ties at 53 bits: 2^60 + 2^7 rounds to even (down), 2^60 + 3*2^7 up
            vals += [2 ** 60 + 2 ** 7, 2 ** 60 + 3 * 2 ** 7, -(2 ** 60 + 2 ** 7), 2 ** 60 + 2 ** 7 + 1]
        res = np.array([[v % m for v in vals] for m in ms], dtype=np.uint8)
        out = orc.crt(res)
        for v, o in zip(vals, out):
            assert o == float(v), (nm, v, o)


def test_modprod_II_brute_force(orc):
    nm, m, n, k = 5, 3, 4, 30
    A, B = synth.gemm_pair(m, n, k, 2.0, 3)
    b = orc.scale_bits_II(nm, k)
    RA = orc.residues_II_rows(A, nm, b)
    RB = orc.residues_II_rows(B.T, nm, b)
    O = orc.modprod_II(RA, RB)
    E = orc.row_exponents(A)
    F = orc.col_exponents(B)
    Ai = [[exact_trunc(A[i, h], b - int(E[i])) for h in range(k)] for i in range(m)]
    Bi = [[exact_trunc(B[h, j], b - int(F[j])) for j in range(n)] for h in range(k)]
    for l, ml in enumerate(orc.moduli(nm)):
        for i in range(m):
            for j in range(n):
                # Eq. (4): (A'B') mod m == ((A' mod m)(B' mod m)) mod m
                full = sum(Ai[i][h] * Bi[h][j] for h in range(k))
                assert int(O[l, i, j]) == full % ml


def test_scheme_II_exact_on_integers(orc):
    """Integer inputs with b >= E: a' = a 2^(b-E) exactly, CRT recovers A'B' exactly,
    and the inverse scaling returns A@B (textbook integer GEMM)."""
    m, n, k = 6, 7, 25
    A = synth.integer_matrix(m, k, -1000, 1000, 31)
    B = synth.integer_matrix(k, n, -1000, 1000, 32)
    for nm in (6, 9, 14):
        assert orc.scale_bits_II(nm, k) >= 10
        C = orc.emu_II(A, B, nm)
        ref = _int_matmul(A, B)
        assert all(C[i, j] == ref[i][j] for i in range(m) for j in range(n)), nm


@pytest.mark.parametrize("phi", [0.5, 4.0])
def test_scheme_II_error_falls_with_moduli(orc, phi):
    """log2 P grows ~7.7 bits per modulus and b by half of that: the error falls
    about 7.7 bits per two moduli until the binary64 level."""
    m = n = k = 40
    A, B = synth.gemm_pair(m, n, k, phi, 6)
    ref = orc.dd_gemm(A, B)
    errs = {nm: orc.err_metric(orc.emu_II(A, B, nm), ref, A, B) for nm in range(6, 21, 2)}
    first = 6 if phi < 1 else 8
    last = 12 if phi < 1 else 18
    for nm in range(first, last + 1, 2):
        assert errs[nm + 2] <= errs[nm] * 2.0 ** -6, errs
    assert errs[20] <= 4 * k * 2.0 ** -53
    if phi < 1:
        assert errs[16] <= 4 * k * 2.0 ** -53


def test_scheme_II_alpha_beta(orc):
    m, n, k = 4, 5, 12
    A, B = synth.gemm_pair(m, n, k, 1.0, 7)
    C0 = synth.test_matrix(m, n, 1.0, 70)
    base = orc.emu_II(A, B, 14)
    C = orc.emu_II(A, B, 14, alpha=0.75, beta=-2.0, C=C0)
    assert np.array_equal(C, np.array([[fma(0.75, base[i, j], -2.0 * C0[i, j]) for j in range(n)]
                                       for i in range(m)]))


# ------------------------------------------------------------ 3M complex
def test_3m_residues_equal_4m(orc):
    """Eq. (16): 3M residues equal the 4M residues exactly in modular arithmetic."""
    nm, m, n, k = 4, 3, 3, 11
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 2)
    b = orc.scale_bits_II(nm, k, True)
    Bt = np.ascontiguousarray(B.T)
    A3 = [orc.residues_Z_rows(A, nm, b, q) for q in range(3)]
    B3 = [orc.residues_Z_rows(Bt, nm, b, q) for q in range(3)]
    ORe, OIm = orc.modprod_Z3M(A3, B3)
    E = orc.row_exponents_z(A)
    F = orc.row_exponents_z(Bt)
    for l, ml in enumerate(orc.moduli(nm)):
        for i in range(m):
            for j in range(n):
                re = im = 0
                for h in range(k):
                    ar = exact_trunc(A[i, h].real, b - int(E[i]))
                    ai = exact_trunc(A[i, h].imag, b - int(E[i]))
                    br = exact_trunc(B[h, j].real, b - int(F[j]))
                    bi = exact_trunc(B[h, j].imag, b - int(F[j]))
                    re += ar * br - ai * bi
                    im += ar * bi + ai * br
                assert int(ORe[l, i, j]) == re % ml and int(OIm[l, i, j]) == im % ml


def test_3m_exact_on_complex_integers(orc):
    m, n, k = 5, 4, 19
    rng = np.random.Generator(np.random.PCG64(12))
    A = rng.integers(-500, 501, (m, k)) + 1j * rng.integers(-500, 501, (m, k))
    B = rng.integers(-500, 501, (k, n)) + 1j * rng.integers(-500, 501, (k, n))
    C = orc.emu_Z3M(A, B, 12)
    for i in range(m):
        for j in range(n):
            re = sum(int(A[i, h].real) * int(B[h, j].real) - int(A[i, h].imag) * int(B[h, j].imag) for h in range(k))
            im = sum(int(A[i, h].real) * int(B[h, j].imag) + int(A[i, h].imag) * int(B[h, j].real) for h in range(k))
            assert C[i, j] == complex(re, im)


def test_3m_error_and_alpha_beta(orc):
    m = n = k = 24
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 4)
    ref = orc.dd_zgemm(A, B)
    errs = [orc.err_metric(orc.emu_Z3M(A, B, nm), ref, A, B) for nm in (8, 12, 16, 20)]
    assert errs[1] < errs[0] * 2.0 ** -10 and errs[2] < errs[1] * 2.0 ** -10
    assert errs[3] <= 4 * k * 2.0 ** -53
    base = orc.emu_Z3M(A, B, 16)
    C0 = synth.test_matrix_complex(m, n, 1.0, 5)
    C = orc.emu_Z3M(A, B, 16, alpha=0.5 - 0.25j, beta=1.0 + 2.0j, C=C0)
    al, be = 0.5 - 0.25j, 1.0 + 2.0j
    for i in (0, 7, 23):
        for j in (0, 11):
            r, c = base[i, j], C0[i, j]
            tr = fma(al.real, r.real, -(al.imag * r.imag)) + fma(be.real, c.real, -(be.imag * c.imag))
            ti = fma(al.real, r.imag, al.imag * r.real) + fma(be.real, c.imag, be.imag * c.real)
            assert C[i, j] == complex(tr, ti)


# ------------------------------------------------------------ double-double reference
def test_dd_gemm_vs_exact_rationals(orc):
    for seed, phi in ((1, 0.5), (2, 4.0), (3, 8.0)):
        m, n, k = 4, 5, 8
        A, B = synth.gemm_pair(m, n, k, phi, seed)
        A[0, :4] = [1e16, 1.0, -1e16, 3.0]  # adversarial cancellation
        B[:4, 0] = [1.0, 1.0, 1.0, 1.0]
        hi, lo = orc.dd_gemm(A, B)
        for i in range(m):
            for j in range(n):
                ex = sum(Fraction(A[i, h]) * Fraction(B[h, j]) for h in range(k))
                den = sum(abs(Fraction(A[i, h]) * Fraction(B[h, j])) for h in range(k))
                assert abs(Fraction(hi[i, j]) + Fraction(lo[i, j]) - ex) <= den * Fraction(2) ** -100


@pytest.mark.parametrize("seed,phi,cancel", [(8, 2.0, False), (9, 8.0, False), (10, 0.5, True), (11, 4.0, True)])
def test_dd_zgemm_vs_exact_rationals(orc, seed, phi, cancel):
    # k = 4 complex terms: 2k = 8 real products per part, so the compensated
    # dot product errs by at most gamma_8^2 ~ 8^2 2^-106 = 2^-100 of the
    # part's own sum of |products| (Ogita-Rump-Oishi Dot2, unevaluated hi + lo)
    m, n, k = 3, 4, 4
    A, B = synth.gemm_pair_complex(m, n, k, phi, seed)
    if cancel:  # real and imaginary parts both cancel to small integers
        A[0, :4] = [1e16 + 3j, 1.0 + 1e16j, -1e16 + 2j, 3.0 - 1e16j]
        B[:4, 0] = [1.0 + 1.0j] * 4
        A[1, :4] = [2.0 ** 60 + 1j, -1.0 + 2.0 ** 60 * 1j, -(2.0 ** 60) + 1j, 5.0 - 2.0 ** 60 * 1j]
        B[:4, 1] = [1.0 - 1.0j, 1.0 + 1.0j, 1.0 - 1.0j, 1.0 + 1.0j]
    hi, lo = orc.dd_zgemm(A, B)
    F = Fraction
    tight = F(2) ** -100 * (1 + F(2) ** -40)
    for i in range(m):
        for j in range(n):
            ar = [F(A[i, h].real) for h in range(k)]
            ai = [F(A[i, h].imag) for h in range(k)]
            br = [F(B[h, j].real) for h in range(k)]
            bi = [F(B[h, j].imag) for h in range(k)]
            re = sum(ar[h] * br[h] - ai[h] * bi[h] for h in range(k))
            im = sum(ar[h] * bi[h] + ai[h] * br[h] for h in range(k))
            den_re = sum(abs(ar[h] * br[h]) + abs(ai[h] * bi[h]) for h in range(k))
            den_im = sum(abs(ar[h] * bi[h]) + abs(ai[h] * br[h]) for h in range(k))
            assert abs(F(hi[i, j].real) + F(lo[i, j].real) - re) <= den_re * tight
            assert abs(F(hi[i, j].imag) + F(lo[i, j].imag) - im) <= den_im * tight
    if cancel:
        assert hi[0, 0] + lo[0, 0] == -1.0 + 9.0j


def test_golden_gemm_counts():
    g = golden()
    assert [p * (p + 1) // 2 for p in range(1, 9)] == [int(v) for v in g["scheme_I_int8_gemms"]]
    assert (8 + 1) / 2 == float(g["fusion_intensity_gain_p8"][0])


def test_3m_cgemm_is_zgemm_rounded_once(orc):
    """CGEMM by 3M: the complex64 inputs widened exactly, the update in
    binary64, each part rounded once to binary32."""
    m, n, k = 14, 9, 33
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 51)
    Af, Bf = A.astype(np.complex64), B.astype(np.complex64)
    Aw, Bw = Af.astype(np.complex128), Bf.astype(np.complex128)
    C0 = synth.test_matrix_complex(m, n, 1.0, 52).astype(np.complex64)
    for al, be in ((1.0, 0.0), (0.5 - 2.0j, 1.5 + 0.25j)):
        Cf = orc.emu_Z3M(Af, Bf, 10, alpha=al, beta=be, C=C0, out_f32=True)
        Cz = orc.emu_Z3M(Aw, Bw, 10, alpha=al, beta=be, C=C0.astype(np.complex128))
        assert Cf.dtype == np.complex64
        assert np.array_equal(Cf.real, Cz.real.astype(np.float32))
        assert np.array_equal(Cf.imag, Cz.imag.astype(np.float32))
