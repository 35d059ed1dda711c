"""Pins for the Scheme I complex (4M) oracle, reading R8: shared complex
row/column exponents, the four real triangle sums of Eq. (2) combined exactly
(the Im A x Im B term from the slices of -Im B), one rounding, the complex
BLAS update.  Checked against values fixed by other means: the real Scheme I
oracle on real inputs and on the real embedding of the complex product,
exact Gaussian-integer products, the error bound, and the update formula."""
from fractions import Fraction

import numpy as np
import pytest

import synth


def fma(a: float, b: float, c: float) -> float:
    return float(Fraction(a) * Fraction(b) + Fraction(c))


@pytest.mark.parametrize("f8,p", [(False, 3), (False, 7), (True, 5), (True, 11)])
def test_real_inputs_reduce_to_real_scheme_I(orc, f8, p):
    m, n, k = 13, 9, 41
    A, B = synth.gemm_pair(m, n, k, 2.0, 31)
    C = orc.emu_Z4M_I(A.astype(np.complex128), B.astype(np.complex128), p, f8=f8)
    ref = orc.emu_F8(A, B, p) if f8 else orc.emu_I(A, B, p)
    assert np.array_equal(C.real, ref)
    assert np.array_equal(C.imag, np.zeros_like(ref))


def _embed(A, B):
    """Real embedding: [Re A, Im A] (m x 2k) and the 2k x 2n matrix whose
    column 2j is [Re B_j; -Im B_j] and column 2j+1 is [Im B_j; Re B_j], so the
    real product holds (Re C, Im C) interleaved."""
    m, k = A.shape
    n = B.shape[1]
    Ae = np.concatenate([A.real, A.imag], axis=1)
    Be = np.empty((2 * k, 2 * n))
    Be[:k, 0::2], Be[k:, 0::2] = B.real, -B.imag
    Be[:k, 1::2], Be[k:, 1::2] = B.imag, B.real
    return Ae, Be


@pytest.mark.parametrize("f8,p", [(False, 4), (False, 8), (True, 8), (True, 12)])
def test_equals_scheme_I_on_the_real_embedding(orc, f8, p):
    m, n, k = 17, 11, 70
    A, B = synth.gemm_pair_complex(m, n, k, 3.0, 8)
    C = orc.emu_Z4M_I(A, B, p, f8=f8)
    Ae, Be = _embed(A, B)
    R = orc.emu_F8(Ae, Be, p) if f8 else orc.emu_I(Ae, Be, p)
    assert np.array_equal(C.real, R[:, 0::2])
    assert np.array_equal(C.imag, R[:, 1::2])


@pytest.mark.parametrize("f8,p", [(False, 3), (True, 4)])
def test_exact_on_gaussian_integers(orc, f8, p):
    m, n, k = 5, 4, 23
    rng = np.random.Generator(np.random.PCG64(21))
    A = rng.integers(-100, 101, (m, k)) + 1j * rng.integers(-100, 101, (m, k))
    B = rng.integers(-100, 101, (k, n)) + 1j * rng.integers(-100, 101, (k, n))
    C = orc.emu_Z4M_I(A, B, p, f8=f8)
    for i in range(m):
        for j in range(n):
            re = sum(int(A[i, h].real) * int(B[h, j].real) - int(A[i, h].imag) * int(B[h, j].imag)
                     for h in range(k))
            im = sum(int(A[i, h].real) * int(B[h, j].imag) + int(A[i, h].imag) * int(B[h, j].real)
                     for h in range(k))
            assert C[i, j] == complex(re, im)


@pytest.mark.parametrize("f8", [False, True])
def test_error_falls_to_fp64_level(orc, f8):
    m = n = k = 32
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 6)
    ref = orc.dd_zgemm(A, B)
    ps = (3, 5, 7, 8) if not f8 else (5, 8, 11, 12)
    errs = [orc.err_metric(orc.emu_Z4M_I(A, B, p, f8=f8), ref, A, B) for p in ps]
    bits_per_slice = 5 if f8 else 8
    # at least (bits per slice - 2) bits per slice until the binary64 floor
    assert errs[1] < errs[0] * 2.0 ** (-(bits_per_slice - 2) * (ps[1] - ps[0]))
    assert errs[-1] <= 4 * 2 * k * 2.0 ** -53


def test_alpha_beta_and_cgemm(orc):
    m, n, k, p = 12, 10, 30, 8
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 14)
    base = orc.emu_Z4M_I(A, B, p)
    C0 = synth.test_matrix_complex(m, n, 1.0, 15)
    al, be = 0.5 - 0.25j, 1.0 + 2.0j
    C = orc.emu_Z4M_I(A, B, p, alpha=al, beta=be, C=C0)
    for i in (0, 5, 11):
        for j in (0, 9):
            r, c = base[i, j], C0[i, j]
            tr = fma(al.real, r.real, -(al.imag * r.imag)) + fma(be.real, c.real, -(be.imag * c.imag))
            ti = fma(al.real, r.imag, al.imag * r.real) + fma(be.real, c.imag, be.imag * c.real)
            assert C[i, j] == complex(tr, ti)
    # beta = 0: C is not read (NaN in C has no effect)
    Cn = np.full((m, n), np.nan + 1j * np.nan)
    assert np.array_equal(orc.emu_Z4M_I(A, B, p, C=Cn), base)
    # CGEMM: complex64 inputs widened exactly, each component rounded once to binary32
    Af, Bf = A.astype(np.complex64), B.astype(np.complex64)
    Cf = orc.emu_Z4M_I(Af, Bf, 4, out_f32=True)
    ref = orc.emu_Z4M_I(Af.astype(np.complex128), Bf.astype(np.complex128), 4)
    assert Cf.dtype == np.complex64
    assert np.array_equal(Cf.real, ref.real.astype(np.float32))
    assert np.array_equal(Cf.imag, ref.imag.astype(np.float32))


def test_nonfinite_rejected(orc):
    A, B = synth.gemm_pair_complex(4, 3, 5, 1.0, 2)
    A[1, 2] = complex(0.0, np.inf)
    with pytest.raises(ValueError):
        orc.emu_Z4M_I(A, B, 4)
