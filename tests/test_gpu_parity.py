"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work (exponents, slices, residues, INT32 partials, per-modulus
residues) must be bit-exact.  Final floating-point results must be bit-exact
as well: the oracle fixes every rounding (one rounding of the exact
shift-reduce / CRT integer, then the BLAS update), so any difference is a
bug.  Sizes span several 64 x 32 output tiles and ragged edges.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_25453_gb300 as emu  # noqa: E402


@pytest.fixture(scope="module")
def h():
    hd = emu.Handle(0)
    yield hd
    hd.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def colmajor(x):
    """Same logical matrix stored column-major (Fortran order) on the GPU."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda()
    return t.t()


def deinterleave(hat: np.ndarray, rows: int, k: int, p: int) -> np.ndarray:
    """Eq. (11) layout back to digits [p, rows, k] (slice 0 signed, tails unsigned)."""
    nck = -(-k // 32)
    blk = hat[:rows, :nck * 32 * p].reshape(rows, nck, p, 32)
    d = np.transpose(blk, (2, 0, 1, 3)).reshape(p, rows, nck * 32)[:, :, :k]
    out = d.astype(np.uint8).astype(np.int16)
    out[0] = d[0].astype(np.int8).astype(np.int16)
    return out


# ---------------------------------------------------------------- split I
def padded(x, extra):
    """Row-major copy of x inside a buffer `extra` columns wider (leading
    dimension = columns + extra)."""
    buf = torch.zeros((x.shape[0], x.shape[1] + extra), dtype=torch.float64, device="cuda")
    buf[:, :x.shape[1]] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return buf[:, :x.shape[1]]


@pytest.mark.parametrize("p", [1, 3, 7, 8, 12])
@pytest.mark.parametrize("operand", [0, 1])
@pytest.mark.parametrize("col", [False, True, "padded"])
def test_split_I_bit_exact(orc, h, p, operand, col):
    # 77 x 101 with the minimal (odd) leading dimension takes the scalar
    # loads; "padded" gives an even leading dimension (16-byte loads) with a
    # ragged K tail and an odd vector count
    rows, k = 77, 101
    X = synth.test_matrix(rows, k, 4.0, 100 + p) if operand == 0 else synth.test_matrix(k, rows, 4.0, 100 + p)
    X[3] = 0.0 if operand == 0 else X[3]
    Xd = padded(X, 3) if col == "padded" else colmajor(X) if col else dev(X)
    hat, E = emu.split_I(Xd, p, operand=operand, handle=h)
    torch.cuda.synchronize()
    Xr = X if operand == 0 else X.T
    D = orc.split_I_rows(Xr, p)
    assert np.array_equal(E.cpu().numpy(), orc.row_exponents(Xr))
    hn = hat.cpu().numpy()
    assert np.array_equal(deinterleave(hn, rows, k, p), D)
    # padding rows and the K tail are zero
    assert not hn[rows:].any()
    nck = -(-k // 32)
    tail = hn[:rows].reshape(rows, nck, p, 32)[:, -1, :, k % 32:] if k % 32 else None
    if tail is not None:
        assert not tail.any()


# ---------------------------------------------------------------- partials / fused I
@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_partials_I_bit_exact(orc, h, p):
    m, n, k = 130, 97, 257
    A, B = synth.gemm_pair(m, n, k, 2.0, 7 + p)
    Cs = emu.partials_I(dev(A), dev(B), p, handle=h)
    ref = orc.partials_I(A, B, p)
    assert ref.shape[0] == 1
    assert np.array_equal(Cs.cpu().numpy().astype(np.int64), ref[0])


CASES_I = [
    # m, n, k, p, phi, seed
    (256, 256, 256, 7, 0.5, 0),     # the small workload of the method (p = 7, phi = 0.5, seed 0)
    (200, 130, 300, 3, 1.0, 1),
    (65, 33, 31, 1, 0.5, 2),
    (1, 1, 1, 4, 2.0, 3),
    (129, 70, 500, 8, 4.0, 4),
    (96, 64, 200, 12, 4.0, 5),
    (64, 40, 5000, 8, 2.0, 6),      # k > K_c(8) = 4608: two INT32 chunks
]


@pytest.mark.parametrize("m,n,k,p,phi,seed", CASES_I)
def test_dgemm_I_bit_exact(orc, h, m, n, k, p, phi, seed):
    A, B = synth.gemm_pair(m, n, k, phi, seed)
    C = emu.dgemm(dev(A), dev(B), scheme="I", p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    ref = orc.emu_I(A, B, p)
    got = C.cpu().numpy()
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


def test_dgemm_I_config1_accuracy(orc, h):
    """M = N = K = 256, phi = 0.5, seed 0, p = 7: within 4 k 2^-53 of the double-double product."""
    A, B = synth.gemm_pair(256, 256, 256, 0.5, 0)
    C = emu.dgemm(dev(A), dev(B), scheme="I", p=7, handle=h).cpu().numpy()
    err = orc.err_metric(C, orc.dd_gemm(A, B), A, B)
    assert err <= 4 * 256 * 2.0 ** -53, err


@pytest.mark.parametrize("col", [False, True])
def test_dgemm_I_alpha_beta_layouts(orc, h, col):
    m, n, k, p = 150, 90, 120, 6
    A, B = synth.gemm_pair(m, n, k, 1.0, 21)
    C0 = synth.test_matrix(m, n, 1.0, 22)
    wrap = colmajor if col else dev
    Cd = wrap(C0)
    emu.dgemm(wrap(A), wrap(B), Cd, alpha=-0.75, beta=1.5, scheme="I", p=p, handle=h)
    ref = orc.emu_I(A, B, p, alpha=-0.75, beta=1.5, C=C0)
    assert np.array_equal(Cd.cpu().numpy(), ref)
    # beta = 0 never reads C
    Cn = wrap(np.full((m, n), np.nan))
    emu.dgemm(wrap(A), wrap(B), Cn, alpha=2.0, beta=0.0, scheme="I", p=p, handle=h)
    assert np.array_equal(Cn.cpu().numpy(), orc.emu_I(A, B, p, alpha=2.0))


@pytest.mark.parametrize("p", [3, 4])
def test_sgemm_I_bit_exact(orc, h, p):
    m, n, k = 140, 72, 333
    A, B = synth.gemm_pair(m, n, k, 1.0, 30 + p, dtype=np.float32)
    C0 = synth.test_matrix(m, n, 1.0, 40, dtype=np.float32)
    Cd = dev(C0)
    emu.sgemm(dev(A), dev(B), Cd, alpha=1.25, beta=-0.5, scheme="I", p=p, handle=h)
    ref = orc.emu_I(A.astype(np.float64), B.astype(np.float64), p, alpha=1.25, beta=-0.5, C=C0,
                    out_f32=True)
    assert np.array_equal(Cd.cpu().numpy(), ref)


# ---------------------------------------------------------------- Scheme II
@pytest.mark.parametrize("nm", [1, 8, 15, 20])
@pytest.mark.parametrize("operand", [0, 1])
@pytest.mark.parametrize("shape", [(70, 150, 0), (71, 151, 5)])
def test_split_II_bit_exact(orc, h, nm, operand, shape):
    # even leading dimensions (16-byte loads); the second shape stores the
    # operand inside a wider buffer with an odd vector count and a ragged K tail
    rows, k, extra = shape
    X = synth.test_matrix(rows, k, 3.0, nm) if operand == 0 else synth.test_matrix(k, rows, 3.0, nm)
    res, E = emu.split_II(padded(X, extra) if extra else dev(X), nm, operand=operand, handle=h)
    Xr = X if operand == 0 else X.T
    b = orc.scale_bits_II(nm, k)
    ref = orc.residues_II_rows(Xr, nm, b)
    got = res.cpu().numpy()
    assert np.array_equal(got[:, :rows, :k], ref)
    assert not got[:, rows:].any() and not got[:, :, k:].any()
    assert np.array_equal(E.cpu().numpy(), orc.row_exponents(Xr))


@pytest.mark.parametrize("nm", [1, 5, 14, 20])
def test_residues_II_bit_exact(orc, h, nm):
    m, n, k = 100, 70, 300
    A, B = synth.gemm_pair(m, n, k, 2.0, 50 + nm)
    R = emu.residues_II(dev(A), dev(B), nm, handle=h).cpu().numpy()
    b = orc.scale_bits_II(nm, k)
    ref = orc.modprod_II(orc.residues_II_rows(A, nm, b), orc.residues_II_rows(B.T, nm, b))
    assert np.array_equal(R, ref)


CASES_II = [
    (256, 256, 256, 14, 0.5, 0),
    (130, 70, 300, 12, 4.0, 1),
    (65, 33, 50, 20, 1.0, 2),
    (1, 1, 1, 1, 1.0, 3),
    (97, 64, 1000, 16, 4.0, 4),
    (64, 32, 129, 7, 2.0, 5),
]


@pytest.mark.parametrize("m,n,k,nm,phi,seed", CASES_II)
def test_dgemm_II_bit_exact(orc, h, m, n, k, nm, phi, seed):
    A, B = synth.gemm_pair(m, n, k, phi, seed)
    C = emu.dgemm(dev(A), dev(B), scheme="II", p=nm, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    ref = orc.emu_II(A, B, nm)
    got = C.cpu().numpy()
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


def test_dgemm_II_alpha_beta_colmajor_and_f32(orc, h):
    m, n, k, nm = 90, 75, 140, 13
    A, B = synth.gemm_pair(m, n, k, 1.0, 60)
    C0 = synth.test_matrix(m, n, 1.0, 61)
    Cd = colmajor(C0)
    emu.dgemm(colmajor(A), colmajor(B), Cd, alpha=0.5, beta=-1.0, scheme="II", p=nm, handle=h)
    assert np.array_equal(Cd.cpu().numpy(), orc.emu_II(A, B, nm, alpha=0.5, beta=-1.0, C=C0))
    Af, Bf = A.astype(np.float32), B.astype(np.float32)
    Cf = emu.sgemm(dev(Af), dev(Bf), scheme="II", p=10, handle=h).cpu().numpy()
    assert np.array_equal(Cf, orc.emu_II(Af.astype(np.float64), Bf.astype(np.float64), 10, out_f32=True))


@pytest.mark.parametrize("m,n,k,nm,seed", [(96, 64, 128, 16, 0), (70, 45, 77, 12, 1), (1, 3, 5, 20, 2)])
def test_zgemm_3m_bit_exact(orc, h, m, n, k, nm, seed):
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, seed)
    C0 = synth.test_matrix_complex(m, n, 1.0, 90 + seed)
    Cd = dev(C0)
    emu.zgemm(dev(A), dev(B), Cd, alpha=0.5 - 1.0j, beta=0.25 + 0.5j, nm=nm, handle=h)
    ref = orc.emu_Z3M(A, B, nm, alpha=0.5 - 1.0j, beta=0.25 + 0.5j, C=C0)
    assert np.array_equal(Cd.cpu().numpy(), ref)


# ---------------------------------------------------------------- edge cases
def test_k_zero_and_empty(h):
    A = torch.empty((5, 0), dtype=torch.float64, device="cuda")
    B = torch.empty((0, 4), dtype=torch.float64, device="cuda")
    C = torch.full((5, 4), 3.0, dtype=torch.float64, device="cuda")
    emu.dgemm(A, B, C, alpha=2.0, beta=0.5, handle=h)
    assert torch.all(C == 1.5)
    emu.dgemm(A, B, C, alpha=2.0, beta=0.0, handle=h)
    assert torch.all(C == 0.0)
    E = torch.empty((0, 7), dtype=torch.float64, device="cuda")
    F = torch.empty((7, 3), dtype=torch.float64, device="cuda")
    out = emu.dgemm(E, F, handle=h)
    assert out.shape == (0, 3)


def test_nonfinite_sets_status(h):
    A = torch.ones((40, 30), dtype=torch.float64, device="cuda")
    B = torch.ones((30, 20), dtype=torch.float64, device="cuda")
    A[3, 4] = float("nan")
    emu.dgemm(A, B, handle=h, p=3)
    assert h.status() == 3  # EMU_ERR_NONFINITE
    A[3, 4] = 1.0
    B[2, 2] = float("inf")
    emu.dgemm(A, B, handle=h, scheme="II", p=8)
    assert h.status() == 3
    B[2, 2] = 1.0
    emu.dgemm(A, B, handle=h, p=3)
    assert h.status() == 0


def test_invalid_arguments(h):
    A = torch.ones((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(emu.EmuError) as e:
        emu.dgemm(A, A, scheme="I", p=13, handle=h)
    assert e.value.code == 2
    with pytest.raises(emu.EmuError) as e:
        emu.dgemm(A, A, scheme="II", p=21, handle=h)
    assert e.value.code == 2
    code = emu.emu_dgemm(h.h, 0, 4, 4, 4, 1.0, A.data_ptr(), 2, A.data_ptr(), 4, 0.0, A.data_ptr(), 4, 1, 3,
                         None)
    assert code == 1  # lda < k


def test_zero_rows_and_subnormals(orc, h):
    m, n, k = 40, 36, 64
    A, B = synth.gemm_pair(m, n, k, 1.0, 77)
    A[5] = 0.0
    B[:, 7] = 0.0
    A[9] *= 2.0 ** -1060  # subnormal / tiny row
    B[:, 3] *= 2.0 ** 900
    for scheme, p in (("I", 6), ("II", 15)):
        got = emu.dgemm(dev(A), dev(B), scheme=scheme, p=p, handle=h).cpu().numpy()
        ref = orc.emu_I(A, B, p) if scheme == "I" else orc.emu_II(A, B, p)
        assert np.array_equal(got, ref), scheme


# ---------------------------------------------------------------- full size, sampled
@pytest.mark.parametrize("scheme,p", [("I", 8), ("II", 15)])
def test_full_size_sampled_rows(orc, h, scheme, p):
    """n = 8192 (the benchmark size): a few sampled rows of C against the oracle,
    which computes row i of C from row i of A and all of B (scales are per row/col)."""
    n = 8192
    A, B = synth.gemm_pair(n, n, n, 2.0, 123)
    C = emu.dgemm(dev(A), dev(B), scheme=scheme, p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    rows = [0, 4097, 8191]
    got = C[rows].cpu().numpy()
    ref = orc.emu_I(A[rows], B, p) if scheme == "I" else orc.emu_II(A[rows], B, p)
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------- Scheme I on E4M3 slices
def e4m3_to_int(b: np.ndarray) -> np.ndarray:
    """Decode E4M3 bytes that hold integers (sign, exponent bias 7, 3-bit mantissa)."""
    b = b.astype(np.uint8).astype(np.int64)
    e = (b >> 3) & 15
    m = b & 7
    mag = np.where(e == 0, 0, ((8 + m) << np.maximum(e - 7, 0)) >> 3)
    return np.where(b & 0x80, -mag, mag)


@pytest.mark.parametrize("p", [1, 4, 11, 12])
@pytest.mark.parametrize("operand", [0, 1])
def test_split_F8_bit_exact(orc, h, p, operand):
    rows, k = 70, 77
    X = synth.test_matrix(rows, k, 4.0, 300 + p) if operand == 0 else synth.test_matrix(k, rows, 4.0, 300 + p)
    hat, E = emu.split_I(dev(X), p, operand=operand, handle=h, f8=True)
    Xr = X if operand == 0 else X.T
    hn = hat.cpu().numpy()
    nck = -(-k // 32)
    blk = hn[:rows, :nck * 32 * p].reshape(rows, nck, p, 32)
    got = e4m3_to_int(np.transpose(blk, (2, 0, 1, 3)).reshape(p, rows, nck * 32))
    assert np.array_equal(got[:, :, :k], orc.split_F8_rows(Xr, p))
    assert not got[:, :, k:].any() and not hn[rows:].any()
    assert np.array_equal(E.cpu().numpy(), orc.row_exponents(Xr))


@pytest.mark.parametrize("p", [2, 5, 11])
def test_partials_F8_bit_exact(orc, h, p):
    m, n, k = 130, 97, 1000
    A, B = synth.gemm_pair(m, n, k, 2.0, 20 + p)
    Cs = emu.partials_I(dev(A), dev(B), p, handle=h, f8=True)
    ref = orc.partials_F8(A, B, p)
    assert ref.shape[0] == 1
    assert np.array_equal(Cs.cpu().numpy().astype(np.int64), ref[0])


CASES_F8 = [
    (256, 256, 256, 11, 0.5, 0),
    (200, 130, 300, 4, 1.0, 1),
    (65, 33, 31, 1, 0.5, 2),
    (129, 70, 500, 12, 4.0, 4),
    (64, 40, 6000, 11, 2.0, 6),     # k > K_c(11) = 5888: two FP32-exact chunks
    (1000, 1000, 96, 12, 1.0, 7),   # several tiles per cluster of CTAs; 32 column tiles
    (300, 170, 64, 10, 0.5, 8),     # 6 column tiles: the last cluster group half empty
]


@pytest.mark.parametrize("m,n,k,p,phi,seed", CASES_F8)
def test_dgemm_F8_bit_exact(orc, h, m, n, k, p, phi, seed):
    A, B = synth.gemm_pair(m, n, k, phi, seed)
    C = emu.dgemm(dev(A), dev(B), scheme="I_F8", p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), orc.emu_F8(A, B, p))


def test_dgemm_F8_layouts_alpha_beta_f32(orc, h):
    m, n, k, p = 150, 90, 120, 9
    A, B = synth.gemm_pair(m, n, k, 1.0, 41)
    C0 = synth.test_matrix(m, n, 1.0, 42)
    Cd = colmajor(C0)
    emu.dgemm(colmajor(A), colmajor(B), Cd, alpha=1.5, beta=-0.25, scheme="I_F8", p=p, handle=h)
    assert np.array_equal(Cd.cpu().numpy(), orc.emu_F8(A, B, p, alpha=1.5, beta=-0.25, C=C0))
    Af, Bf = A.astype(np.float32), B.astype(np.float32)
    Cf = emu.sgemm(dev(Af), dev(Bf), scheme="I_F8", p=6, handle=h).cpu().numpy()
    assert np.array_equal(Cf, orc.emu_F8(Af.astype(np.float64), Bf.astype(np.float64), 6, out_f32=True))


def test_F8_full_size_sampled_rows(orc, h):
    n, p = 8192, 11
    A, B = synth.gemm_pair(n, n, n, 0.5, 321)
    C = emu.dgemm(dev(A), dev(B), scheme="I_F8", p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    rows = [1, 5000]
    assert np.array_equal(C[rows].cpu().numpy(), orc.emu_F8(A[rows], B, p))
