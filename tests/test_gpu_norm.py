"""Scheme II with norm-based scaling (EMU_SCHEME_II_NORM) on the GPU: bit-exact
against the oracle (reading R9) for real and 3M complex products, both
layouts, FP32, zero and subnormal rows, K spread over many segments of the
norm scan, and sampled rows of a large product."""
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
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().t()


CASES = [(130, 70, 90, 12, 0.5, 1), (64, 33, 5000, 16, 4.0, 2), (200, 129, 300, 8, 8.0, 3),
         (33, 65, 4097, 20, 2.0, 4)]


@pytest.mark.parametrize("m,n,k,nm,phi,seed", CASES)
def test_dgemm_norm_bit_exact(orc, h, m, n, k, nm, phi, seed):
    A, B = synth.gemm_pair(m, n, k, phi, seed)
    A[3] = 0.0
    A[5, : k // 2] = 2.0 ** -1060  # subnormal entries in a row with normal ones
    B[:, 2] = 0.0
    C = emu.dgemm(dev(A), dev(B), scheme="II_NORM", p=nm, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), orc.emu_II(A, B, nm, norm=True))
    # column-major, alpha/beta
    C0 = synth.test_matrix(m, n, 1.0, seed + 10)
    Cd = colmajor(C0)
    emu.dgemm(colmajor(A), colmajor(B), Cd, alpha=0.5, beta=-1.5, scheme="II_NORM", p=nm, handle=h)
    assert np.array_equal(Cd.cpu().numpy(), orc.emu_II(A, B, nm, alpha=0.5, beta=-1.5, C=C0, norm=True))


def test_sgemm_norm(orc, h):
    A, B = synth.gemm_pair(100, 80, 700, 4.0, 20, dtype=np.float32)
    C = emu.sgemm(dev(A), dev(B), scheme="II_NORM", p=10, handle=h)
    ref = orc.emu_II(A.astype(np.float64), B.astype(np.float64), 10, out_f32=True, norm=True)
    assert np.array_equal(C.cpu().numpy(), ref)


def test_complex_norm(orc, h):
    m, n, k = 90, 70, 3000
    A, B = synth.gemm_pair_complex(m, n, k, 4.0, 30)
    Z = emu.zgemm(dev(A), dev(B), nm=14, scheme="II_NORM", handle=h)
    assert np.array_equal(Z.cpu().numpy(), orc.emu_Z3M(A, B, 14, norm=True))
    Af, Bf = A.astype(np.complex64), B.astype(np.complex64)
    Cf = emu.cgemm(dev(Af), dev(Bf), p=10, scheme="II_NORM", handle=h)
    assert np.array_equal(Cf.cpu().numpy(), orc.emu_Z3M(Af, Bf, 10, norm=True, out_f32=True))
    Zc = colmajor(np.zeros((m, n), np.complex128))
    emu.zgemm(colmajor(A), colmajor(B), Zc, alpha=1 - 1j, nm=12, scheme="II_NORM", handle=h)
    assert np.array_equal(Zc.cpu().numpy(), orc.emu_Z3M(A, B, 12, alpha=1 - 1j, norm=True))


def test_norm_large_sampled_rows_and_gain(orc, h):
    n, nm = 4096, 14
    A, B = synth.gemm_pair(n, n, n, 4.0, 77)
    Ad, Bd = dev(A), dev(B)
    C = emu.dgemm(Ad, Bd, scheme="II_NORM", p=nm, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    rows = [0, 2049]
    assert np.array_equal(C[rows].cpu().numpy(), orc.emu_II(A[rows], B, nm, norm=True))
    # the norm bound keeps more bits than the worst-case scaling at the same N
    Cw = emu.dgemm(Ad, Bd, scheme="II", p=nm, handle=h)
    cols = np.arange(0, n, 64)
    ref = orc.dd_gemm(A[rows], B[:, cols])
    e_norm = orc.err_metric(C[rows][:, cols].cpu().numpy(), ref, A[rows], B[:, cols])
    e_worst = orc.err_metric(Cw[rows][:, cols].cpu().numpy(), ref, A[rows], B[:, cols])
    assert e_norm < e_worst / 8
