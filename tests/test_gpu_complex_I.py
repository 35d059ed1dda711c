"""GPU parity of Scheme I complex (4M) ZGEMM / CGEMM through the C ABI:
bit-exact against the oracle (reading R8) for INT8 and E4M3 slices, both
layouts, complex alpha/beta, beta = 0 with NaN in C, k = 0, and sampled rows
of a large product."""
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


CASES = [
    (130, 70, 90, 8, False, 0.5, 1),
    (64, 33, 300, 5, False, 2.0, 2),
    (33, 65, 700, 3, False, 1.0, 3),
    (200, 100, 150, 12, True, 1.0, 4),
    (65, 40, 3000, 11, True, 0.5, 5),   # 2K = 6000 > K_c(11) = 5888: two FP32-exact chunks
    (129, 31, 64, 6, True, 4.0, 6),
]


@pytest.mark.parametrize("m,n,k,p,f8,phi,seed", CASES)
def test_zgemm_4m_bit_exact(orc, h, m, n, k, p, f8, phi, seed):
    A, B = synth.gemm_pair_complex(m, n, k, phi, seed)
    C = emu.zgemm(dev(A), dev(B), scheme="I_F8" if f8 else "I", p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), orc.emu_Z4M_I(A, B, p, f8=f8))


@pytest.mark.parametrize("f8", [False, True])
def test_zgemm_4m_layouts_alpha_beta(orc, h, f8):
    m, n, k, p = 90, 75, 120, 7 if not f8 else 10
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 20)
    C0 = synth.test_matrix_complex(m, n, 1.0, 21)
    al, be = 0.75 - 0.5j, -1.0 + 0.25j
    sc = "I_F8" if f8 else "I"
    Cd = colmajor(C0)
    emu.zgemm(colmajor(A), colmajor(B), Cd, alpha=al, beta=be, scheme=sc, p=p, handle=h)
    assert np.array_equal(Cd.cpu().numpy(), orc.emu_Z4M_I(A, B, p, f8=f8, alpha=al, beta=be, C=C0))
    Cr = dev(C0)
    emu.zgemm(dev(A), dev(B), Cr, alpha=al, beta=be, scheme=sc, p=p, handle=h)
    assert np.array_equal(Cr.cpu().numpy(), orc.emu_Z4M_I(A, B, p, f8=f8, alpha=al, beta=be, C=C0))
    # beta = 0 with NaN in C: C is not read
    Cn = dev(np.full((m, n), np.nan + 1j * np.nan))
    emu.zgemm(dev(A), dev(B), Cn, alpha=al, beta=0.0, scheme=sc, p=p, handle=h)
    assert np.array_equal(Cn.cpu().numpy(), orc.emu_Z4M_I(A, B, p, f8=f8, alpha=al))


def test_zgemm_4m_k0_and_empty(orc, h):
    C0 = synth.test_matrix_complex(5, 4, 1.0, 30)
    A = torch.zeros((5, 0), dtype=torch.complex128, device="cuda")
    B = torch.zeros((0, 4), dtype=torch.complex128, device="cuda")
    Cd = dev(C0)
    emu.zgemm(A, B, Cd, alpha=2.0, beta=0.5 - 1.0j, scheme="I", p=4, handle=h)
    assert np.array_equal(Cd.cpu().numpy(), orc.emu_Z4M_I(np.zeros((5, 0)), np.zeros((0, 4)), 4, alpha=2.0,
                                                           beta=0.5 - 1.0j, C=C0))
    E = emu.zgemm(torch.zeros((0, 7), dtype=torch.complex128, device="cuda"),
                  torch.zeros((7, 3), dtype=torch.complex128, device="cuda"), scheme="I", p=4, handle=h)
    assert E.shape == (0, 3)


@pytest.mark.parametrize("f8,p", [(False, 4), (True, 6)])
def test_cgemm_4m_bit_exact(orc, h, f8, p):
    m, n, k = 100, 70, 200
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 40)
    Af, Bf = A.astype(np.complex64), B.astype(np.complex64)
    sc = "I_F8" if f8 else "I"
    C = emu.cgemm(dev(Af), dev(Bf), p=p, scheme=sc, handle=h)
    assert C.dtype == torch.complex64
    assert np.array_equal(C.cpu().numpy(), orc.emu_Z4M_I(Af, Bf, p, f8=f8, out_f32=True))
    C0 = synth.test_matrix_complex(m, n, 1.0, 41).astype(np.complex64)
    al, be = 0.5 + 0.5j, 2.0 - 1.0j
    Cd = dev(C0)
    emu.cgemm(dev(Af), dev(Bf), Cd, alpha=al, beta=be, p=p, scheme=sc, handle=h)
    assert np.array_equal(Cd.cpu().numpy(), orc.emu_Z4M_I(Af, Bf, p, f8=f8, alpha=al, beta=be, C=C0, out_f32=True))


def test_zgemm_4m_large_sampled_rows(orc, h):
    n, p = 2048, 12
    A, B = synth.gemm_pair_complex(n, n, n, 0.5, 77)
    C = emu.zgemm(dev(A), dev(B), scheme="I_F8", p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    rows = [3, 1500]
    assert np.array_equal(C[rows].cpu().numpy(), orc.emu_Z4M_I(A[rows], B, p, f8=True))


def test_zgemm_4m_accuracy_vs_double_double(orc, h):
    m = n = k = 256
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 90)
    ref = orc.dd_zgemm(A, B)
    e8 = orc.err_metric(emu.zgemm(dev(A), dev(B), scheme="I", p=8, handle=h).cpu().numpy(), ref, A, B)
    e12 = orc.err_metric(emu.zgemm(dev(A), dev(B), scheme="I_F8", p=12, handle=h).cpu().numpy(), ref, A, B)
    assert e8 <= 4 * 2 * k * 2.0 ** -53 and e12 <= 4 * 2 * k * 2.0 ** -53


def test_cgemm_3m_scheme_II_bit_exact(orc, h):
    m, n, k, nm = 120, 80, 150, 10
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 60)
    Af, Bf = A.astype(np.complex64), B.astype(np.complex64)
    C = emu.cgemm(dev(Af), dev(Bf), p=nm, scheme="II", handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), orc.emu_Z3M(Af, Bf, nm, out_f32=True))
    C0 = synth.test_matrix_complex(m, n, 1.0, 61).astype(np.complex64)
    al, be = -0.5 + 1.0j, 0.25 - 0.75j
    Cd = colmajor(C0)
    emu.cgemm(colmajor(Af), colmajor(Bf), Cd, alpha=al, beta=be, p=nm, scheme="II", handle=h)
    assert np.array_equal(Cd.cpu().numpy(), orc.emu_Z3M(Af, Bf, nm, alpha=al, beta=be, C=C0, out_f32=True))
