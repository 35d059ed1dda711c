"""emu_dgemm_noalloc: the allocation-free Scheme I DGEMM.

Callers that may not allocate device memory while they run (a program whose
device memory is reserved by its own pool, latency-critical code that cannot
take cudaMalloc's implicit synchronisation, a plugin whose host forbids
allocation) use this entry point; its scratch is a fixed device array inside
the library.  The test calls it through the C ABI twice in a row -- the
second call finds the first call's data still in the shared array -- and
checks both results bit for bit against emu_dgemm, the tolerance used by the
other parity tests.  The file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_25453_gb300 as emu  # noqa: E402


def _noalloc(A, B, C, p, alpha=1.0, beta=0.0, status=None):
    m, k = A.shape
    n = B.shape[1]
    stream = torch.cuda.current_stream().cuda_stream
    return emu.emu_dgemm_noalloc(emu.EMU_ROW_MAJOR, m, n, k, alpha, A.data_ptr(), max(k, 1), B.data_ptr(),
                                 max(n, 1), beta, C.data_ptr(), max(n, 1), p,
                                 None if status is None else status.data_ptr(), stream)


def _colmajor_padded(x, pad):
    """The matrix x stored column-major with leading dimension rows + pad:
    returns (storage tensor, leading dimension)."""
    r, c = x.shape
    buf = np.full((c, r + pad), np.nan)
    buf[:, :r] = x.T
    return torch.from_numpy(buf).cuda(), r + pad


def test_noalloc_matches_emu_dgemm_twice():
    h = emu.Handle(0)
    cases = [(300, 200, 700, 8, 2.0, 1), (1024, 1024, 1024, 7, 0.5, 2)]
    for m, n, k, p, phi, seed in cases:
        A, B = synth.gemm_pair(m, n, k, phi, seed)
        Ad = torch.from_numpy(A).cuda()
        Bd = torch.from_numpy(B).cuda()
        ref = emu.dgemm(Ad, Bd, scheme="I", p=p, handle=h)
        torch.cuda.synchronize()
        assert h.status() == 0
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        for call in range(2):  # second call reuses the array left by the first
            C = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
            assert _noalloc(Ad, Bd, C, p, status=status) == 0
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            assert torch.equal(C, ref), (m, n, k, p, call)
    h.close()


def test_noalloc_alpha_beta_and_limits():
    h = emu.Handle(0)
    m, n, k, p = 130, 90, 257, 6
    A, B = synth.gemm_pair(m, n, k, 1.0, 5)
    C0 = synth.test_matrix(m, n, 1.0, 6)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ref = torch.from_numpy(C0).cuda()
    emu.dgemm(Ad, Bd, ref, alpha=-0.5, beta=2.0, scheme="I", p=p, handle=h)
    for _ in range(2):
        C = torch.from_numpy(C0).cuda()
        assert _noalloc(Ad, Bd, C, p, alpha=-0.5, beta=2.0) == 0
        torch.cuda.synchronize()
        assert torch.equal(C, ref)
    # a product whose scratch exceeds the fixed array is rejected, nothing runs
    big = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
    out = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
    assert _noalloc(big, big, out, 8) == 2  # EMU_ERR_UNSUPPORTED
    h.close()


def test_noalloc_against_oracle_colmajor_padded(orc):
    # column-major A, B, C with leading dimensions larger than the minimum
    # (the call maps the product onto the transposed row-major one)
    h = emu.Handle(0)
    m, n, k, p = 150, 97, 333, 7
    A, B = synth.gemm_pair(m, n, k, 2.0, 21)
    C0 = synth.test_matrix(m, n, 1.0, 22)
    Ad, lda = _colmajor_padded(A, 5)
    Bd, ldb = _colmajor_padded(B, 3)
    want = orc.emu_I(A, B, p, alpha=1.5, beta=-0.25, C=C0)
    stream = torch.cuda.current_stream().cuda_stream
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        Cd, ldc = _colmajor_padded(C0, 7)
        assert emu.emu_dgemm_noalloc(emu.EMU_COL_MAJOR, m, n, k, 1.5, Ad.data_ptr(), lda, Bd.data_ptr(), ldb,
                                     -0.25, Cd.data_ptr(), ldc, p, status.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = Cd.cpu().numpy()
        assert np.array_equal(got[:, :m].T, want)
        assert np.all(np.isnan(got[:, m:]))  # the padding is not touched
    # the same product through emu_dgemm (handle API), also column-major
    Cref, _ = _colmajor_padded(C0, 7)
    assert emu.emu_dgemm(h.h, emu.EMU_COL_MAJOR, m, n, k, 1.5, Ad.data_ptr(), lda, Bd.data_ptr(), ldb, -0.25,
                         Cref.data_ptr(), ldc, emu.EMU_SCHEME_I, p, stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(Cref[:, :m], Cd[:, :m])  # the NaN padding compares unequal, so only C itself
    h.close()


def test_noalloc_k_zero_and_nan_status(orc):
    h = emu.Handle(0)
    m, n = 70, 45
    C0 = synth.test_matrix(m, n, 1.0, 31)
    e = torch.zeros((m, 0), dtype=torch.float64, device="cuda")
    f = torch.zeros((0, n), dtype=torch.float64, device="cuda")
    for beta in (0.0, -3.0):
        C = torch.from_numpy(C0).cuda()
        ref = torch.from_numpy(C0).cuda()
        emu.dgemm(e, f, ref, alpha=2.0, beta=beta, scheme="I", p=5, handle=h)
        for _ in range(2):
            C.copy_(torch.from_numpy(C0))
            assert _noalloc(e, f, C, 5, alpha=2.0, beta=beta) == 0
            torch.cuda.synchronize()
            assert torch.equal(C, ref)
            assert np.array_equal(C.cpu().numpy(), np.zeros_like(C0) if beta == 0.0 else beta * C0)
    # a NaN in A: bit 1 (non-finite input) reaches the caller's status word
    A, B = synth.gemm_pair(64, 64, 96, 1.0, 32)
    A[5, 7] = np.nan
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    assert _noalloc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, 6, status=status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) & 1
    # and the next call, on finite input, is clean again
    status.zero_()
    A[5, 7] = 0.5
    assert _noalloc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, 6, status=status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(C.cpu().numpy(), orc.emu_I(A, B, 6))
    h.close()
