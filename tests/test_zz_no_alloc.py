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
    return emu.emu_dgemm_noalloc(emu.EMU_ROW_MAJOR, m, n, k, alpha, A.data_ptr(), k, B.data_ptr(), n, beta,
                                 C.data_ptr(), n, p, None if status is None else status.data_ptr(), stream)


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
