"""The largest sizes of the benchmark configurations, on sampled outputs the
oracle computes row by row (every scale is per row of A and per column of
B, so row i of C needs only row i of A and all of B): DGEMM and SGEMM with
Scheme I and DGEMM with Scheme II at M = N = K = 16384, and ZGEMM 3M at
8192, in the launch configuration the benchmark times (row-major, the
library's default engines)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_25453_gb300 as emu  # noqa: E402

N = 16384
ROWS = [0, 8191, 16383]


@pytest.fixture(scope="module")
def h():
    hd = emu.Handle(0)
    yield hd
    hd.close()


@pytest.fixture(scope="module")
def big():
    A, B = synth.gemm_pair(N, N, N, 0.5, 161)
    return A, B, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()


@pytest.mark.parametrize("scheme,p", [("I", 8), ("II", 16)])
def test_dgemm_16384_sampled_rows(orc, h, big, scheme, p):
    A, B, Ad, Bd = big
    C = emu.dgemm(Ad, Bd, scheme=scheme, p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    got = C[ROWS].cpu().numpy()
    del C
    ref = orc.emu_I(A[ROWS], B, p) if scheme == "I" else orc.emu_II(A[ROWS], B, p)
    assert np.array_equal(got, ref)


def test_sgemm_16384_sampled_rows(orc, h, big):
    A, B, Ad, Bd = big
    C = emu.sgemm(Ad.float(), Bd.float(), scheme="I", p=4, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    got = C[ROWS].cpu().numpy()
    del C
    ref = orc.emu_I(A[ROWS].astype(np.float32), B.astype(np.float32), 4, out_f32=True)
    assert np.array_equal(got, ref)


def test_zgemm_3m_8192_sampled_rows(orc, h):
    n, nm = 8192, 16
    A, B = synth.gemm_pair_complex(n, n, n, 1.0, 162)
    C = emu.zgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), nm=nm, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    rows = [0, 4095, 8191]
    assert np.array_equal(C[rows].cpu().numpy(), orc.emu_Z3M(A[rows], B, nm))
