"""The unfused ("naive") Scheme I pipeline -- INT32 partials of Eq. (2) to
HBM, then the separate shift-reduce of Eq. (3) -- gives exactly the fused
kernel's result (and the oracle's) whenever k <= K_c."""
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


@pytest.mark.parametrize("f8,p,m,n,k", [(False, 7, 300, 200, 1000), (False, 8, 64, 33, 4608),
                                        (True, 11, 250, 130, 900), (True, 4, 65, 70, 5000)])
def test_partials_then_reduce_equals_fused(orc, h, f8, p, m, n, k):
    A, B = synth.gemm_pair(m, n, k, 1.5, 70 + p)
    Ad, Bd = dev(A), dev(B)
    _, EA = emu.split_I(Ad, p, operand=0, handle=h, f8=f8)
    _, FB = emu.split_I(Bd, p, operand=1, handle=h, f8=f8)
    Cs = emu.partials_I(Ad, Bd, p, handle=h, f8=f8)
    C = emu.shift_reduce_I(Cs, EA, FB, p, f8=f8, handle=h)
    fused = emu.dgemm(Ad, Bd, scheme="I_F8" if f8 else "I", p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert torch.equal(C, fused)
    ref = orc.emu_F8(A, B, p) if f8 else orc.emu_I(A, B, p)
    assert np.array_equal(C.cpu().numpy(), ref)
    # BLAS update in the separate epilogue as well
    C0 = synth.test_matrix(m, n, 1.0, 3)
    Cd = dev(C0)
    emu.shift_reduce_I(Cs, EA, FB, p, f8=f8, C=Cd, alpha=-0.5, beta=2.0, handle=h)
    ref2 = (orc.emu_F8 if f8 else orc.emu_I)(A, B, p, alpha=-0.5, beta=2.0, C=C0)
    assert np.array_equal(Cd.cpu().numpy(), ref2)
