"""Emulated GEMMs captured into a CUDA graph: after one uncaptured call of
the same shape (which sizes the handle's workspace) DGEMM with every scheme
and ZGEMM 3M capture on the caller's stream and, replayed after the inputs
were overwritten in place, give bit for bit what an uncaptured call on the
new inputs gives.  A call that would have to grow the workspace while its
stream is capturing is refused with EMU_ERR_ALLOC before it enqueues
anything, and the handle keeps working afterwards."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_25453_gb300 as emu  # noqa: E402


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("scheme,p", [("I", 7), ("I_F8", 11), ("II", 16), ("II_NORM", 14)])
def test_dgemm_capture_and_replay(scheme, p):
    h = emu.Handle(0)
    m, n, k = 300, 260, 1100
    A, B = synth.gemm_pair(m, n, k, 1.0, 171)
    A2, B2 = synth.gemm_pair(m, n, k, 2.0, 172)
    Ad, Bd = dev(A), dev(B)
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    emu.dgemm(Ad, Bd, C, scheme=scheme, p=p, handle=h, stream=s)  # sizes the workspace
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        emu.dgemm(Ad, Bd, C, alpha=0.5, scheme=scheme, p=p, handle=h, stream=s)
    Ad.copy_(dev(A2))
    Bd.copy_(dev(B2))
    C.fill_(float("nan"))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert h.status() == 0
    ref = emu.dgemm(dev(A2), dev(B2), alpha=0.5, scheme=scheme, p=p, handle=h)
    assert np.array_equal(C.cpu().numpy(), ref.cpu().numpy())
    h.close()


def test_zgemm_capture_and_replay():
    h = emu.Handle(0)
    m, n, k, nm = 200, 150, 700, 12
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 173)
    Ad, Bd = dev(A), dev(B)
    C = torch.empty((m, n), dtype=torch.complex128, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    emu.zgemm(Ad, Bd, C, nm=nm, handle=h, stream=s)
    s.synchronize()
    ref = C.cpu().numpy()
    C.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        emu.zgemm(Ad, Bd, C, nm=nm, handle=h, stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), ref)
    h.close()


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # nothing was enqueued, as intended
def test_workspace_growth_refused_while_capturing(orc):
    h = emu.Handle(0)  # no workspace yet
    A, B = synth.gemm_pair(128, 96, 256, 1.0, 174)
    Ad, Bd = dev(A), dev(B)
    C = torch.zeros((128, 96), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(emu.EmuError) as e:
        with torch.cuda.graph(g, stream=s):
            emu.dgemm(Ad, Bd, C, scheme="I", p=6, handle=h, stream=s)
    assert e.value.code == 5  # EMU_ERR_ALLOC
    torch.cuda.synchronize()
    assert h.status() == 0
    # outside the capture the same call allocates and runs
    emu.dgemm(Ad, Bd, C, scheme="I", p=6, handle=h)
    assert np.array_equal(C.cpu().numpy(), orc.emu_I(A, B, 6))
    h.close()
