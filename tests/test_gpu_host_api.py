"""emu_dgemm_host (host-resident A, B, C; Scheme I and the bf16 Scheme II
engine in row chunks whose copies overlap the computation) against
emu_dgemm on device copies of the same matrices, bit for bit, and against
the oracle: several chunks with a ragged last one, both layouts with padded
leading dimensions, beta != 0, pinned and pageable host memory, Scheme II
with worst-case and norm scaling, k = 0, and a product below the chunk
size."""
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


def padded_host(x, extra, pinned):
    """Row-major host copy of x inside a buffer `extra` columns wider."""
    buf = torch.zeros((x.shape[0], x.shape[1] + extra), dtype=torch.float64)
    if pinned:
        buf = buf.pin_memory()
    buf[:, :x.shape[1]] = torch.from_numpy(np.ascontiguousarray(x))
    return buf[:, :x.shape[1]]


@pytest.mark.parametrize("scheme,p", [("I", 7), ("I_F8", 11)])
@pytest.mark.parametrize("pinned", [True, False])
def test_scheme_I_chunks_bit_exact(orc, h, scheme, p, pinned):
    # M = 2100: two chunks of 1152 and 948 rows
    m, n, k = 2100, 500, 700
    A, B = synth.gemm_pair(m, n, k, 2.0, 81)
    C0 = synth.test_matrix(m, n, 1.0, 82)
    Ah, Bh = padded_host(A, 3, pinned), padded_host(B, 5, pinned)
    Ch = padded_host(C0, 1, pinned)
    emu.dgemm_host(Ah, Bh, Ch, alpha=0.75, beta=-0.5, scheme=scheme, p=p, handle=h)
    Cd = torch.from_numpy(C0).cuda()
    emu.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, alpha=0.75, beta=-0.5, scheme=scheme, p=p,
              handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    got = Ch.numpy()
    assert np.array_equal(got, Cd.cpu().numpy())
    ref = orc.emu_I(A, B, p, alpha=0.75, beta=-0.5, C=C0) if scheme == "I" else None
    if ref is not None:
        assert np.array_equal(got, ref)


def test_column_major_four_chunks(h):
    # column-major: the row-major view is C^T = B^T A^T, chunked along the
    # columns of C (n = 4500: four chunks of 1152 and a ragged last one)
    m, n, k = 300, 4500, 600
    A, B = synth.gemm_pair(m, n, k, 1.0, 83)
    At, Bt = np.asfortranarray(A), np.asfortranarray(B)
    Ch = np.asfortranarray(np.full((m, n), np.nan))
    emu.dgemm_host(At, Bt, Ch, scheme="I", p=6, handle=h)
    Cd = emu.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), scheme="I", p=6, handle=h)
    assert np.array_equal(Ch, Cd.cpu().numpy())


@pytest.mark.parametrize("scheme,p", [("II", 14), ("II_NORM", 12)])
@pytest.mark.parametrize("m", [1100, 2100])
def test_scheme_II_chunks(orc, h, scheme, p, m):
    # 1100 rows: one chunk through the split-B-then-A phases; 2100: two
    # chunks (1152 and 948 rows) sharing B's split, beta != 0
    n, k = 300, 2000
    A, B = synth.gemm_pair(m, n, k, 1.0, 84)
    C0 = synth.test_matrix(m, n, 1.0, 87)
    Ch = padded_host(C0, 2, True)
    emu.dgemm_host(padded_host(A, 1, True), B, Ch, alpha=1.5, beta=0.25, scheme=scheme, p=p, handle=h)
    Cd = torch.from_numpy(C0).cuda()
    emu.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Cd, alpha=1.5, beta=0.25, scheme=scheme, p=p,
              handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(Ch.numpy(), Cd.cpu().numpy())
    assert np.array_equal(Ch.numpy(), orc.emu_II(A, B, p, alpha=1.5, beta=0.25, C=C0, norm=scheme == "II_NORM"))


def test_small_and_k0(orc, h):
    A, B = synth.gemm_pair(100, 90, 80, 1.0, 85)
    C = emu.dgemm_host(A, B, scheme="I", p=7, handle=h)
    assert np.array_equal(C, orc.emu_I(A, B, 7))
    C0 = synth.test_matrix(40, 30, 1.0, 86)
    Ch = C0.copy()
    emu.dgemm_host(np.zeros((40, 0)), np.zeros((0, 30)), Ch, alpha=1.0, beta=2.0, scheme="I", p=7, handle=h)
    assert np.array_equal(Ch, 2.0 * C0)
