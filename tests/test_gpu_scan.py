"""The exponent scan (the scale vectors of Eq. 1 and the Scheme II scaling)
on its 16-byte-load path and on the scalar path it falls back to: operands
given as views with padded leading dimensions (16-byte aligned or not) and
offset base pointers, vector counts that leave a ragged last group of a
16-byte load, K that leaves a ragged end of a 2048-scalar segment, and the
one largest element of each row planted first, last, in that ragged end or
at random.  Binary64 exponents must equal the oracle's; binary32 and complex
operands go through the full Scheme II product (3M for complex), which
depends on every exponent."""
import numpy as np
import pytest

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


def planted(rows, k, dtype, seed):
    """rows x k: each row scaled by its own power of two, with one element
    four times the row scale (the unique maximum) at a chosen position."""
    rng = np.random.default_rng(seed)
    s = 2.0 ** rng.integers(-30, 30, (rows, 1))
    X = rng.uniform(-1.0, 1.0, (rows, k)) * s
    pos = rng.integers(0, k, rows)
    pos[0], pos[1], pos[2] = 0, k - 1, k - 1 - (k % 2048) // 2
    X[np.arange(rows), pos] = np.where(rng.random(rows) < 0.5, -4.0, 4.0) * s[:, 0]
    return X.astype(dtype)


def view(X, pad, off, dtype):
    """X as a row-major view of a larger device buffer: leading dimension
    cols + pad, first column off."""
    r, c = X.shape
    base = torch.zeros((r, c + pad + off), dtype=dtype, device="cuda")
    v = base[:, off:off + c]
    v.copy_(torch.from_numpy(np.ascontiguousarray(X)).cuda())
    return v


def padding(cols, itemsize, ldk):
    """Columns to add to a row of `cols` elements: "a" makes the leading
    dimension a multiple of 16 bytes (the 16-byte path), "a+" adds 16 bytes
    more, "u" leaves it off a multiple of 16 bytes (the scalar path)."""
    per16 = 16 // itemsize
    return (-cols) % per16 + {"a": 0, "a+": per16, "u": 1}[ldk]


# (leading dimension, offset): an offset base pointer takes the scalar path
LAYOUTS = [("a", 0), ("a+", 0), ("u", 0), ("a", 1)]


@pytest.mark.parametrize("ldk,off", LAYOUTS)
@pytest.mark.parametrize("operand", [0, 1])
def test_scan_exponents_f64(orc, h, ldk, off, operand):
    rows, k = 131, 4133  # 131 = 32 * 4 + 3 vectors; K = 2 * 2048 + 37
    Xr = planted(rows, k, np.float64, 7 + operand)
    Xd = Xr if operand == 0 else Xr.T
    X = view(Xd, padding(Xd.shape[1], 8, ldk), off, torch.float64)
    _, E = emu.split_I(X, 2, operand=operand, handle=h)
    torch.cuda.synchronize()
    assert np.array_equal(E.cpu().numpy(), orc.row_exponents(Xr))


@pytest.mark.parametrize("ldk,off", [("a", 0), ("a+", 0), ("u", 0), ("a", 2)])
def test_scan_f32_sgemm(orc, h, ldk, off):
    # binary32 operands: every exponent enters the Scheme II product
    m, n, k, nm = 131, 67, 4133, 6  # 67 = 4 * 16 + 3 columns of B
    A = planted(m, k, np.float32, 11)
    B = planted(n, k, np.float32, 12).T
    Ad = view(A, padding(k, 4, ldk), off, torch.float32)
    Bd = view(B, padding(n, 4, ldk), off, torch.float32)
    C = emu.sgemm(Ad, Bd, scheme="II", p=nm, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), orc.emu_II(A, B, nm, out_f32=True))


@pytest.mark.parametrize("cdt,pad", [(torch.complex128, 0), (torch.complex128, 1),
                                     (torch.complex64, 0), (torch.complex64, 2), (torch.complex64, 1)])
def test_scan_complex_views(orc, h, cdt, pad):
    m, n, k, nm = 37, 45, 300, 8  # n odd: a ragged pair of complex64 columns
    npdt = np.complex128 if cdt == torch.complex128 else np.complex64
    fdt = np.float64 if cdt == torch.complex128 else np.float32
    A = (planted(m, k, fdt, 1) + 1j * planted(m, k, fdt, 2)).astype(npdt)
    B = (planted(n, k, fdt, 3) + 1j * planted(n, k, fdt, 4)).T.astype(npdt)
    Ad, Bd = view(A, pad, 0, cdt), view(B, pad, 0, cdt)
    if cdt == torch.complex128:
        C = emu.zgemm(Ad, Bd, nm=nm, handle=h)
        ref = orc.emu_Z3M(A, B, nm)
    else:
        C = emu.cgemm(Ad, Bd, p=nm, scheme="II", handle=h)
        ref = orc.emu_Z3M(A, B, nm, out_f32=True)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), ref)
