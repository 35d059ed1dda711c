"""Randomised parity sweep: small products of random shape (including 1 and
sizes just past the tile and chunk edges), random layout, padded leading
dimensions (even and odd, so both the 16-byte and the scalar load paths
run), random alpha and beta, every scheme of emu_dgemm, and the
host-buffer entry point -- each bit for bit against the oracle.  Seeded, so
a failure names a reproducible case."""
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


SIZES = [1, 2, 31, 33, 64, 127, 129, 200, 255, 257, 400]


def case(i):
    rng = np.random.Generator(np.random.PCG64(9000 + i))
    m, n, k = (int(rng.choice(SIZES)) for _ in range(3))
    scheme = ["I", "I_F8", "II", "II_NORM"][i % 4]
    p = int(rng.integers(3, 9)) if scheme == "I" else int(rng.integers(6, 13)) if scheme == "I_F8" else \
        int(rng.integers(4, 21))
    layout = "col" if rng.random() < 0.5 else "row"
    pad = int(rng.integers(0, 4))
    phi = float(rng.choice([0.0, 0.5, 2.0, 4.0]))
    alpha = float(rng.choice([1.0, -0.75, 3.0]))
    beta = float(rng.choice([0.0, 0.0, 1.0, -0.5]))
    return m, n, k, scheme, p, layout, pad, phi, alpha, beta


def on_device(x, layout, pad):
    """x on the GPU in the given layout, inside a buffer `pad` wider in the
    leading dimension."""
    if layout == "row":
        buf = torch.zeros((x.shape[0], x.shape[1] + pad), dtype=torch.float64, device="cuda")
        buf[:, :x.shape[1]] = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        return buf[:, :x.shape[1]]
    buf = torch.zeros((x.shape[1], x.shape[0] + pad), dtype=torch.float64, device="cuda")
    buf[:, :x.shape[0]] = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    return buf[:, :x.shape[0]].t()


def oracle(orc, scheme, A, B, p, alpha, beta, C0):
    if scheme == "I":
        return orc.emu_I(A, B, p, alpha=alpha, beta=beta, C=C0)
    if scheme == "I_F8":
        return orc.emu_F8(A, B, p, alpha=alpha, beta=beta, C=C0)
    return orc.emu_II(A, B, p, alpha=alpha, beta=beta, C=C0, norm=scheme == "II_NORM")


@pytest.mark.parametrize("i", range(96))
def test_random_case(orc, h, i):
    m, n, k, scheme, p, layout, pad, phi, alpha, beta = case(i)
    A, B = synth.gemm_pair(m, n, k, phi, 9500 + i)
    C0 = synth.test_matrix(m, n, 1.0, 9600 + i)
    Cd = on_device(C0, layout, pad)
    emu.dgemm(on_device(A, layout, pad), on_device(B, layout, pad), Cd, alpha=alpha, beta=beta, scheme=scheme, p=p,
              handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0, case(i)
    ref = oracle(orc, scheme, A, B, p, alpha, beta, C0)
    assert np.array_equal(Cd.cpu().numpy(), ref), case(i)
    if i % 3 == 0:  # the host-buffer entry point on the same case
        Ch = np.array(C0, order="F" if layout == "col" else "C")
        Ah = np.array(A, order="F" if layout == "col" else "C")
        Bh = np.array(B, order="F" if layout == "col" else "C")
        emu.dgemm_host(Ah, Bh, Ch, alpha=alpha, beta=beta, scheme=scheme, p=p, handle=h)
        assert np.array_equal(Ch, ref), case(i)


def zcase(i):
    rng = np.random.Generator(np.random.PCG64(19000 + i))
    m, n, k = (int(rng.choice(SIZES)) for _ in range(3))
    scheme = ["II", "I", "I_F8", "II_NORM"][i % 4]
    p = int(rng.integers(4, 21)) if scheme.startswith("II") else int(rng.integers(3, 9)) if scheme == "I" else \
        int(rng.integers(6, 13))
    alpha = complex(rng.choice([1.0, -0.5])) + 1j * float(rng.choice([0.0, 0.75]))
    beta = complex(rng.choice([0.0, 0.0, 1.0])) + 1j * float(rng.choice([0.0, -0.25]))
    f32 = rng.random() < 0.3
    return m, n, k, scheme, p, alpha, beta, f32


@pytest.mark.parametrize("i", range(32))
def test_random_complex_case(orc, h, i):
    m, n, k, scheme, p, alpha, beta, f32 = zcase(i)
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, 19500 + i)
    C0 = synth.test_matrix_complex(m, n, 1.0, 19600 + i)
    if f32:  # CGEMM (complex64): the oracle takes the rounded inputs as given
        A, B, C0 = A.astype(np.complex64), B.astype(np.complex64), C0.astype(np.complex64)
    Cd = torch.from_numpy(np.ascontiguousarray(C0)).cuda()
    Ad, Bd = torch.from_numpy(np.ascontiguousarray(A)).cuda(), torch.from_numpy(np.ascontiguousarray(B)).cuda()
    if f32:
        emu.cgemm(Ad, Bd, Cd, alpha=alpha, beta=beta, p=p, scheme=scheme, handle=h)
    else:
        emu.zgemm(Ad, Bd, Cd, alpha=alpha, beta=beta, nm=p, scheme=scheme, p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0, zcase(i)
    if scheme.startswith("II"):
        ref = orc.emu_Z3M(A, B, p, alpha=alpha, beta=beta, C=C0, out_f32=f32, norm=scheme == "II_NORM")
    else:
        ref = orc.emu_Z4M_I(A, B, p, f8=scheme == "I_F8", alpha=alpha, beta=beta, C=C0, out_f32=f32)
    assert np.array_equal(Cd.cpu().numpy(), ref), zcase(i)


@pytest.mark.parametrize("count", [1, 7, 8, 9, 40])
def test_random_grouped_batch(orc, tmp_path, count):
    # batch sizes around the staging threshold (one stage below 8 products),
    # random shapes with padded leading dimensions, alpha/beta per product,
    # random configurations per shape bucket from a tuning file
    rng = np.random.Generator(np.random.PCG64(29000 + count))
    p = int(rng.integers(3, 9))
    lines = ['  "p%d_s%d_k%d": %d' % (p, sc, kc, int(rng.integers(0, 6))) for sc in range(5) for kc in range(5)]
    path = tmp_path / "tune.json"
    path.write_text("{\n" + ",\n".join(lines) + "\n}\n")
    hd = emu.Handle(0)
    emu.check(emu.emu_load_tuning(hd.h, str(path).encode()))
    mats, As, Bs, Cs, C0s, al, be = [], [], [], [], [], [], []
    for i in range(count):
        m, n, k = (int(rng.choice(SIZES)) for _ in range(3))
        A, B = synth.gemm_pair(m, n, k, float(rng.choice([0.5, 2.0])), 29100 + 50 * count + i)
        C0 = synth.test_matrix(m, n, 1.0, 29200 + 50 * count + i)
        mats.append((A, B))
        As.append(on_device(A, "row", int(rng.integers(0, 3))))
        Bs.append(on_device(B, "row", int(rng.integers(0, 3))))
        Cs.append(on_device(C0, "row", int(rng.integers(0, 3))))
        C0s.append(C0)
        al.append(float(rng.choice([1.0, -2.0])))
        be.append(float(rng.choice([0.0, 0.5])))
    emu.dgemm_grouped(emu.grouped_descs(As, Bs, Cs, al, be), p, handle=hd)
    torch.cuda.synchronize()
    assert hd.status() == 0
    for (A, B), C, C0, a, b in zip(mats, Cs, C0s, al, be):
        assert np.array_equal(C.cpu().numpy(), orc.emu_I(A, B, p, alpha=a, beta=b, C=C0))
    hd.close()
