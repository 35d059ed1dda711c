"""Scheme II on the bf16 tcgen05 engine (the default) against the oracle:
products whose K spans several exact FP32 segments (960 K each) with ragged
tails, several 128 x 256 tiles with ragged edges, 1 to 20 moduli, the
largest segment sum (every residue modulo 256 equal to -128), K beyond the
INT32 range of the INT8 engine, 3M complex, both GEMM forms (single CTAs on
128 x 256 tiles, the default, and CTA pairs on 256 x 256 tiles with
EMU_II_CLUSTER=2) and the INT8 mma.sync engine (EMU_II_ENGINE=mma); both
settings are read once per process, so those runs use child processes."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_25453_gb300 as emu  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def h():
    hd = emu.Handle(0)
    yield hd
    hd.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


CASES = [
    (300, 600, 3000, 16, 1.0, 11),   # 3 x 3 tiles, K over four segments (the last one short)
    (129, 257, 961, 20, 4.0, 12),    # one row and one column past a tile, K one past a segment
    (200, 130, 1920, 5, 0.5, 13),    # two full segments
    (64, 64, 2050, 4, 2.0, 14),
    (33, 300, 700, 1, 1.0, 15),      # one modulus
    (257, 129, 4100, 12, 8.0, 16),
]


@pytest.mark.parametrize("m,n,k,nm,phi,seed", CASES)
def test_dgemm_II_tc_bit_exact(orc, h, m, n, k, nm, phi, seed):
    A, B = synth.gemm_pair(m, n, k, phi, seed)
    C = emu.dgemm(dev(A), dev(B), scheme="II", p=nm, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), orc.emu_II(A, B, nm))


def test_largest_segment_sum(orc, h):
    # x = 1/2 + 2^(7-b) scales to a' = 2^(b-1) + 2^7, whose residue modulo 256
    # is -128: every product of the first modulus is 2^14 and each full
    # segment sums to 960 * 2^14 (the FP32 accumulator's exact-integer bound)
    m, n, k, nm = 128, 64, 2880, 16
    b = orc.scale_bits_II(nm, k)
    x = 0.5 + 2.0 ** (7 - b)
    A = np.full((m, k), x)
    A[::3] *= -1.0
    B = np.full((k, n), x)
    res = orc.residues_II_rows(A[:1], nm, b)
    assert res[0, 0, 0] == -128
    C = emu.dgemm(dev(A), dev(B), scheme="II", p=nm, handle=h)
    assert np.array_equal(C.cpu().numpy(), orc.emu_II(A, B, nm))


def test_k_beyond_int32_sums(orc, h):
    m, n, k, nm = 16, 24, 140000, 12
    A, B = synth.gemm_pair(m, n, k, 1.0, 21)
    C = emu.dgemm(dev(A), dev(B), scheme="II", p=nm, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), orc.emu_II(A, B, nm))


@pytest.mark.parametrize("m,n,k,nm,seed", [(140, 70, 2000, 18, 31), (33, 97, 300, 6, 32)])
def test_zgemm_cgemm_3m_tc_bit_exact(orc, h, m, n, k, nm, seed):
    A, B = synth.gemm_pair_complex(m, n, k, 1.0, seed)
    C0 = synth.test_matrix_complex(m, n, 1.0, seed + 1)
    Cd = dev(C0)
    emu.zgemm(dev(A), dev(B), Cd, alpha=0.5 - 1.0j, beta=0.25 + 0.5j, nm=nm, handle=h)
    assert np.array_equal(Cd.cpu().numpy(), orc.emu_Z3M(A, B, nm, alpha=0.5 - 1.0j, beta=0.25 + 0.5j, C=C0))
    Af, Bf = A.astype(np.complex64), B.astype(np.complex64)
    Cf = emu.cgemm(dev(Af), dev(Bf), p=nm, scheme="II", handle=h)
    assert np.array_equal(Cf.cpu().numpy(), orc.emu_Z3M(Af, Bf, nm, out_f32=True))


CHILD = r"""
import sys
import numpy as np
import torch
import synth
import paper_2606_25453_gb300 as emu
out = sys.argv[1]
h = emu.Handle(0)
A, B = synth.gemm_pair(300, 200, 3000, 1.0, 11)
C = emu.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), scheme="II", p=16, handle=h)
Az, Bz = synth.gemm_pair_complex(140, 70, 2000, 1.0, 31)
Z = emu.zgemm(torch.from_numpy(Az).cuda(), torch.from_numpy(Bz).cuda(), nm=18, handle=h)
torch.cuda.synchronize()
assert h.status() == 0
A2, B2 = synth.gemm_pair(4, 4, 140000, 1.0, 21)
try:
    emu.dgemm(torch.from_numpy(A2).cuda(), torch.from_numpy(B2).cuda(), scheme="II", p=12, handle=h)
    big = "accepted"
except emu.EmuError as e:
    big = str(e)
np.savez(out, C=C.cpu().numpy(), Z=Z.cpu().numpy(), big=np.array(big))
"""


def test_int8_engine_matches(orc, tmp_path):
    out = tmp_path / "mma.npz"
    env = dict(os.environ, EMU_II_ENGINE="mma")
    subprocess.run([sys.executable, "-c", CHILD, str(out)], cwd=ROOT, env=env, check=True, timeout=600)
    r = np.load(out)
    A, B = synth.gemm_pair(300, 200, 3000, 1.0, 11)
    assert np.array_equal(r["C"], orc.emu_II(A, B, 16))
    Az, Bz = synth.gemm_pair_complex(140, 70, 2000, 1.0, 31)
    assert np.array_equal(r["Z"], orc.emu_Z3M(Az, Bz, 18))
    # the INT8 engine sums a modulus's products in INT32: K > 131071 is refused
    assert "UNSUPPORTED" in str(r["big"])


CHILD_CL = r"""
import sys
import numpy as np
import torch
import synth
import paper_2606_25453_gb300 as emu
out = sys.argv[1]
h = emu.Handle(0)
A, B = synth.gemm_pair(300, 130, 2000, 2.0, 41)
C = emu.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), scheme="II", p=14, handle=h)
Az, Bz = synth.gemm_pair_complex(140, 70, 1000, 1.0, 42)
Z = emu.zgemm(torch.from_numpy(Az).cuda(), torch.from_numpy(Bz).cuda(), nm=9, handle=h)
torch.cuda.synchronize()
assert h.status() == 0
np.savez(out, C=C.cpu().numpy(), Z=Z.cpu().numpy())
"""


@pytest.mark.parametrize("cl", [1, 2])
def test_cluster_sizes(orc, tmp_path, cl):
    # 2: a CTA pair per 256 x 256 tile (300 rows: the odd CTA of the second
    # pair tile has no rows of A); 1: one CTA per 128 x 256 tile
    out = tmp_path / "cl.npz"
    env = dict(os.environ, EMU_II_CLUSTER=str(cl))
    subprocess.run([sys.executable, "-c", CHILD_CL, str(out)], cwd=ROOT, env=env, check=True, timeout=600)
    r = np.load(out)
    A, B = synth.gemm_pair(300, 130, 2000, 2.0, 41)
    assert np.array_equal(r["C"], orc.emu_II(A, B, 14))
    Az, Bz = synth.gemm_pair_complex(140, 70, 1000, 1.0, 42)
    assert np.array_equal(r["Z"], orc.emu_Z3M(Az, Bz, 9))


def test_zgemm_3m_sampled_rows_n4096(orc, h):
    # many waves of 128 x 256 tiles over all 3 x 16 planes; the oracle computes
    # row i of C from row i of A and all of B (the scales are per row / column)
    n, nm = 4096, 16
    A, B = synth.gemm_pair_complex(n, n, n, 1.0, 51)
    C = emu.zgemm(dev(A), dev(B), nm=nm, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    rows = [1, 3000]
    assert np.array_equal(C[rows].cpu().numpy(), orc.emu_Z3M(A[rows], B, nm))


def test_trace_splits_residue_gemm_and_crt(h):
    # the traced "gemm" phase of the bf16 engine is the residue GEMM alone;
    # the CRT kernel is recorded as "other"
    A, B = synth.gemm_pair(512, 512, 1000, 1.0, 61)
    Ad, Bd = dev(A), dev(B)
    emu.dgemm(Ad, Bd, scheme="II", p=16, handle=h)
    torch.cuda.synchronize()
    h.trace(True)
    h.trace_read()
    emu.dgemm(Ad, Bd, scheme="II", p=16, handle=h)
    tr = h.trace_read()
    h.trace(False)
    assert tr["gemm_launches"] == 1
    assert tr["kernel_launches"] == 6  # two scans, two splits, residue GEMM, CRT
    assert tr["ms_gemm"] > 0 and tr["ms_other"] > 0 and tr["ms_scan"] > 0 and tr["ms_split"] > 0
