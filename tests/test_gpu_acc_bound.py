"""The FP32 tensor-core accumulators of both tcgen05 engines at their
exact-integer bound, against the oracle bit for bit.

Inputs from tests/acc_bound_inputs.py (their properties are checked on the
CPU in tests/test_acc_bound_inputs.py): segment sums of the bf16 Scheme II
engine reach 960 * 127^2 (2^23.88) for the moduli 256 and 255 and within
2^23.7 for the next four, E4M3 chunk sums reach 2^23.95 (p = 11) and
2^23.82 (p = 12), and odd MMA-block sums are added while a running sum is at
or above 2^23, at the first, last and block-boundary K positions of a
segment (chunk) and at random ones.  Each product also runs on the INT8
mma.sync engine of its scheme (and Scheme II on the CTA-pair tcgen05
kernel); those settings are read once per process, so they run in child
processes."""
import os
import subprocess
import sys

import numpy as np
import pytest

from acc_bound_inputs import NM_II, SEG, f8_inputs, scheme_II_inputs

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


CHILD = r"""
import sys
import numpy as np
import torch
import paper_2606_25453_gb300 as emu
inp, out, scheme, p = sys.argv[1], sys.argv[2], sys.argv[3], int(sys.argv[4])
d = np.load(inp)
h = emu.Handle(0)
C = emu.dgemm(torch.from_numpy(d["A"]).cuda(), torch.from_numpy(d["B"]).cuda(), scheme=scheme, p=p, handle=h)
torch.cuda.synchronize()
assert h.status() == 0
np.save(out, C.cpu().numpy())
"""


def run_child(tmp_path, A, B, scheme, p, env_extra):
    inp = tmp_path / "in.npz"
    out = tmp_path / "out.npy"
    np.savez(inp, A=A, B=B)
    env = dict(os.environ, **env_extra)
    subprocess.run([sys.executable, "-c", CHILD, str(inp), str(out), scheme, str(p)], cwd=ROOT, env=env,
                   check=True, timeout=600)
    return np.load(out)


@pytest.fixture(scope="module")
def ii_case(orc):
    m, n, k = 300, 300, 3 * SEG + 37  # 2 x 2 pair tiles with ragged edges, 3 full segments + a short one
    A, B, _ = scheme_II_inputs(m, n, k, orc.moduli(NM_II), seed=7)
    return A, B, orc.emu_II(A, B, NM_II)


def test_scheme_II_bf16_at_bound(ii_case, h):
    A, B, ref = ii_case
    C = emu.dgemm(dev(A), dev(B), scheme="II", p=NM_II, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), ref)


@pytest.mark.parametrize("env", [{"EMU_II_ENGINE": "mma"}, {"EMU_II_CLUSTER": "2"}], ids=["int8", "cta_pair"])
def test_scheme_II_other_engines_at_bound(ii_case, tmp_path, env):
    A, B, ref = ii_case
    assert np.array_equal(run_child(tmp_path, A, B, "II", NM_II, env), ref)


@pytest.fixture(scope="module", params=[11, 12])
def f8_case(orc, request):
    p = request.param
    kc = orc.chunk_len_F8(p)
    m, n, k = 130, 70, 2 * kc + 77  # 2 x 3 tiles, two full K_c chunks and a short one
    A, B, _ = f8_inputs(m, n, k, p, kc, seed=11 + p)
    return p, A, B, orc.emu_F8(A, B, p)


def test_f8_tcgen05_at_bound(f8_case, h):
    p, A, B, ref = f8_case
    C = emu.dgemm(dev(A), dev(B), scheme="I_F8", p=p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), ref)


def test_f8_mma_engine_at_bound(f8_case, tmp_path):
    p, A, B, ref = f8_case
    assert np.array_equal(run_child(tmp_path, A, B, "I_F8", p, {"EMU_F8_ENGINE": "mma"}), ref)


def test_int8_scheme_I_on_bound_inputs(orc, f8_case, h):
    # the same large-digit operands through the INT8 Scheme I kernel (p = 8)
    p, A, B, _ = f8_case
    C = emu.dgemm(dev(A), dev(B), scheme="I", p=8, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert np.array_equal(C.cpu().numpy(), orc.emu_I(A, B, 8))
