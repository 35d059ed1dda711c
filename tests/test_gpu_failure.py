"""Failure detection without faulting the GPU: a bounded device wait that is
made to run out reports EMU_ERR_TIMEOUT through the status word and leaves
the context usable; host-side fault injection: EMU_FAULT=alloc turns
workspace allocation into EMU_ERR_ALLOC while a caller-owned workspace still
works, and EMU_FAULT=launch makes every fused GEMM launch fail on the host
(EMU_ERR_CUDA, C untouched, context intact)."""
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


def test_bounded_wait_times_out_and_context_survives(orc):
    h = emu.Handle(0)
    emu.check(emu.emu_selftest_wait(h.h, 2_000_000, None))  # ~1 ms at 2 GHz
    assert h.status() == 6  # EMU_ERR_TIMEOUT, read and cleared
    assert h.status() == 0
    A, B = synth.gemm_pair(70, 50, 90, 1.0, 3)
    C = emu.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), scheme="I", p=5, handle=h)
    assert np.array_equal(C.cpu().numpy(), orc.emu_I(A, B, 5))
    h.close()


CHILD = r"""
import sys, ctypes, torch
sys.path.insert(0, %r)
import paper_2606_25453_gb300 as emu
h = emu.Handle(0)
A = torch.ones((64, 64), dtype=torch.float64, device="cuda")
try:
    emu.dgemm(A, A, scheme="I", p=4, handle=h)
    print("no-error")
except emu.EmuError as e:
    print("code", e.code)
sz = ctypes.c_size_t()
emu.check(emu.emu_workspace_size(1, 64, 64, 64, 4, 0, ctypes.byref(sz)))
ws = torch.empty(sz.value + 256, dtype=torch.uint8, device="cuda")
emu.check(emu.emu_set_workspace(h.h, ws.data_ptr(), sz.value))
C = emu.dgemm(A, A, scheme="I", p=4, handle=h)
torch.cuda.synchronize()
print("user-ws", float(C[0, 0]))
"""


def test_alloc_fault_injection():
    env = dict(os.environ, EMU_FAULT="alloc")
    r = subprocess.run([sys.executable, "-c", CHILD % ROOT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "code 5" in r.stdout  # EMU_ERR_ALLOC
    assert "user-ws 64.0" in r.stdout


CHILD_LAUNCH = r"""
import sys, torch
sys.path.insert(0, %r)
import paper_2606_25453_gb300 as emu
h = emu.Handle(0)
A = torch.ones((64, 64), dtype=torch.float64, device="cuda")
for scheme, p in (("I", 4), ("I_F8", 8), ("II", 10)):
    C = torch.full((64, 64), 7.0, dtype=torch.float64, device="cuda")
    try:
        emu.dgemm(A, A, C, scheme=scheme, p=p, handle=h)
        print(scheme, "no-error")
    except emu.EmuError as e:
        torch.cuda.synchronize()
        print(scheme, "code", e.code, "untouched", bool((C == 7.0).all()), "|", str(e))
try:
    emu.zgemm(A.to(torch.complex128), A.to(torch.complex128), nm=8, handle=h)
except emu.EmuError as e:
    print("Z code", e.code)
print("status", h.status(), "ctx", float((A @ A)[0, 0]))
"""


def test_launch_fault_injection():
    # EMU_FAULT=launch: each fused GEMM launch fails on the host side after
    # the scan and split were enqueued; the caller gets EMU_ERR_CUDA with
    # the runtime's text, C is not written, nothing faults on the device,
    # and the context stays usable
    env = dict(os.environ, EMU_FAULT="launch")
    r = subprocess.run([sys.executable, "-c", CHILD_LAUNCH % ROOT], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    for scheme in ("I", "I_F8", "II"):
        assert "%s code 4 untouched True" % scheme in r.stdout, r.stdout
    assert "unspecified launch failure" in r.stdout
    assert "Z code 4" in r.stdout
    assert "status 0 ctx 64.0" in r.stdout
