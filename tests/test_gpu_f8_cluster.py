"""The E4M3 tcgen05 kernel with each cluster size (1, 2 and 4 CTAs sharing
the A slices through TMA multicast) gives the oracle's result bit for bit.
The cluster size is read once per process from EMU_TC_CLUSTER, so each size
runs in a child process."""
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

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
import synth
import paper_2606_25453_gb300 as emu
m, n, k, p, phi, seed = (float(x) if "." in x else int(x) for x in sys.argv[1:7])
A, B = synth.gemm_pair(m, n, k, phi, seed)
h = emu.Handle(0)
C = emu.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), scheme="I_F8", p=p, handle=h)
torch.cuda.synchronize()
assert h.status() == 0, h.status()
np.save(sys.argv[7], C.cpu().numpy())
"""

CASES = [(700, 450, 200, 11, 1.0, 51), (129, 33, 64, 5, 0.5, 52)]


@pytest.mark.parametrize("cl", [1, 2, 4])
@pytest.mark.parametrize("m,n,k,p,phi,seed", CASES)
def test_f8_cluster_sizes(orc, tmp_path, cl, m, n, k, p, phi, seed):
    out = tmp_path / "c.npy"
    env = dict(os.environ, EMU_TC_CLUSTER=str(cl))
    subprocess.run([sys.executable, "-c", CHILD, str(m), str(n), str(k), str(p), repr(float(phi)), str(seed),
                    str(out)], cwd=ROOT, env=env, check=True, timeout=300)
    A, B = synth.gemm_pair(m, n, k, phi, seed)
    assert np.array_equal(np.load(out), orc.emu_F8(A, B, p))
