"""Grouped emulated DGEMM (persistent launches per tile shape under one CUDA
graph) against the oracle, the per-product loop, mixed tile shapes per
shape bucket, and the autotuner's interface."""
import json
import os

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


def make_problems(count, seed, mn=(1, 200), kr=(1, 300)):
    shapes = synth.grouped_shapes(count, seed, mn_range=mn, k_range=kr)
    mats = []
    for i, (m, n, k) in enumerate(shapes):
        A, B = synth.gemm_pair(m, n, k, 1.0, 1000 * seed + i)
        mats.append((A, B))
    return shapes, mats


def test_grouped_bit_exact_and_replay(orc, h):
    p = 6
    shapes, mats = make_problems(40, 3)
    As = [torch.from_numpy(A).cuda() for A, _ in mats]
    Bs = [torch.from_numpy(B).cuda() for _, B in mats]
    Cs = [torch.full((m, n), np.nan, dtype=torch.float64, device="cuda") for m, n, _ in shapes]
    d = emu.grouped_descs(As, Bs, Cs)
    emu.dgemm_grouped(d, p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    for (A, B), C in zip(mats, Cs):
        assert np.array_equal(C.cpu().numpy(), orc.emu_I(A, B, p))
    # replay of the captured graph reads the current data behind the same pointers
    for i, (A, B) in enumerate(mats):
        As[i].mul_(-2.0)
    emu.dgemm_grouped(d, p, handle=h)
    torch.cuda.synchronize()
    for (A, B), C in zip(mats, Cs):
        assert np.array_equal(C.cpu().numpy(), orc.emu_I(-2.0 * A, B, p))


def test_grouped_alpha_beta_matches_loop(h):
    p = 4
    shapes, mats = make_problems(25, 5, mn=(20, 300), kr=(10, 700))
    As = [torch.from_numpy(A).cuda() for A, _ in mats]
    Bs = [torch.from_numpy(B).cuda() for _, B in mats]
    C0 = [torch.from_numpy(synth.test_matrix(m, n, 1.0, 70 + i)).cuda() for i, (m, n, _) in enumerate(shapes)]
    Cg = [c.clone() for c in C0]
    Cl = [c.clone() for c in C0]
    al = [0.5 + i for i in range(len(shapes))]
    be = [(-1.0) ** i for i in range(len(shapes))]
    emu.dgemm_grouped(emu.grouped_descs(As, Bs, Cg, al, be), p, handle=h)
    emu.dgemm_grouped(emu.grouped_descs(As, Bs, Cl, al, be), p, handle=h, loop=True)
    torch.cuda.synchronize()
    for a, b in zip(Cg, Cl):
        assert torch.equal(a, b)


def test_autotuner_and_cache(h, tmp_path):
    p = 6
    shapes, mats = make_problems(30, 9, mn=(32, 256), kr=(64, 512))
    As = [torch.from_numpy(A).cuda() for A, _ in mats]
    Bs = [torch.from_numpy(B).cuda() for _, B in mats]
    Cs = [torch.empty((m, n), dtype=torch.float64, device="cuda") for m, n, _ in shapes]
    d = emu.grouped_descs(As, Bs, Cs)
    path = str(tmp_path / "tune.json")
    timed = emu.tune_grouped(d, p, path=path, handle=h)
    cache = json.load(open(path))
    # one choice per shape bucket (3 tile shapes x 2 slice-pair orders) and
    # the stage setting; for each of the two settings (three stages, one):
    # the whole batch in the current choices and the five other single
    # configurations, six timings of each bucket alone, then at most one
    # whole batch with all candidates and one per changed bucket
    assert cache.pop("p6_stages") in (1, 3)
    nb = len(cache)
    assert nb >= 2 and all(v in range(6) for v in cache.values())
    assert all(k.startswith("p6_s") for k in cache)
    assert 2 * (6 + 6 * nb) <= timed <= 2 * (7 + 7 * nb)
    ref = [c.clone() for c in Cs]
    h2 = emu.Handle(0)
    emu.check(emu.emu_load_tuning(h2.h, path.encode()))
    emu.dgemm_grouped(d, p, handle=h2)
    torch.cuda.synchronize()
    for a, b in zip(Cs, ref):
        assert torch.equal(a, b)
    h2.close()


@pytest.mark.parametrize("stages", [None, 1])
def test_mixed_tile_shapes_bit_exact(orc, tmp_path, stages):
    """A tuning that gives the shape buckets different configurations (tile
    shape x slice-pair order): the products run in up to six GEMM launches
    per stage on parallel graph branches (three stages by default, one with
    "p5_stages": 1), each bit-exact against the oracle (ragged edges
    exercise the patches that lie wholly outside a product)."""
    p = 5
    shapes, mats = make_problems(60, 11, mn=(20, 700), kr=(60, 1500))
    path = tmp_path / "mixed.json"
    lines = ['  "p5_s%d_k%d": %d' % (sc, kc, (sc + 2 * kc) % 6) for sc in range(5) for kc in range(5)]
    if stages is not None:
        lines.append('  "p5_stages": %d' % stages)
    with open(path, "w") as fh:
        fh.write("{\n" + ",\n".join(lines) + "\n}\n")
    hd = emu.Handle(0)
    emu.check(emu.emu_load_tuning(hd.h, str(path).encode()))
    As = [torch.from_numpy(A).cuda() for A, _ in mats]
    Bs = [torch.from_numpy(B).cuda() for _, B in mats]
    Cs = [torch.full((m, n), np.nan, dtype=torch.float64, device="cuda") for m, n, _ in shapes]
    d = emu.grouped_descs(As, Bs, Cs)
    for _ in range(2):  # capture, then replay
        emu.dgemm_grouped(d, p, handle=hd)
        torch.cuda.synchronize()
        assert hd.status() == 0
        for (A, B), C in zip(mats, Cs):
            assert np.array_equal(C.cpu().numpy(), orc.emu_I(A, B, p))
        for C in Cs:
            C.fill_(np.nan)
    hd.close()


def test_grouped_512_problems_sampled(orc, h):
    """512 products, M, N log-uniform in [32, 1024], K in [64, 2048], phi = 1, p = 6."""
    p = 6
    shapes = synth.grouped_shapes(512, 0)
    As, Bs, Cs, host = [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B = synth.gemm_pair(m, n, k, 1.0, 5000 + i)
        host.append((A, B))
        As.append(torch.from_numpy(A).cuda())
        Bs.append(torch.from_numpy(B).cuda())
        Cs.append(torch.empty((m, n), dtype=torch.float64, device="cuda"))
    emu.dgemm_grouped(emu.grouped_descs(As, Bs, Cs), p, handle=h)
    torch.cuda.synchronize()
    assert h.status() == 0
    for i in (0, 7, 100, 255, 511):
        A, B = host[i]
        rows = [0, A.shape[0] - 1]
        assert np.array_equal(Cs[i][rows].cpu().numpy(), orc.emu_I(A[rows], B, p)), i
