"""Learned slice-count selector on the GPU: the feature, MLP forward/backward,
Adam and double-double probe kernels against the CPU oracle, the auto-
precision entry point, a small training run that must beat the fixed
choice of p at the same tolerance, and training resumed from a checkpoint."""
import ctypes
import math

import numpy as np
import pytest

import synth
from oracle import selector as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2606_25453_gb300 as emu  # noqa: E402
from paper_2606_25453_gb300 import selector as sel  # noqa: E402


@pytest.fixture(scope="module")
def h():
    hd = emu.Handle(0)
    yield hd
    hd.close()


def test_features_exact(h):
    for sample, (m, n, k) in ((0, (40, 30, 50)), (8, (100, 70, 64))):
        A, B = synth.gemm_pair(m, n, k, 5.0, 3)
        A[2, :7] = 0.0
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        f = torch.empty(66, dtype=torch.float32, device="cuda")
        emu.check(emu.emu_sel_features(h.h, 0, m, n, k, Ad.data_ptr(), k, Bd.data_ptr(), n, 1e-12, sample,
                                       f.data_ptr(), None))
        assert np.array_equal(f.cpu().numpy(), S.features(A, B, 1e-12, sample))


def test_forward_backward_adam_vs_oracle(h):
    rng = np.random.Generator(np.random.PCG64(5))
    theta = rng.normal(0, 0.3, S.NPARAM).astype(np.float32)
    X = rng.random((70, S.IN)).astype(np.float32)
    y = rng.integers(0, 8, 70).astype(np.int32)
    prm = torch.from_numpy(theta).cuda()
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    P = torch.empty((70, 8), dtype=torch.float32, device="cuda")
    act = torch.empty((70, 128), dtype=torch.float32, device="cuda")
    emu.check(emu.emu_sel_forward(h.h, 70, prm.data_ptr(), Xd.data_ptr(), P.data_ptr(), act.data_ptr(), None))
    Pref, _ = S.mlp_forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.allclose(P.cpu().numpy(), Pref, rtol=2e-5, atol=1e-6)
    grad = torch.empty_like(prm)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    emu.check(emu.emu_sel_backward(h.h, 70, prm.data_ptr(), Xd.data_ptr(), act.data_ptr(), P.data_ptr(), yd.data_ptr(),
                                   grad.data_ptr(), loss.data_ptr(), None))
    gref = S.mlp_backward(theta.astype(np.float64), X.astype(np.float64), y)
    g = grad.cpu().numpy()
    assert np.allclose(g, gref, rtol=1e-3, atol=2e-6), np.max(np.abs(g - gref))
    assert abs(float(loss.item()) - S.loss(theta.astype(np.float64), X.astype(np.float64), y)) < 1e-4
    m = torch.zeros_like(prm)
    v = torch.zeros_like(prm)
    emu.check(emu.emu_sel_adam(h.h, prm.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), 1, 1e-3, 0.9, 0.999,
                               1e-8, None))
    tref, _, _ = S.adam(theta.astype(np.float64), g.astype(np.float64), np.zeros(S.NPARAM), np.zeros(S.NPARAM), 1)
    assert np.allclose(prm.cpu().numpy(), tref, rtol=1e-5, atol=1e-7)


def test_probe_dd_vs_oracle(orc, h):
    m, n, k = 30, 20, 777
    A, B = synth.gemm_pair(m, n, k, 4.0, 9)
    idx = np.array([[0, 0], [29, 19], [7, 3], [15, 11]], dtype=np.int32)
    for layout in (0, 1):
        if layout == 0:
            Ad, Bd, lda, ldb = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), k, n
        else:
            Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
            Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
            lda, ldb = m, k
        ref = torch.empty((4, 2), dtype=torch.float64, device="cuda")
        ab = torch.empty(4, dtype=torch.float64, device="cuda")
        di = torch.from_numpy(idx.ravel()).cuda()
        emu.check(emu.emu_probe_dd(h.h, layout, m, n, k, Ad.data_ptr(), lda, Bd.data_ptr(), ldb, 4, di.data_ptr(),
                                   ref.data_ptr(), ab.data_ptr(), None))
        hi, lo = orc.dd_gemm(A, B)
        r = ref.cpu().numpy()
        den = np.abs(A) @ np.abs(B)
        for q, (i, j) in enumerate(idx):
            d = abs((r[q, 0] - hi[i, j]) + (r[q, 1] - lo[i, j]))
            assert d <= den[i, j] * 2.0 ** -95
            assert abs(ab.cpu().numpy()[q] - den[i, j]) <= 1e-13 * den[i, j]


def test_auto_without_weights_uses_bound_and_escalates(h):
    m, n, k = 200, 150, 300
    A, B = synth.gemm_pair(m, n, k, 1.0, 4)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    pb = ctypes.c_int()
    emu.check(emu.emu_bound_p(h.h, 0, m, n, k, Ad.data_ptr(), k, Bd.data_ptr(), n, 1e-10, ctypes.byref(pb), None))
    C, p, code = emu.dgemm_auto(Ad, Bd, 1e-10, handle=h)
    assert code == 0 and p >= pb.value
    ref = emu.dgemm(Ad, Bd, scheme="I", p=p, handle=h)
    assert torch.equal(C, ref)
    # a tolerance no p can meet: escalation up to the maximum, then EMU_ERR_TOL_NOT_MET
    C2, p2, code2 = emu.dgemm_auto(Ad, Bd, 1e-300, handle=h)
    assert code2 == 7 and p2 == emu.EMU_P_MAX


def test_training_beats_fixed_p(h):
    """Small version of the selector experiment: train on 768 products, evaluate on
    256 held out; at every tolerance the learned choice (with probe escalation)
    passes as often as the fixed p (within 3 points), and at tol = 1e-8 it costs
    clearly less on average."""
    ftr, etr, ktr, _ = sel.build_dataset(768, 11)
    fev, eev, kev, _ = sel.build_dataset(256, 12)
    X, y, _ = sel.expand(ftr, etr)
    params, hist = sel.train(X, y, epochs=40, batch=256, lr=3e-3)
    assert hist[-1] < 0.8 * hist[0]
    res = sel.evaluate(params, fev, eev, kev, etr)
    for tol, r in res.items():
        assert r["learned"]["pass_rate"] >= r["fixed"]["pass_rate"] - 0.03, (tol, r)
    # at the loosest tolerance the learned choice is clearly cheaper than the
    # fixed p that every training product needs
    assert res["1e-08"]["speedup_vs_fixed"] > 1.15, res["1e-08"]
    # weights install into a handle and drive emu_dgemm_auto
    sel.install(params, h)
    A, B = synth.gemm_pair(256, 256, 512, 2.0, 77)
    C, p, code = emu.dgemm_auto(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 1e-8, handle=h)
    assert code == 0 and 3 <= p <= emu.EMU_P_MAX


def test_training_resumes_from_checkpoint(tmp_path):
    """A run stopped after 3 of 6 epochs and resumed from its checkpoint ends
    where the uninterrupted run ends: the same shuffles and Adam state, so the
    same loss curve and parameters up to the order of the gradient atomics."""
    ftr, etr, _, _ = sel.build_dataset(256, 21)
    X, y, _ = sel.expand(ftr, etr)
    full, hist_full = sel.train(X, y, epochs=6, batch=256, lr=3e-3, seed=4)
    ck = str(tmp_path / "sel.ckpt")
    _, hist_a = sel.train(X, y, epochs=3, batch=256, lr=3e-3, seed=4, checkpoint=ck)
    assert sel.load_checkpoint(ck)["epoch"] == 3
    resumed, hist_b = sel.train(X, y, epochs=6, batch=256, lr=3e-3, seed=4, checkpoint=ck, resume=True)
    assert len(hist_b) == 6 and hist_b[:3] == hist_a
    assert np.allclose(hist_b, hist_full, rtol=1e-3)
    assert np.allclose(resumed, full, rtol=1e-2, atol=1e-3)
    assert sel.load_checkpoint(ck)["epoch"] == 6
    with pytest.raises(ValueError):  # another learning rate is refused
        sel.train(X, y, epochs=8, batch=256, lr=1e-3, seed=4, checkpoint=ck, resume=True)


def test_auto_II_bound_and_escalation(h):
    m, n, k = 200, 150, 300
    A, B = synth.gemm_pair(m, n, k, 1.0, 5)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    nb = ctypes.c_int()
    emu.check(emu.emu_bound_nm(h.h, 0, m, n, k, Ad.data_ptr(), k, Bd.data_ptr(), n, 1e-10, ctypes.byref(nb), None))
    assert nb.value in sel.NM_CLASSES
    h2 = emu.Handle(0)  # no Scheme II weights: the bound decides
    try:
        C, nm, code = emu.dgemm_auto(Ad, Bd, 1e-10, handle=h2, scheme="II")
        assert code == 0 and nm >= nb.value and nm % 2 == 0
        assert torch.equal(C, emu.dgemm(Ad, Bd, scheme="II_NORM", p=nm, handle=h2))
        C2, nm2, code2 = emu.dgemm_auto(Ad, Bd, 1e-300, handle=h2, scheme="II")
        assert code2 == 7 and nm2 == emu.EMU_NM_MAX
    finally:
        h2.close()


def test_training_II_beats_fixed_nm(h):
    """The Scheme II variant: train on 768 products, evaluate on 256; the
    learned N (with probe escalation) passes as often as the fixed N and costs
    less at tol = 1e-8."""
    ftr, etr, ktr, _ = sel.build_dataset_II(768, 21)
    fev, eev, kev, _ = sel.build_dataset_II(256, 22)
    X, y, _ = sel.expand(ftr, etr)
    params, hist = sel.train(X, y, epochs=40, batch=256, lr=3e-3)
    assert hist[-1] < 0.8 * hist[0]
    res = sel.evaluate_II(params, fev, eev, kev, etr)
    for tol, r in res.items():
        assert r["learned"]["pass_rate"] >= r["fixed"]["pass_rate"] - 0.03, (tol, r)
    assert res["1e-08"]["speedup_vs_fixed"] > 1.1, res["1e-08"]
    sel.install_II(params, h)
    A, B = synth.gemm_pair(256, 256, 512, 2.0, 78)
    C, nm, code = emu.dgemm_auto(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), 1e-8, handle=h, scheme="II")
    assert code == 0 and nm in sel.NM_CLASSES


def test_committed_selector_end_to_end_gain_at_1e8():
    """The committed Scheme I network, timed end to end through
    emu_dgemm_auto -- feature scan, MLP, probe and every escalation inside
    the CUDA-event interval -- against emu_dgemm at the fixed p = 12 (the
    smallest p passing every training product) on held-out products: faster
    in total at tol = 1e-8, and passing on exactly the products the fixed p
    passes (checked on 256 sampled entries against the double-double probe)."""
    hd = emu.Handle(0)
    sel.install_default(hd)
    dev = torch.device("cuda", 0)
    rng = np.random.Generator(np.random.PCG64(31337))
    prods = [(int(round(float(np.exp(rng.uniform(np.log(1024), np.log(2048)))) / 64)) * 64,
              float(rng.uniform(0.0, 8.0)), 8_000_000 + 2 * i) for i in range(8)]
    warm = synth.test_matrix_torch(2048, 2048, 1.0, 1, dev)
    emu.dgemm(warm, warm, scheme="I", p=12, handle=hd)
    emu.dgemm_auto(warm, warm, 1e-8, handle=hd)
    del warm
    t_auto = t_fixed = 0.0
    pass_auto, pass_fixed = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for n, phi, seed in prods:
        A = synth.test_matrix_torch(n, n, phi, seed, dev)
        B = synth.test_matrix_torch(n, n, phi, seed + 1, dev)
        C = torch.empty((n, n), dtype=torch.float64, device=dev)
        Ca = torch.empty((n, n), dtype=torch.float64, device=dev)
        pairs = rng.integers(0, n, size=(256, 2)).astype(np.int32)
        idx = torch.from_numpy(pairs.reshape(-1)).to(dev)
        ref = torch.empty(512, dtype=torch.float64, device=dev)
        ab = torch.empty(256, dtype=torch.float64, device=dev)
        emu.check(emu.emu_probe_dd(hd.h, emu.EMU_ROW_MAJOR, n, n, n, A.data_ptr(), n, B.data_ptr(), n, 256,
                                   idx.data_ptr(), ref.data_ptr(), ab.data_ptr(), None))
        r = ref.cpu().numpy().reshape(256, 2)
        den = ab.cpu().numpy()

        def err(Cx):
            c = Cx.cpu().numpy()[pairs[:, 0], pairs[:, 1]]
            return float(np.max(np.abs((c - r[:, 0]) - r[:, 1]) / den))

        torch.cuda.synchronize()
        e0.record()
        emu.dgemm(A, B, C, scheme="I", p=12, handle=hd)
        e1.record()
        torch.cuda.synchronize()
        t_fixed += e0.elapsed_time(e1)
        pass_fixed.append(err(C) <= 1e-8)
        e0.record()
        Ca, used, code = emu.dgemm_auto(A, B, 1e-8, handle=hd, C=Ca)
        e1.record()
        torch.cuda.synchronize()
        t_auto += e0.elapsed_time(e1)
        assert code == 0 and 3 <= used <= 12
        pass_auto.append(err(Ca) <= 1e-8)
    hd.close()
    assert pass_auto == pass_fixed
    assert t_fixed / t_auto >= 1.05, (t_fixed, t_auto)
