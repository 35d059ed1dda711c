"""Training and evaluation of the learned slice-count selector (Scheme I).

Everything numeric runs on the GPU through the C ABI: the feature kernel,
the grouped emulated GEMM that produces the errors the network learns from,
the double-double probe that measures them, and the FP32 MLP forward,
backward and Adam kernels.  Python only orchestrates.

Data (one "matrix" = one product): phi ~ U(0, 8), K log-uniform in
[256, 4096], a 64-row sample of A and a 64-column sample of B drawn from the
test-matrix generator (Sec. VI-B, Eq. 19).  Because Scheme I scales every
row of A and every column of B on its own, the 64 x 64 block of C computed
from these samples is exactly the corresponding block of the full product,
so the sampled rows carry the labels: for p = 3..10 the emulated block is
compared with the double-double product and the label for tolerance tol is
the smallest p with max |C_p - C| / (|A||B|) <= tol (class 7 = "p >= 10").
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import time

import numpy as np

from . import (EMU_COL_MAJOR, EMU_ROW_MAJOR, EMU_SCHEME_II_NORM, GemmDesc, SEL_NPARAM, check, default_handle,
               emu_dgemm, emu_dgemm_grouped, emu_moduli, emu_probe_dd, emu_sel_adam, emu_sel_backward,
               emu_sel_features, emu_sel_forward, emu_sel_load, emu_sel_load_II, _stream_ptr)

P0, NCLS = 3, 8
P_TOP = 12  # escalation goes up to the library's largest p
TOLS = (1e-8, 1e-12, 1e-15)
SUB = 64
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.json")
# Scheme II (norm-based scaling): classes N = 6, 8, .., 20 moduli
NM_CLASSES = tuple(range(6, 21, 2))
WEIGHTS_II = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights_II.json")


def _torch():
    import torch
    return torch


def gen_batch(seeds, device, k_range=(256, 4096), phi_range=(0.0, 8.0)):
    """Sampled operands for a list of integer seeds: [(phi, k, A_sub, B_sub)]."""
    torch = _torch()
    out = []
    for s in seeds:
        g = torch.Generator(device="cpu").manual_seed(int(s))
        phi = float(torch.rand((), generator=g)) * (phi_range[1] - phi_range[0]) + phi_range[0]
        lk = float(torch.rand((), generator=g)) * (math.log(k_range[1]) - math.log(k_range[0])) + math.log(k_range[0])
        k = int(round(math.exp(lk)))
        gd = torch.Generator(device=device).manual_seed(int(s) * 7 + 1)
        A = (torch.rand((SUB, k), generator=gd, device=device, dtype=torch.float64) - 0.5) * torch.exp(
            phi * torch.randn((SUB, k), generator=gd, device=device, dtype=torch.float64))
        B = (torch.rand((k, SUB), generator=gd, device=device, dtype=torch.float64) - 0.5) * torch.exp(
            phi * torch.randn((k, SUB), generator=gd, device=device, dtype=torch.float64))
        out.append((phi, k, A, B))
    return out


def batch_errors(batch, h, stream=None, ps=range(P0, P_TOP + 1)):
    """err[i, j] = max-relative error of the emulated block at p = ps[j]
    (p = 3..12: the classes 3..10 plus the escalation range)."""
    torch = _torch()
    dev = batch[0][2].device
    n = len(batch)
    C = [torch.empty((SUB, SUB), dtype=torch.float64, device=dev) for _ in range(n)]
    descs = (GemmDesc * n)()
    for i, (_, k, A, B) in enumerate(batch):
        descs[i] = GemmDesc(SUB, SUB, k, 1.0, 0.0, A.data_ptr(), k, B.data_ptr(), SUB, C[i].data_ptr(), SUB)
    # double-double reference of every entry of each block
    ii, jj = np.meshgrid(np.arange(SUB), np.arange(SUB), indexing="ij")
    idx = torch.from_numpy(np.stack([ii.ravel(), jj.ravel()], 1).astype(np.int32).ravel()).to(dev)
    ref = torch.empty((n, SUB * SUB, 2), dtype=torch.float64, device=dev)
    ab = torch.empty((n, SUB * SUB), dtype=torch.float64, device=dev)
    sp = _stream_ptr(stream)
    for i, (_, k, A, B) in enumerate(batch):
        check(emu_probe_dd(h.h, 0, SUB, SUB, k, A.data_ptr(), k, B.data_ptr(), SUB, SUB * SUB, idx.data_ptr(),
                           ref[i].data_ptr(), ab[i].data_ptr(), sp), "emu_probe_dd")
    hi, lo = ref[..., 0], ref[..., 1]
    errs = torch.empty((n, len(list(ps))), dtype=torch.float64, device=dev)
    for j, p in enumerate(ps):
        check(emu_dgemm_grouped(h.h, n, descs, p, sp), "emu_dgemm_grouped")
        Cs = torch.stack(C).reshape(n, SUB * SUB)
        d = ((Cs - hi) - lo).abs()
        rel = torch.where(ab > 0, d / torch.where(ab > 0, ab, torch.ones_like(ab)), torch.where(d > 0, math.inf, 0.0))
        errs[:, j] = rel.max(dim=1).values
    return errs.cpu().numpy()


def batch_features(batch, h, stream=None):
    """Histogram features (tolerance entry set later): float32 [n, 66]."""
    torch = _torch()
    dev = batch[0][2].device
    out = torch.empty((len(batch), 66), dtype=torch.float32, device=dev)
    sp = _stream_ptr(stream)
    for i, (_, k, A, B) in enumerate(batch):
        check(emu_sel_features(h.h, 0, SUB, SUB, k, A.data_ptr(), k, B.data_ptr(), SUB, 1.0, 0, out[i].data_ptr(),
                               sp), "emu_sel_features")
    return out.cpu().numpy()


def labels_from_errors(errs, tol):
    """Class of the smallest p in 3..10 meeting tol; class 7 means "10 or more"."""
    ok = errs[:, :NCLS] <= tol
    lab = np.full(errs.shape[0], NCLS - 1, dtype=np.int32)
    for i in range(errs.shape[0]):
        w = np.nonzero(ok[i])[0]
        if len(w):
            lab[i] = w[0]
    return lab


def build_dataset(n_mats, seed, device="cuda", batch=256, log=None):
    """features [n, 66] (tol entry 0), errors [n, 10] for p = 3..12, k [n], phi [n]."""
    h = default_handle(0)
    feats, errs, ks, phis = [], [], [], []
    t0 = time.time()
    for b0 in range(0, n_mats, batch):
        seeds = [seed * 1000003 + i for i in range(b0, min(n_mats, b0 + batch))]
        bt = gen_batch(seeds, device)
        feats.append(batch_features(bt, h))
        errs.append(batch_errors(bt, h))
        ks += [k for _, k, _, _ in bt]
        phis += [phi for phi, _, _, _ in bt]
        if log:
            log("dataset %d/%d %.1fs" % (min(n_mats, b0 + batch), n_mats, time.time() - t0))
    return np.concatenate(feats), np.concatenate(errs), np.array(ks), np.array(phis)


def expand(feats, errs):
    """One sample per (matrix, tolerance): X [3n, 66], y [3n], tol index [3n]."""
    X, y, ti = [], [], []
    for t, tol in enumerate(TOLS):
        f = feats.copy()
        f[:, 65] = np.float32(-math.log10(tol) / 16.0)
        X.append(f)
        y.append(labels_from_errors(errs, tol))
        ti.append(np.full(len(f), t))
    return np.concatenate(X).astype(np.float32), np.concatenate(y).astype(np.int32), np.concatenate(ti)


def init_params(seed=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fan_in, fan_out in ((66, 64), (64, 64), (64, 8)):
        parts.append(rng.normal(0.0, math.sqrt(2.0 / fan_in), (fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == SEL_NPARAM
    return theta


CKPT_VERSION = 1


def save_checkpoint(path, params, m, v, step, epoch, rng_state, hist, seed, lr):
    """Training state after `epoch` finished epochs: the parameters, Adam's
    moment estimates and step count, the state of the shuffling generator
    and the loss history, written atomically (a temporary file, then a
    rename), so that an interrupted run leaves the last complete state."""
    meta = {"version": CKPT_VERSION, "n_param": int(SEL_NPARAM), "step": int(step), "epoch": int(epoch),
            "rng": rng_state, "hist": [float(x) for x in hist], "seed": int(seed), "lr": float(lr)}
    tmp = "%s.tmp.%d" % (path, os.getpid())
    try:
        with open(tmp, "wb") as fh:
            np.savez(fh, params=np.asarray(params, dtype=np.float32), m=np.asarray(m, dtype=np.float32),
                     v=np.asarray(v, dtype=np.float32), meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8))
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.remove(tmp)
        raise


def load_checkpoint(path):
    """The state save_checkpoint wrote: dict with params, m, v (float32
    arrays) and step, epoch, rng, hist, seed, lr; ValueError for another
    format version or network size."""
    with np.load(path) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        if meta.get("version") != CKPT_VERSION or meta.get("n_param") != SEL_NPARAM:
            raise ValueError("selector checkpoint %s: version %s, %s parameters (expected %d, %d)" %
                             (path, meta.get("version"), meta.get("n_param"), CKPT_VERSION, SEL_NPARAM))
        out = {k: np.array(z[k], dtype=np.float32) for k in ("params", "m", "v")}
    out.update({k: meta[k] for k in ("step", "epoch", "rng", "hist", "seed", "lr")})
    return out


def train(X, y, epochs=60, batch=512, lr=2e-3, seed=0, log=None, checkpoint=None, resume=False):
    """Adam on the mean cross-entropy with the library's kernels; returns
    (params float32 [8968], loss history).  checkpoint: a file that receives
    the training state after every epoch; resume: continue from it (same
    data, seed and learning rate) up to `epochs` epochs in total."""
    torch = _torch()
    h = default_handle(0)
    dev = torch.device("cuda")
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    step, start, hist = 0, 0, []
    if resume and checkpoint and os.path.exists(checkpoint):
        ck = load_checkpoint(checkpoint)
        if ck["seed"] != seed or ck["lr"] != lr:
            raise ValueError("selector checkpoint %s was written with seed %d, lr %g" %
                             (checkpoint, ck["seed"], ck["lr"]))
        prm, m, v = (torch.from_numpy(ck[k]).to(dev) for k in ("params", "m", "v"))
        step, start, hist = ck["step"], ck["epoch"], list(ck["hist"])
        rng.bit_generator.state = ck["rng"]
        if log:
            log("resumed from %s after epoch %d (step %d)" % (checkpoint, start, step))
    else:
        prm = torch.from_numpy(init_params(seed)).to(dev)
        m = torch.zeros_like(prm)
        v = torch.zeros_like(prm)
    grad = torch.zeros_like(prm)
    lossd = torch.zeros(1, dtype=torch.float32, device=dev)
    Xd = torch.from_numpy(X).to(dev)
    yd = torch.from_numpy(y).to(dev)
    n = len(y)
    P = torch.empty((batch, 8), dtype=torch.float32, device=dev)
    act = torch.empty((batch, 128), dtype=torch.float32, device=dev)
    sp = _stream_ptr(None)
    for ep in range(start, epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(dev)
        tot = 0.0
        nb = 0
        for b0 in range(0, n, batch):
            sel = perm[b0:b0 + batch]
            xb = Xd[sel].contiguous()
            ybt = yd[sel].contiguous()
            bs = len(sel)
            check(emu_sel_forward(h.h, bs, prm.data_ptr(), xb.data_ptr(), P.data_ptr(), act.data_ptr(), sp))
            check(emu_sel_backward(h.h, bs, prm.data_ptr(), xb.data_ptr(), act.data_ptr(), P.data_ptr(),
                                   ybt.data_ptr(), grad.data_ptr(), lossd.data_ptr(), sp))
            step += 1
            check(emu_sel_adam(h.h, prm.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), step, lr, 0.9,
                               0.999, 1e-8, sp))
            tot += float(lossd.item())
            nb += 1
        hist.append(tot / max(nb, 1))
        if checkpoint:
            save_checkpoint(checkpoint, prm.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy(), step, ep + 1,
                            rng.bit_generator.state, hist, seed, lr)
        if log and (ep % 10 == 0 or ep == epochs - 1):
            log("epoch %d loss %.4f" % (ep, hist[-1]))
    return prm.cpu().numpy(), hist


def predict(params, X, q=0.8):
    """Probabilities by the library's forward kernel, then the smallest class
    whose cumulative probability reaches q (the emu_dgemm_auto rule)."""
    torch = _torch()
    h = default_handle(0)
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    prm = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).to(dev)
    P = torch.empty((len(X), 8), dtype=torch.float32, device=dev)
    check(emu_sel_forward(h.h, len(X), prm.data_ptr(), Xd.data_ptr(), P.data_ptr(), None, _stream_ptr(None)))
    Pn = P.cpu().numpy()
    c = np.cumsum(Pn, axis=1)
    return np.argmax(c >= q, axis=1), Pn


def bound_class(feats, ks, tols):
    """Bound-based choice (the emu_bound_p rule) as a class index."""
    out = []
    for f, k, tol in zip(feats, ks, tols):
        spread = max([3 * (i % 32) + 2 for i in range(64) if f[i] > 0] or [0])
        cls = NCLS - 1
        for p in range(P0, P0 + NCLS):
            if math.ldexp(1.0, -8 * p + 3 + spread) * k <= tol:
                cls = p - P0
                break
        out.append(cls)
    return np.array(out)


def cost(p):
    return p * (p + 1)  # INT8 GEMMs of Scheme I, proportional to the run time


def evaluate(params, feats, errs, ks, train_errs):
    """Per tolerance: pass rate, mean p and mean cost (INT8 GEMM count summed
    over attempts) of
      learned -- the selector's p (the open-ended top class "10 or more"
                 starts at 12), checked by the probe; on a miss p is raised to
                 max(p + 1, bound p), then to 12 (the emu_dgemm_auto rule);
      fixed   -- the smallest p in 3..12 that passes every training product;
      bound   -- the bound-based p alone.
    errs / train_errs: [n, 10] errors for p = 3..12."""
    res = {}
    top = P_TOP - P0
    for t, tol in enumerate(TOLS):
        f = feats.copy()
        f[:, 65] = np.float32(-math.log10(tol) / 16.0)
        cls, _ = predict(params, f)
        bcls = bound_class(f, ks, [tol] * len(f))
        ok_train = train_errs <= tol
        fixed = top
        for c in range(top + 1):
            if np.all(ok_train[:, c]):
                fixed = c
                break
        learned_p, learned_cost, learned_pass = [], [], []
        for i in range(len(f)):
            c = int(cls[i])
            if c == NCLS - 1:  # open-ended top class: start at the largest p
                c = top
            cst = cost(P0 + c)
            tries = [max(c + 1, int(bcls[i])) if c < NCLS - 1 else top, top]
            for nxt in tries:
                if errs[i, c] <= tol or c >= top:
                    break
                c = min(nxt, top)
                cst += cost(P0 + c)
            learned_p.append(P0 + c)
            learned_cost.append(cst)
            learned_pass.append(errs[i, c] <= tol)
        fixed_pass = errs[:, fixed] <= tol
        bound_pass = errs[np.arange(len(f)), bcls] <= tol
        bound_cost = float(np.mean([cost(P0 + c) for c in bcls]))
        res["%g" % tol] = {
            "learned": {"pass_rate": float(np.mean(learned_pass)), "mean_p": float(np.mean(learned_p)),
                        "mean_cost": float(np.mean(learned_cost)),
                        "first_try_rate": float(np.mean(errs[np.arange(len(f)), np.where(cls == NCLS - 1, top, cls)] <= tol))},
            "fixed": {"p": P0 + fixed, "pass_rate": float(np.mean(fixed_pass)), "mean_cost": float(cost(P0 + fixed))},
            "bound": {"pass_rate": float(np.mean(bound_pass)), "mean_p": float(np.mean(P0 + bcls)),
                      "mean_cost": bound_cost},
            "speedup_vs_fixed": float(cost(P0 + fixed) / np.mean(learned_cost)),
            "speedup_vs_bound": float(bound_cost / np.mean(learned_cost)),
        }
    return res


# ---------------------------------------------------------------- Scheme II
def batch_errors_II(batch, h, stream=None, nms=NM_CLASSES):
    """err[i, j] = max-relative error of the 64 x 64 block with Scheme II
    (norm-based scaling) and N = nms[j] moduli.  Scheme II scales every row
    of A and column of B on its own too, so the block equals that block of
    the full product."""
    torch = _torch()
    dev = batch[0][2].device
    n = len(batch)
    ii, jj = np.meshgrid(np.arange(SUB), np.arange(SUB), indexing="ij")
    idx = torch.from_numpy(np.stack([ii.ravel(), jj.ravel()], 1).astype(np.int32).ravel()).to(dev)
    ref = torch.empty((n, SUB * SUB, 2), dtype=torch.float64, device=dev)
    ab = torch.empty((n, SUB * SUB), dtype=torch.float64, device=dev)
    C = torch.empty((n, len(nms), SUB, SUB), dtype=torch.float64, device=dev)
    sp = _stream_ptr(stream)
    for i, (_, k, A, B) in enumerate(batch):
        check(emu_probe_dd(h.h, 0, SUB, SUB, k, A.data_ptr(), k, B.data_ptr(), SUB, SUB * SUB, idx.data_ptr(),
                           ref[i].data_ptr(), ab[i].data_ptr(), sp), "emu_probe_dd")
        for j, nm in enumerate(nms):
            check(emu_dgemm(h.h, EMU_ROW_MAJOR, SUB, SUB, k, 1.0, A.data_ptr(), k, B.data_ptr(), SUB, 0.0,
                            C[i, j].data_ptr(), SUB, EMU_SCHEME_II_NORM, nm, sp), "emu_dgemm")
    hi, lo = ref[..., 0].unsqueeze(1), ref[..., 1].unsqueeze(1)
    d = ((C.reshape(n, len(nms), SUB * SUB) - hi) - lo).abs()
    abb = ab.unsqueeze(1)
    rel = torch.where(abb > 0, d / torch.where(abb > 0, abb, torch.ones_like(abb)), torch.where(d > 0, math.inf, 0.0))
    return rel.max(dim=2).values.cpu().numpy()


def build_dataset_II(n_mats, seed, device="cuda", batch=256, log=None):
    """features [n, 66] (tol entry 0), errors [n, 8] for N = 6, 8, .., 20, k [n], phi [n]."""
    h = default_handle(0)
    feats, errs, ks, phis = [], [], [], []
    t0 = time.time()
    for b0 in range(0, n_mats, batch):
        seeds = [seed * 1000003 + i for i in range(b0, min(n_mats, b0 + batch))]
        bt = gen_batch(seeds, device)
        feats.append(batch_features(bt, h))
        errs.append(batch_errors_II(bt, h))
        ks += [k for _, k, _, _ in bt]
        phis += [phi for phi, _, _, _ in bt]
        if log:
            log("dataset II %d/%d %.1fs" % (min(n_mats, b0 + batch), n_mats, time.time() - t0))
    return np.concatenate(feats), np.concatenate(errs), np.array(ks), np.array(phis)


def _scale_bits_II(nm):
    """Shared scale bits h of the norm-based scaling: floor((floor(log2 P) - 1) / 2)."""
    mods = (ctypes.c_int32 * nm)()
    emu_moduli(nm, mods)
    P = math.prod(int(x) for x in mods)
    return (P.bit_length() - 2) // 2


def bound_class_II(feats, ks, tols):
    """Bound-based N (the emu_bound_nm rule) as a class index."""
    hs = [_scale_bits_II(nm) for nm in NM_CLASSES]
    out = []
    for f, k, tol in zip(feats, ks, tols):
        spread = max([3 * (i % 32) + 2 for i in range(64) if f[i] > 0] or [0])
        half_lk = 0
        while (1 << (2 * half_lk)) < k:
            half_lk += 1
        cls = NCLS - 1
        for c, h in enumerate(hs):
            if math.ldexp(1.0, -h + spread + half_lk + 3) <= tol:
                cls = c
                break
        out.append(cls)
    return np.array(out)


def evaluate_II(params, feats, errs, ks, train_errs):
    """As evaluate for Scheme II: classes N = 6, 8, .., 20, cost N (INT8 GEMMs);
    the top class is N = 20 itself, a miss escalates to max(N + 2, bound N),
    then to 20."""
    res = {}
    top = NCLS - 1
    for tol in TOLS:
        f = feats.copy()
        f[:, 65] = np.float32(-math.log10(tol) / 16.0)
        cls, _ = predict(params, f)
        bcls = bound_class_II(f, ks, [tol] * len(f))
        ok_train = train_errs <= tol
        fixed = top
        for c in range(top + 1):
            if np.all(ok_train[:, c]):
                fixed = c
                break
        used, costs, passed = [], [], []
        for i in range(len(f)):
            c = int(cls[i])
            cst = NM_CLASSES[c]
            tries = [max(c + 1, int(bcls[i])) if c < top else top, top]
            for nxt in tries:
                if errs[i, c] <= tol or c >= top:
                    break
                c = min(nxt, top)
                cst += NM_CLASSES[c]
            used.append(NM_CLASSES[c])
            costs.append(cst)
            passed.append(errs[i, c] <= tol)
        bound_cost = float(np.mean([NM_CLASSES[c] for c in bcls]))
        res["%g" % tol] = {
            "learned": {"pass_rate": float(np.mean(passed)), "mean_nm": float(np.mean(used)),
                        "mean_cost": float(np.mean(costs)),
                        "first_try_rate": float(np.mean(errs[np.arange(len(f)), cls] <= tol))},
            "fixed": {"nm": NM_CLASSES[fixed], "pass_rate": float(np.mean(errs[:, fixed] <= tol)),
                      "mean_cost": float(NM_CLASSES[fixed])},
            "bound": {"pass_rate": float(np.mean(errs[np.arange(len(f)), bcls] <= tol)),
                      "mean_nm": float(np.mean([NM_CLASSES[c] for c in bcls])), "mean_cost": bound_cost},
            "speedup_vs_fixed": float(NM_CLASSES[fixed] / np.mean(costs)),
            "speedup_vs_bound": float(bound_cost / np.mean(costs)),
        }
    return res


def install_II(params, handle=None):
    h = handle or default_handle(0)
    arr = np.ascontiguousarray(params, dtype=np.float32)
    check(emu_sel_load_II(h.h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "emu_sel_load_II")


def save_weights(params, path=WEIGHTS, meta=None):
    with open(path, "w") as fh:
        json.dump({"n_param": int(SEL_NPARAM), "params": [float(x) for x in params], "meta": meta or {}}, fh)


def load_weights(path=WEIGHTS):
    with open(path) as fh:
        d = json.load(fh)
    return np.array(d["params"], dtype=np.float32), d.get("meta", {})


def install(params, handle=None):
    h = handle or default_handle(0)
    arr = np.ascontiguousarray(params, dtype=np.float32)
    check(emu_sel_load(h.h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "emu_sel_load")


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="train / evaluate the learned slice-count selector")
    ap.add_argument("--n-train", type=int, default=20000)
    ap.add_argument("--n-eval", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--report", default=None)
    ap.add_argument("--scheme", default="I", choices=["I", "II"],
                    help="I: slices p = 3..10; II: moduli N = 6..20 of Scheme II with norm scaling")
    ap.add_argument("--checkpoint", default=None, help="file for the training state after every epoch")
    ap.add_argument("--resume", action="store_true", help="continue the training from --checkpoint")
    a = ap.parse_args(argv)
    if a.scheme == "II" and a.out == WEIGHTS:
        a.out = WEIGHTS_II
    log = lambda s: print(s, flush=True)  # noqa: E731
    build = build_dataset_II if a.scheme == "II" else build_dataset
    t0 = time.time()
    ftr, etr, ktr, _ = build(a.n_train, 1, log=log)
    fev, eev, kev, _ = build(a.n_eval, 2, log=log)
    t_data = time.time() - t0
    X, y, _ = expand(ftr, etr)
    t1 = time.time()
    params, hist = train(X, y, epochs=a.epochs, log=log, checkpoint=a.checkpoint, resume=a.resume)
    t_train = time.time() - t1
    res = (evaluate_II if a.scheme == "II" else evaluate)(params, fev, eev, kev, etr)
    meta = {"scheme": a.scheme, "n_train": a.n_train, "n_eval": a.n_eval, "epochs": a.epochs, "final_loss": hist[-1],
            "first_loss": hist[0], "data_seconds": t_data, "train_seconds": t_train}
    save_weights(params, a.out, meta)
    report = {"meta": meta, "eval": res}
    print(json.dumps(report, indent=1), flush=True)
    if a.report:
        with open(a.report, "w") as fh:
            json.dump(report, fh, indent=1)


def install_default(handle=None):
    """Install the committed weights of both selectors (Scheme I p and
    Scheme II N) in a handle, so emu_dgemm_auto / emu_dgemm_auto_II use them."""
    if os.path.exists(WEIGHTS):
        install(load_weights(WEIGHTS)[0], handle)
    if os.path.exists(WEIGHTS_II):
        install_II(load_weights(WEIGHTS_II)[0], handle)


if __name__ == "__main__":
    main()
