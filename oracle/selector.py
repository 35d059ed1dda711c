"""CPU oracle for the learned slice-count selector -- TEST INFRASTRUCTURE ONLY.

Plain numpy float64 restatement of what the selector kernels compute (the
paper has no selector; the definitions are the library's own and are stated
in the C ABI header):

* features(A, B, tol): 32-bin histogram of d = E_i - e(a_ij) over the
  sampled rows of A (e = frexp exponent, E_i the row maximum's) in bins of 3
  exponents, bin = min(d // 3, 31), zeros in bin 31, normalised to sum 1; the
  same for the columns of B; log2(k)/16; -log10(tol)/16.
* mlp_forward / mlp_backward: 66 -> 64 -> 64 -> 8, ReLU, softmax, mean
  cross-entropy, parameters packed as W1[64][66], b1, W2[64][64], b2,
  W3[8][64], b3.
* adam: one Adam step with bias correction.

Pinned by central finite differences (tests/test_selector_oracle.py).
"""
from __future__ import annotations

import math

import numpy as np

IN, HID, OUT = 66, 64, 8
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (OUT, HID)), ("b3", (OUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, off = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def _frexp_exp(x: float) -> int:
    return math.frexp(abs(x))[1] if x != 0.0 else 0


def _hist_rows(X, idx):
    h = np.zeros(32, dtype=np.int64)
    for r in idx:
        row = X[r]
        E = _frexp_exp(float(np.max(np.abs(row)))) if row.size else 0
        for v in row:
            if v == 0.0:
                h[31] += 1
            else:
                d = E - _frexp_exp(float(v))
                h[min(max(d, 0) // 3, 31)] += 1
    return h


def sample_index(count: int, sample: int):
    if sample <= 0:
        return list(range(count))
    step = max(1, count // sample)
    return list(range(0, count, step))[:sample]


def features(A, B, tol: float, sample: int = 0) -> np.ndarray:
    A = np.asarray(A, dtype=np.float64)
    Bt = np.ascontiguousarray(np.asarray(B, dtype=np.float64).T)
    k = A.shape[1]
    ha = _hist_rows(A, sample_index(A.shape[0], sample))
    hb = _hist_rows(Bt, sample_index(Bt.shape[0], sample))
    f = np.zeros(IN, dtype=np.float32)
    f[:32] = ha.astype(np.float32) / np.float32(max(ha.sum(), 1))
    f[32:64] = hb.astype(np.float32) / np.float32(max(hb.sum(), 1))
    f[64] = np.float32(math.log2(k) / 16.0)
    f[65] = np.float32(-math.log10(tol) / 16.0)
    return f


def mlp_forward(theta, X):
    """Returns (probabilities [b, 8], cache)."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["W3"].T + p["b3"]
    z3 = z3 - z3.max(axis=1, keepdims=True)
    e = np.exp(z3)
    P = e / e.sum(axis=1, keepdims=True)
    return P, (X, z1, h1, z2, h2)


def loss(theta, X, y) -> float:
    P, _ = mlp_forward(theta, X)
    return float(-np.mean(np.log(P[np.arange(len(y)), y])))


def mlp_backward(theta, X, y):
    """Gradient of the mean cross-entropy with respect to the packed parameters."""
    p = unpack(theta)
    P, (X, z1, h1, z2, h2) = mlp_forward(theta, X)
    b = X.shape[0]
    dz3 = P.copy()
    dz3[np.arange(b), y] -= 1.0
    dz3 /= b
    g = {"W3": dz3.T @ h2, "b3": dz3.sum(axis=0)}
    dh2 = dz3 @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return pack(g)


def adam(theta, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    c1 = 1 - b1 ** step
    c2 = 1 - b2 ** step
    theta = theta - lr * (m / c1) / (np.sqrt(v / c2) + eps)
    return theta, m, v
