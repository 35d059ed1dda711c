"""Pins of the selector oracle (oracle/selector.py): central finite
differences for the MLP gradient, the Adam update written out by hand, and
histogram features on inputs whose exponents are known."""
import math

import numpy as np

from oracle import selector as S


def test_gradient_matches_finite_differences():
    rng = np.random.Generator(np.random.PCG64(0))
    theta = rng.normal(0, 0.3, S.NPARAM)
    X = rng.random((7, S.IN))
    y = rng.integers(0, S.OUT, 7)
    g = S.mlp_backward(theta, X, y)
    # twelve entries of every parameter block (W1, b1, W2, b2, W3, b3), so a
    # mistake confined to one small block cannot hide between samples
    idx, off = [], 0
    for _, shape in S.SIZES:
        n = int(np.prod(shape))
        idx += list(off + rng.choice(n, min(n, 12), replace=False))
        off += n
    for i in idx:
        e = np.zeros(S.NPARAM)
        e[i] = 1e-6
        num = (S.loss(theta + e, X, y) - S.loss(theta - e, X, y)) / 2e-6
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_forward_is_a_distribution_and_loss_positive():
    rng = np.random.Generator(np.random.PCG64(1))
    theta = rng.normal(0, 0.5, S.NPARAM)
    P, _ = S.mlp_forward(theta, rng.random((5, S.IN)))
    assert np.allclose(P.sum(axis=1), 1.0) and np.all(P > 0)
    assert S.loss(theta, rng.random((5, S.IN)), np.array([0, 1, 2, 3, 4])) > 0


def test_adam_first_step_moves_by_lr():
    theta = np.zeros(4)
    g = np.array([1.0, -2.0, 0.5, 0.0])
    t, m, v = S.adam(theta, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # bias-corrected first step: -lr * g / (|g| + eps)
    assert np.allclose(t[:3], -0.01 * np.sign(g[:3]), atol=1e-9) and t[3] == 0.0


def test_features_known_exponents():
    A = np.array([[1.0, 0.5, 0.25, 0.0], [-3.0, 3.0, 2.0 ** -40, 1.0]])
    A2 = np.array([[2.0 ** -100, 1.0]])  # deficit 100 -> clipped to bin 31
    assert S.features(A2, np.ones((2, 1)), 1e-8)[31] == np.float32(0.5)
    B = np.ones((4, 2))
    f = S.features(A, B, 1e-12)
    # bins of 3 exponents: row 0 (E = 1): deficits 0, 1, 2 -> bin 0, zero -> bin 31
    # row 1 (E = 2, max 3): 3, 3 -> d 0 (bin 0); 2^-40 -> d 41 (bin 13); 1.0 -> d 1 (bin 0)
    expect = np.zeros(32)
    expect[0], expect[13], expect[31] = 6, 1, 1
    assert np.array_equal(f[:32], (expect / 8).astype(np.float32))
    assert f[32] == 1.0 and np.all(f[33:64] == 0)
    assert f[64] == np.float32(math.log2(4) / 16) and f[65] == np.float32(12 / 16)


def test_features_use_the_columns_of_B():
    # B (3 x 2): column 0 = 1, 0.5, 0.25 (E = 1: deficits 0, 1, 2 -> bin 0);
    # column 1 = 8, 2^-10, 0 (E = 4: 8 -> bin 0, 2^-10 has e = -9, deficit 13
    # -> bin 4, the zero -> bin 31).  Its rows would give other bins.
    B = np.array([[1.0, 8.0], [0.5, 2.0 ** -10], [0.25, 0.0]])
    f = S.features(np.ones((1, 3)), B, 1e-6)
    expect = np.zeros(32)
    expect[0], expect[4], expect[31] = 4, 1, 1
    assert np.array_equal(f[32:64], (expect / 6).astype(np.float32))
