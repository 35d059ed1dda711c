"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the emulation method: it only draws
random matrices and shape lists.  Both the CUDA path and the CPU oracle are
fed from it, so the two sides see the same inputs.

Test matrices follow the generator of the EmuGEMM evaluation (Sec. VI-B,
Eq. 19): a_ij = (u - 0.5) * exp(phi * g) with u ~ U(0, 1) and g ~ N(0, 1);
phi widens the exponent range.  Draws use numpy's PCG64 with a fixed seed:
u is drawn first, then g, for the whole matrix.
"""
from __future__ import annotations

import numpy as np


def test_matrix(rows: int, cols: int, phi: float, seed: int, dtype=np.float64) -> np.ndarray:
    """(u - 0.5) * exp(phi * g), row-major, as float64 (or cast to ``dtype``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((rows, cols))
    g = rng.standard_normal((rows, cols))
    a = (u - 0.5) * np.exp(phi * g)
    return a.astype(dtype) if dtype is not np.float64 else a


def test_matrix_complex(rows: int, cols: int, phi: float, seed: int) -> np.ndarray:
    """Complex test matrix: real and imaginary parts from independent seeds."""
    re = test_matrix(rows, cols, phi, seed)
    im = test_matrix(rows, cols, phi, seed + 7919)
    return re + 1j * im


def gemm_pair(m: int, n: int, k: int, phi: float, seed: int, dtype=np.float64):
    """A (m x k) from ``seed`` and B (k x n) from ``seed + 1``."""
    return test_matrix(m, k, phi, seed, dtype), test_matrix(k, n, phi, seed + 1, dtype)


def gemm_pair_complex(m: int, n: int, k: int, phi: float, seed: int):
    return test_matrix_complex(m, k, phi, seed), test_matrix_complex(k, n, phi, seed + 1)


def integer_matrix(rows: int, cols: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Integer-valued float64 matrix with entries uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=(rows, cols)).astype(np.float64)


def grouped_shapes(count: int, seed: int, mn_range=(32, 1024), k_range=(64, 2048)):
    """Uneven problem list: M, N log-uniform in mn_range, K log-uniform in k_range."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.log(mn_range[0]), np.log(mn_range[1])
    klo, khi = np.log(k_range[0]), np.log(k_range[1])
    out = []
    for _ in range(count):
        m = int(round(float(np.exp(rng.uniform(lo, hi)))))
        n = int(round(float(np.exp(rng.uniform(lo, hi)))))
        k = int(round(float(np.exp(rng.uniform(klo, khi)))))
        out.append((m, n, k))
    return out


def test_matrix_torch(rows: int, cols: int, phi: float, seed: int, device):
    """The same generator drawn on a torch device (u first, then g, each for
    the whole matrix, from torch.Generator(device).manual_seed(seed)): for
    benchmark-size operands, which the CPU would take seconds to draw.  The
    values differ from test_matrix's (another random stream), the
    distribution is the same."""
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    u = torch.rand((rows, cols), generator=g, device=device, dtype=torch.float64)
    gn = torch.randn((rows, cols), generator=g, device=device, dtype=torch.float64)
    return (u - 0.5) * torch.exp(phi * gn)
