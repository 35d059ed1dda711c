"""Inputs that drive the FP32 tensor-core accumulators of the two tcgen05
engines to just below their exact-integer bound (2^24) with odd increments.

Both tcgen05 engines rest on one fact: an FP32 sum of exact integer products
is itself exact while its magnitude stays below 2^24.
* Scheme II on bf16 residues: a segment of 960 K terms of symmetric residue
  products, each |r_a r_b| <= 2^14, sums to at most 960 * 2^14 < 2^24.
* Scheme I on E4M3 digits: accumulator s sums the products of s + 1 digit
  pairs over K_c terms, each |d_a d_b| <= 256, with K_c p 256 <= 2^24.
These inputs make those sums land within a few percent of 2^24 and make the
16- or 32-deep block sums that each MMA adds odd at chosen K positions, so
an accumulator that dropped its last bit near the bound would show up as a
wrong result.

The matrices hold integers whose row (column) maximum sits in the binade
that makes the scaling the identity, so the scaled integers a' of Scheme II
and x of Scheme I are the entries themselves:
* Scheme II: with N_m = 15 and 1024 < k <= 4096 the scale is b = 52 bits;
  every row maximum lies in [2^51, 2^52), so a' = a.  The entries are chosen
  by the CRT so that their residues modulo the first six moduli are the
  largest odd symmetric residues (256, 255 -> 127; 253, 251 -> 125; 247 ->
  123; 241 -> 119).
* Scheme I on E4M3 digits (balanced base-32 digits d_0 in [-16, 16], d_t in
  [-16, 15], x = sum_t d_t 32^(p-1-t)): every entry is x itself (|x| in
  [2^(5p-2), 2^(5p-1)), 53 significant bits) built from digits -15 / -16.
This module holds no arithmetic of the method; it only builds integers.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------- Scheme II
NM_II = 15
SEG = 960  # K terms per exact FP32 segment of the bf16 engine


def _crt_base(mods, targets):
    """Smallest v >= 0 with v = t (mod m) for every (m, t); and prod(mods)."""
    v, M = 0, 1
    for m, t in zip(mods, targets):
        j = ((t - v) * pow(M, -1, m)) % m
        v += M * j
        M *= m
    return v, M


def largest_odd_residue(m: int) -> int:
    half = (m - 1) // 2 if m % 2 else m // 2 - 1  # 256: residues [-128, 127]
    return half if half % 2 else half - 1


def scheme_II_inputs(m: int, n: int, k: int, mods: list[int], seed: int = 0):
    """A (m x k), B (k x n) as described above, plus the list of hole positions.

    `mods` are the first six moduli of the method (the caller takes them from
    its moduli list).  B has "holes" (zeros) at K positions chosen per column
    so that the 16-deep block sums of each segment change parity at offsets
    0, 15, 16 and 959 of a segment, and at random offsets; odd rows of A are
    negated, so half the sums approach -2^24.
    """
    rng = np.random.default_rng(seed)
    ctl = mods[:6]
    targets = [largest_odd_residue(mm) for mm in ctl]
    v0, PiS = _crt_base(ctl, targets)
    lo_q = max(0, -(-(2 ** 51 - v0) // PiS))   # smallest q with v0 + q PiS >= 2^51
    hi_q = (2 ** 52 - 1 - v0) // PiS
    small_q = (2 ** 51 - 1 - v0) // PiS          # entries below 2^51
    assert lo_q <= hi_q and small_q >= 1

    def entries(shape):
        # v0 + q PiS < 2^51: exact in int64 and in binary64
        q = rng.integers(0, small_q + 1, size=shape, dtype=np.int64)
        return (np.int64(v0) + q * np.int64(PiS)).astype(np.float64)

    A = entries((m, k))
    for i in range(m):  # one maximum per row in [2^51, 2^52)
        A[i, rng.integers(0, k)] = float(v0 + int(rng.integers(lo_q, hi_q + 1)) * PiS)
    A[1::2] *= -1.0
    Bt = entries((n, k))
    holes = []
    nseg = -(-k // SEG)
    for j in range(n):
        kind = j % 8
        hj = []
        for s in range(nseg):
            base = s * SEG
            if kind == 0:
                offs = [0]
            elif kind == 1:
                offs = [15]
            elif kind == 2:
                offs = [16]
            elif kind == 3:
                offs = [959]
            elif kind == 4:
                offs = [0, 15, 16, 959]
            elif kind == 5:
                offs = []
            else:
                offs = sorted(rng.choice(SEG, size=3 if kind == 6 else 7, replace=False).tolist())
            hj += [base + o for o in offs if base + o < k]
        Bt[j, hj] = 0.0
        taken = set(hj)
        free = [h for h in range(k) if h not in taken]
        Bt[j, free[int(rng.integers(0, len(free)))]] = float(v0 + int(rng.integers(lo_q, hi_q + 1)) * PiS)
        holes.append(hj)
    return A, np.ascontiguousarray(Bt.T), holes


# ---------------------------------------------------------------- Scheme I, E4M3 digits
def x_from_digits(d) -> int:
    p = len(d)
    return sum(int(v) * 32 ** (p - 1 - t) for t, v in enumerate(d))


def f8_patterns(p: int):
    """Digit patterns (A even rows, A odd rows, B, B hole) for p = 11 or 12.

    A even rows and B: d_0 = -15, d_5 = -15, the other digits -16 (p = 12:
    d_11 = 0, so that x has 53 significant bits).  A odd rows: digits +15
    (the last nonzero one 14, so that x is even), whose products with B are
    negative.  The B hole has d_5 = -16: the product d_5 d_5 of accumulator
    10 turns from 225 (odd) into 240 (even), so a 32-deep block with one hole
    adds an odd number.
    """
    if p == 11:
        base = [-15] + [-16] * 10
        neg = [15] * 10 + [14]
    elif p == 12:
        base = [-15] + [-16] * 10 + [0]
        neg = [15] * 10 + [14, 0]
    else:
        raise ValueError(p)
    pa = list(base)
    pa[5] = -15
    hole = list(base)
    hole[5] = -16
    return pa, neg, list(pa), hole


def f8_inputs(m: int, n: int, k: int, p: int, kc: int, seed: int = 0):
    """A (m x k), B (k x n) for the E4M3 engine, plus the hole positions.

    Every entry is x from the patterns of f8_patterns (an exact binary64
    integer in [2^(5p-2), 2^(5p-1)) in magnitude, so the row / column
    exponent is 5p - 1 and the scaled integer is the entry itself).  B's holes sit at offsets 0, 31, 32 and kc - 1 of
    each K_c chunk, per column kind, and at random offsets.
    """
    rng = np.random.default_rng(seed)
    pa, pn, pb, ph = f8_patterns(p)
    xs = [x_from_digits(d) for d in (pa, pn, pb, ph)]
    for x in xs:
        assert float(x) == x and 2 ** (5 * p - 2) <= abs(x) < 2 ** (5 * p - 1)
    xa, xn, xb, xh = (float(x) for x in xs)
    A = np.full((m, k), xa)
    A[1::2] = xn
    Bt = np.full((n, k), xb)
    holes = []
    nch = -(-k // kc)
    for j in range(n):
        kind = j % 6
        hj = []
        for c in range(nch):
            base = c * kc
            if kind == 0:
                offs = [0]
            elif kind == 1:
                offs = [31]
            elif kind == 2:
                offs = [32]
            elif kind == 3:
                offs = [kc - 1]
            elif kind == 4:
                offs = [0, 31, 32, kc - 1]
            else:
                offs = sorted(rng.choice(kc, size=5, replace=False).tolist())
            hj += [base + o for o in offs if base + o < k]
        Bt[j, hj] = xh
        holes.append(hj)
    return A, np.ascontiguousarray(Bt.T), holes
