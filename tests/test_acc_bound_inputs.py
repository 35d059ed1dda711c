"""The accumulator-bound inputs (tests/acc_bound_inputs.py) do what the GPU
tests need them to do, checked with the oracle on the CPU: the scaled
integers are the entries, the residues / digits are the intended ones, the
exact FP32 segment (chunk) sums land just below 2^24, and MMA-block sums
with odd values are added while a running sum is at or above 2^23 (where an
FP32 value's last bit is worth 1).  Also a pin of the oracle on these
integer inputs: Scheme II returns the exact integer product rounded once."""
import numpy as np
import pytest

from acc_bound_inputs import NM_II, SEG, f8_patterns, f8_inputs, largest_odd_residue, scheme_II_inputs


def _odd_blocks_above(prod_terms: np.ndarray, block: int, seg: int) -> tuple[int, int]:
    """Given the exact products of one dot product [k], return (number of
    block sums that are odd and start while the running segment sum is
    >= 2^23 in magnitude, max |segment sum|)."""
    k = prod_terms.shape[0]
    n_odd, mx = 0, 0
    for s0 in range(0, k, seg):
        run = 0
        for b0 in range(s0, min(s0 + seg, k), block):
            bs = int(prod_terms[b0:min(b0 + block, s0 + seg, k)].sum())
            if abs(run) >= 2 ** 23 and bs % 2:
                n_odd += 1
            run += bs
            mx = max(mx, abs(run))
    return n_odd, mx


def test_scheme_II_bound_inputs(orc):
    m, n, k = 6, 16, 2 * SEG + 37
    mods = orc.moduli(NM_II)
    A, B, holes = scheme_II_inputs(m, n, k, mods, seed=3)
    b = orc.scale_bits_II(NM_II, k)
    assert b == 52
    assert np.all(orc.row_exponents(A) == b) and np.all(orc.col_exponents(B) == b)
    RA = orc.residues_II_rows(A, NM_II, b).astype(np.int64)
    RB = orc.residues_II_rows(np.ascontiguousarray(B.T), NM_II, b).astype(np.int64)
    for l in range(6):
        t = largest_odd_residue(mods[l])
        sign = np.where(np.arange(m) % 2 == 0, 1, -1)[:, None]
        assert np.all(RA[l] == sign * t)
        for j in range(n):
            want = np.full(k, t)
            want[holes[j]] = 0
            assert np.array_equal(RB[l, j], want)
        # exact segment sums of the bf16 engine (16-deep MMA blocks, 960-deep segments)
        tot_odd, tot_max = 0, 0
        for i in range(2):
            for j in range(n):
                n_odd, mx = _odd_blocks_above(RA[l, i] * RB[l, j], 16, SEG)
                tot_odd += n_odd
                tot_max = max(tot_max, mx)
        assert tot_max < 2 ** 24
        assert tot_max == SEG * t * t and tot_max >= 2 ** 23.5, np.log2(tot_max)
        assert tot_odd >= 2 * n  # odd increments near the bound in every column
    # pin: exact integer inputs within the CRT bound give the exact product
    # rounded once (Eq. 8 and the exactness condition after it)
    C = orc.emu_II(A, B, NM_II)
    Ai = [[int(x) for x in row] for row in A]
    Bi = [[int(x) for x in row] for row in B]
    for i in range(m):
        for j in range(0, n, 5):
            ex = sum(Ai[i][h] * Bi[h][j] for h in range(k))
            assert C[i, j] == float(ex)


@pytest.mark.parametrize("p", [11, 12])
def test_f8_bound_inputs(orc, p):
    kc = orc.chunk_len_F8(p)
    m, n, k = 4, 12, kc + 77
    A, B, holes = f8_inputs(m, n, k, p, kc, seed=5)
    assert np.all(orc.row_exponents(A) == 5 * p - 1) and np.all(orc.col_exponents(B) == 5 * p - 1)
    pa, pn, pb, ph = f8_patterns(p)
    DA = orc.split_F8_rows(A, p).astype(np.int64)
    DB = orc.split_F8_rows(np.ascontiguousarray(B.T), p).astype(np.int64)
    assert np.array_equal(DA[:, 0, 0], pa) and np.array_equal(DA[:, 1, 0], pn)
    assert np.array_equal(DB[:, 0, 1], pb) and np.array_equal(DB[:, 0, 0], ph)
    # accumulator s = 10 (and every other) over each K_c chunk, 32-deep MMA blocks
    tot_odd, tot_max = 0, 0
    for r in range(2):  # the positive and the negative row pattern
        r_odd, r_max = 0, 0
        for j in range(n):
            for s in range(p):
                terms = sum(DA[i, r] * DB[s - i, j] for i in range(s + 1))
                n_odd, mx = _odd_blocks_above(terms, 32, kc)
                r_odd += n_odd
                r_max = max(r_max, mx)
        assert r_max <= 2 ** 24
        assert r_max >= 2 ** 23.7, (r, np.log2(r_max))
        tot_odd += r_odd
    assert tot_odd >= n
    # the oracle's own chunk partials agree with the digit sums above
    P = orc.partials_F8(A[:1], B[:, :1], p)
    assert np.abs(P).max() == max(
        abs(int(sum(DA[i, 0, c * kc:(c + 1) * kc] @ DB[s - i, 0, c * kc:(c + 1) * kc] for i in range(s + 1))))
        for c in range(2) for s in range(p))
