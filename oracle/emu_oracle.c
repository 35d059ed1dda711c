/*
 * emu_oracle.c -- plain, slow CPU oracle for the emulated-GEMM hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product path (the CUDA library under paper_2606_25453_gb300/) never links,
 * imports or calls it, and this file shares no code, header, table or
 * constant generator with it.
 *
 * Every function follows the EmuGEMM paper (Lu, Maeder, Luisier, Ziogas,
 * "EmuGEMM: Fused Tensor Core Kernels for Precision Emulation in Matrix
 * Multiplication") step by step, in the paper's order and notation:
 *   Scheme I   -- Sec. II-C-1, Eqs. (1)-(3); interleaving Eq. (11); the
 *                 signed-leading/unsigned-tail slice encoding of Sec. VII.
 *   Scheme II  -- Sec. II-C-2, Eqs. (4)-(8) plus the inverse scaling that
 *                 follows Eq. (8).
 *   3M complex -- Sec. IV-B, Eq. (16).
 * Integer work is exact (int64 / __int128 / multi-word); floating-point
 * work is IEEE binary64 with an explicitly fixed operation order so that a
 * GPU implementation of the same definition can be compared bit for bit.
 * Build with -ffp-contract=off: no implicit fused multiply-adds.
 *
 * Matrices are dense row-major.  The B operand is passed TRANSPOSED
 * (Bt = B^T, N x K row-major) so that columns of B are rows of Bt.
 *
 * Readings of points the paper leaves open (each is also listed in the
 * design notes of the repository):
 *   R1  slice width beta = 8; x = trunc(a * 2^(8p-1-E)) with E the
 *       frexp exponent of the row maximum; slices are the bytes of the
 *       8p-bit two's complement of x, the leading one signed, the rest
 *       unsigned (Sec. II-C-1 and Sec. VII).
 *   R2  The shift-reduce of Eq. (3) is done exactly: the partials C_s are
 *       exact integers, S = sum_s C_s * 256^(p-1-s) is formed in integer
 *       arithmetic and rounded ONCE to binary64 (nearest, ties to even), then
 *       scaled by 2^(E_i + F_j - 14 - 8(p-1)).  This makes the paper's
 *       statement that the shift-reduce adds no rounding error beyond the
 *       decomposition residual (Sec. III-B) hold literally; a binary64 sum
 *       of the p terms would lose bits to cancellation between slices of the
 *       two's-complement encoding.  Because S is exact, the result does not
 *       depend on how K is chunked; a GPU keeps its INT32 accumulators exact
 *       by draining them every K_c (largest multiple of 256 with worst-case
 *       |C_s| <= 2^31-1, orc_chunk_len_I) into an exact wider integer.
 *   R3  Scheme II scaling: b = floor((floor(log2 P) - 1 - ceil(log2 k))/2)
 *       (complex: -2 instead of -1), a' = trunc(a * 2^(b - E_i)); this is
 *       the largest b for which the exactness condition after Eq. (8)
 *       holds for every input.
 *   R4  moduli: the greedy descending pairwise-coprime list 256, 255, 253,
 *       251, ...; operand residues are stored symmetrically in
 *       [-floor(m/2), floor((m-1)/2)]; output residues in [0, m).
 *   R5  CRT result lifted to the symmetric range (-P/2, P/2], rounded to
 *       binary64 (nearest, ties to even), then scaled by a power of two.
 *   R6  BLAS update: beta == 0 -> C = alpha * r (C not read), else
 *       C = fma(alpha, r, beta * C).
 *   R7  Scheme I on FP8 (E4M3) slices -- the FP8 formulation the paper names
 *       as future work (Sec. VII) on the same interleaved layout (Sec. III-A
 *       notes the layout is agnostic to the slice type): beta = 5,
 *       x = trunc(a * 2^(5p-1-E)), balanced base-32 digits (d_t in [-16, 15]
 *       for t >= 1, d_0 in [-16, 16]), all exactly representable in E4M3, so
 *       every slice product is exact and FP32 sums of them are exact while
 *       |sum| <= 2^24.  Result: RN(S) * 2^(E_i + F_j - 8 - 5(p-1)) with
 *       S = sum_s 32^(p-1-s) C_s exact.
 *   R8  Scheme I complex (the 4M formulation the paper uses for its Scheme I
 *       CGEMM/ZGEMM, Sec. VI): one exponent per complex row of A and per
 *       complex column of B (over real and imaginary parts); the four real
 *       products are the triangle sums T_s(X, Y) = sum_{t<=s} <X_t, Y_{s-t}>
 *       of Eq. (2) on the slices of Re A, Im A, Re B, Im B and of -Im B (the
 *       slices of the negated integers, as for any other operand), combined
 *       exactly before the single rounding of R2:
 *         S_re = sum_s w_s (T_s(Re A, Re B) + T_s(Im A, -Im B)),
 *         S_im = sum_s w_s (T_s(Re A, Im B) + T_s(Im A, Re B)),
 *       w_s = 2^(beta (p-1-s)).  This is Scheme I applied to the real
 *       matrices [Re A, Im A] and [[Re B, Im B], [-Im B, Re B]].  The complex
 *       BLAS update is that of R6 for complex numbers.
 *   R9  Scheme II with norm-based scaling (a data-dependent bound for the
 *       exactness condition after Eq. (8), in place of R3's worst case):
 *       Cauchy-Schwarz gives sum_h |a'_ih||b'_hj| <= ||a'_i||_2 ||b'_j||_2,
 *       so with e_i = an integer with ||a_i||_2 < 2^e_i (f_j likewise for the
 *       columns of B) and a' = trunc(a * 2^(h - e_i)), b' = trunc(b *
 *       2^(h - f_j)), h = floor((floor(log2 P) - 1)/2) for both operands (so
 *       the product is symmetric in A and B and does not depend on which one
 *       is stored transposed), the condition 2 sum |a'||b'| < 2^(2h+1)
 *       <= 2^floor(log2 P) <= P holds for every input.  e_i is computed exactly so that any implementation
 *       finds the same value: with E the frexp exponent of the row maximum
 *       and y = a 2^-E (|y| < 1), S = sum_h ceil(y_h^2 2^64) (integers, an
 *       upper bound of 2^64 ||y||^2), e_i = E + ceil((bitlen(S) - 64)/2);
 *       all-zero rows get e_i = 0.  Complex rows use |y|^2 = re^2 + im^2; the
 *       same hA, hB apply (|Re C'|, |Im C'| <= ||a_i|| ||b_j|| over complex
 *       norms).  Result RN(C') * 2^(e_i + f_j - 2h).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;
typedef unsigned __int128 u128;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Power-of-two scale vectors mu, nu (Eq. 1; Scheme II scaling)        */
/* ------------------------------------------------------------------ */

/* E = smallest integer with max_h |x_h| < 2^E (the frexp exponent of the
 * maximum); 0 for an all-zero row.  Returns 1 if the row holds a NaN or an
 * infinity, else 0. */
static int row_exponent(const double *x, int64_t n, int *E) {
  double mx = 0.0;
  for (int64_t h = 0; h < n; ++h) {
    double v = fabs(x[h]);
    if (!(v <= 1.7976931348623157e308)) return 1; /* NaN or inf */
    if (v > mx) mx = v;
  }
  int e = 0;
  if (mx != 0.0) frexp(mx, &e);
  *E = e;
  return 0;
}

/* Row exponents of a rows x cols row-major matrix.  Returns the number of
 * rows that hold non-finite values. */
int64_t orc_row_exponents(int64_t rows, int64_t cols, const double *X, int32_t *E) {
  int64_t bad = 0;
#pragma omp parallel for reduction(+ : bad) schedule(static)
  for (int64_t i = 0; i < rows; ++i) {
    int e = 0;
    bad += row_exponent(X + i * cols, cols, &e);
    E[i] = e;
  }
  return bad;
}

/* Complex variant: one exponent per row over both real and imaginary parts
 * (interleaved re, im pairs). */
int64_t orc_row_exponents_z(int64_t rows, int64_t cols, const double *X, int32_t *E) {
  return orc_row_exponents(rows, 2 * cols, X, E);
}

/* Reading R9: exact norm exponents.  ceil(y^2 2^64) for y = x 2^-E, |y| < 1,
 * from the integer mantissa of x (y^2 = M^2 2^(2(ex - 53 - E)) with
 * x = M 2^(ex-53), 2^52 <= M < 2^53). */
static u128 sq_ceil64(double x, int E) {
  if (x == 0.0) return 0;
  int ex;
  double f = frexp(fabs(x), &ex);
  uint64_t M = (uint64_t)ldexp(f, 53);
  u128 M2 = (u128)M * (u128)M; /* < 2^106 */
  int s = 2 * (ex - 53 - E) + 64;
  if (s >= 0) return M2 << s; /* y^2 2^64 < 2^64 */
  if (-s >= 128) return 1;   /* nonzero, below one unit */
  u128 q = M2 >> (-s);
  if ((q << (-s)) != M2) q += 1;
  return q;
}

static int bitlen128(u128 v) {
  int L = 0;
  while (v) {
    ++L;
    v >>= 1;
  }
  return L;
}

/* e per row of a rows x cols matrix (cw = 1 real, 2 complex interleaved).
 * Returns the number of rows with non-finite entries (then E is unusable). */
int64_t orc_norm_exponents(int64_t rows, int64_t cols, int cw, const double *X, int32_t *E) {
  int64_t bad = 0;
  for (int64_t i = 0; i < rows; ++i) {
    int Emax;
    if (row_exponent(X + i * cols * cw, cols * cw, &Emax)) {
      ++bad;
      E[i] = 0;
      continue;
    }
    u128 S = 0;
    for (int64_t h = 0; h < cols * cw; ++h) S += sq_ceil64(X[i * cols * cw + h], Emax);
    if (S == 0) {
      E[i] = 0;
      continue;
    }
    int d = bitlen128(S) - 64; /* e' = ceil(d / 2) */
    int ep = d >= 0 ? (d + 1) / 2 : -((-d) / 2);
    E[i] = Emax + ep;
  }
  return bad;
}

int orc_log2P_floor(int nm);

/* Reading R9: the scale bits of A and B (equal). */
void orc_norm_halves_II(int nm, int *hA, int *hB) {
  int L = orc_log2P_floor(nm) - 1;
  *hA = L >= 0 ? L / 2 : -((-L + 1) / 2);
  *hB = *hA;
}

/* trunc(a * 2^shift) as an exact integer.  a = M * 2^(e-53) with the
 * 53-bit integer significand M from frexp; the shifted value is
 * M * 2^(e-53+shift), truncated toward zero.  The caller guarantees
 * |result| < 2^126. */
static i128 scaled_trunc(double a, int shift) {
  if (a == 0.0) return 0;
  int e;
  double f = frexp(fabs(a), &e);              /* |a| = f * 2^e, f in [0.5,1) */
  uint64_t M = (uint64_t)ldexp(f, 53);         /* exact: 2^52 <= M < 2^53 */
  int sh = e - 53 + shift;
  u128 mag;
  if (sh >= 0)
    mag = (u128)M << sh;
  else if (sh > -64)
    mag = (u128)(M >> (-sh));
  else
    mag = 0;
  return a < 0 ? -(i128)mag : (i128)mag;
}

/* ------------------------------------------------------------------ */
/* Scheme I                                                            */
/* ------------------------------------------------------------------ */

/* Slice decomposition of one operand (Eq. 1 with beta = 8, reading R1).
 * X: rows x k row-major, E: its row exponents.  D: p x rows x k int16,
 * D[t][i][h] = slice t of x_ih (t = 0 signed in [-128,127], t >= 1 in
 * [0,255]), so that x_ih = sum_t D[t][i][h] * 256^(p-1-t) and
 * a_ih ~= 2^(E_i - 7) * sum_t 2^(-8t) D[t][i][h]. */
void orc_split_I(int64_t rows, int64_t k, const double *X, const int32_t *E, int p, int16_t *D) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < rows; ++i) {
    for (int64_t h = 0; h < k; ++h) {
      i128 x = scaled_trunc(X[i * k + h], 8 * p - 1 - E[i]);
      u128 u = (u128)x; /* two's complement bits */
      for (int t = 0; t < p; ++t) {
        int byte = (int)((u >> (8 * (p - 1 - t))) & 0xFF);
        if (t == 0 && byte >= 128) byte -= 256;
        D[((int64_t)t * rows + i) * k + h] = (int16_t)byte;
      }
    }
  }
}

/* Interleaved layout of Eq. (11): Ahat[i][(c*p + t)*tk + r] = D[t][i][c*tk + r]
 * for K-chunk c of width tk.  K is padded with zero slices up to a multiple
 * of tk; kpad = ceil(k/tk)*tk.  Output is int8 bytes (two's complement for
 * the signed leading slice, raw bytes for unsigned tails). */
void orc_interleave(int64_t rows, int64_t k, int p, int tk, const int16_t *D, int8_t *Ahat) {
  int64_t nck = (k + tk - 1) / tk;
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t c = 0; c < nck; ++c)
      for (int t = 0; t < p; ++t)
        for (int r = 0; r < tk; ++r) {
          int64_t h = c * tk + r;
          int v = h < k ? D[((int64_t)t * rows + i) * k + h] : 0;
          Ahat[i * nck * p * tk + (c * p + t) * tk + r] = (int8_t)(uint8_t)(v & 0xFF);
        }
}

/* Worst-case |C_s| per unit of K over s = 0..p-1 for the slice ranges of R1,
 * and the chunk length K_c of reading R2. */
int64_t orc_chunk_len_I(int p) {
  int64_t bnd = 128 * 128; /* s = 0: signed x signed */
  if (p >= 2) {
    int64_t neg = 2 * 128 * 255;                       /* two signed x unsigned terms */
    int64_t pos = 2 * 127 * 255 + (int64_t)(p - 2) * 255 * 255; /* s = p-1 */
    if (neg > bnd) bnd = neg;
    if (pos > bnd) bnd = pos;
  }
  int64_t lim = 2147483647LL / bnd;
  return (lim / 256) * 256;
}

/* Exact chunked partials of Eq. (2):
 * Cs[c][s][i][j] = sum_{t=0..s} sum_{h in chunk c} DA[t][i][h] * DB[s-t][j][h]
 * with DB the slices of Bt (rows of Bt are columns of B). */
void orc_partials_I(int64_t m, int64_t n, int64_t k, int p, int64_t kc, const int16_t *DA,
                    const int16_t *DB, int64_t *Cs) {
  int64_t nch = (k + kc - 1) / kc;
  if (k == 0) nch = 0;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j)
      for (int64_t c = 0; c < nch; ++c) {
        int64_t h0 = c * kc, h1 = h0 + kc < k ? h0 + kc : k;
        for (int s = 0; s < p; ++s) {
          int64_t acc = 0;
          for (int t = 0; t <= s; ++t) {
            const int16_t *a = DA + ((int64_t)t * m + i) * k;
            const int16_t *b = DB + ((int64_t)(s - t) * n + j) * k;
            for (int64_t h = h0; h < h1; ++h) acc += (int64_t)a[h] * (int64_t)b[h];
          }
          Cs[((c * p + s) * m + i) * n + j] = acc;
        }
      }
}

/* BLAS update of reading R6. */
static double blas_update(double alpha, double r, double beta, double c) {
  if (beta == 0.0) return alpha * r;
  return fma(alpha, r, beta * c);
}

/* Round an exact integer to the nearest binary64, ties to even, from its
 * two's-complement bits (reading R2; no library conversion involved). */
static double i128_to_double(i128 v) {
  int neg = v < 0;
  u128 a = neg ? (u128)0 - (u128)v : (u128)v;
  if (a == 0) return 0.0;
  int L = 0;
  for (u128 t = a; t; t >>= 1) ++L; /* bit length */
  double r;
  if (L <= 53) {
    r = (double)(uint64_t)a; /* exact */
  } else {
    int drop = L - 53;
    uint64_t top = (uint64_t)(a >> drop);
    u128 rest = a - ((u128)top << drop);
    u128 half = (u128)1 << (drop - 1);
    if (rest > half || (rest == half && (top & 1))) top += 1; /* may reach 2^53: exact */
    r = ldexp((double)top, drop);
  }
  return neg ? -r : r;
}

/* Full Scheme I emulated product (Eqs. 1-3, readings R1, R2, R6):
 *   S = sum_s 256^(p-1-s) * sum_{t<=s} sum_h DA[t][i][h] DB[s-t][j][h]  (exact)
 *   r = RN(S) * 2^(E_i + F_j - 14 - 8(p-1))   (ldexp; one more rounding only
 *                                               if the result is subnormal)
 *   C = blas_update(alpha, r, beta, C)
 * A: m x k, Bt: n x k, C: m x n (in/out).
 * If out_f32 is nonzero the binary64 value is rounded once more to binary32
 * and written to Cf (m x n float, in/out, read when beta != 0) instead of C.
 * Returns 0, or -1 on non-finite input. */
int orc_emu_I(int64_t m, int64_t n, int64_t k, int p, double alpha, const double *A,
              const double *Bt, double beta, double *C, float *Cf, int out_f32) {
  int32_t *E = malloc(sizeof(int32_t) * (m > 0 ? m : 1));
  int32_t *F = malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  int16_t *DA = malloc(sizeof(int16_t) * (size_t)(p * m * k > 0 ? p * m * k : 1));
  int16_t *DB = malloc(sizeof(int16_t) * (size_t)(p * n * k > 0 ? p * n * k : 1));
  int rc = 0;
  if (orc_row_exponents(m, k, A, E) || orc_row_exponents(n, k, Bt, F)) {
    rc = -1;
    goto out;
  }
  orc_split_I(m, k, A, E, p, DA);
  orc_split_I(n, k, Bt, F, p, DB);
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      i128 S = 0;
      for (int s = 0; s < p; ++s) {
        int64_t Cs = 0; /* exact: |C_s| < 2^63 for any k used here */
        for (int t = 0; t <= s; ++t) {
          const int16_t *a = DA + ((int64_t)t * m + i) * k;
          const int16_t *b = DB + ((int64_t)(s - t) * n + j) * k;
          for (int64_t h = 0; h < k; ++h) Cs += (int64_t)a[h] * (int64_t)b[h];
        }
        S += (i128)Cs << (8 * (p - 1 - s));
      }
      double r = ldexp(i128_to_double(S), E[i] + F[j] - 14 - 8 * (p - 1));
      if (out_f32)
        Cf[i * n + j] = (float)blas_update(alpha, r, beta, beta == 0.0 ? 0.0 : (double)Cf[i * n + j]);
      else
        C[i * n + j] = blas_update(alpha, r, beta, beta == 0.0 ? 0.0 : C[i * n + j]);
    }
out:
  free(E);
  free(F);
  free(DA);
  free(DB);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Multi-word unsigned integers for the CRT (little-endian 32-bit limbs) */
/* ------------------------------------------------------------------ */

#define NL 8 /* 256 bits: enough for P of up to 24 moduli (< 2^192) plus carries */
typedef struct {
  uint32_t w[NL];
} big;

static void big_zero(big *a) { memset(a, 0, sizeof(*a)); }
static void big_set_u32(big *a, uint32_t v) {
  big_zero(a);
  a->w[0] = v;
}
static int big_cmp(const big *a, const big *b) {
  for (int i = NL - 1; i >= 0; --i)
    if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
  return 0;
}
static void big_add(big *r, const big *a, const big *b) {
  uint64_t c = 0;
  for (int i = 0; i < NL; ++i) {
    c += (uint64_t)a->w[i] + b->w[i];
    r->w[i] = (uint32_t)c;
    c >>= 32;
  }
}
static void big_sub(big *r, const big *a, const big *b) { /* requires a >= b */
  int64_t br = 0;
  for (int i = 0; i < NL; ++i) {
    int64_t d = (int64_t)a->w[i] - b->w[i] - br;
    br = d < 0;
    r->w[i] = (uint32_t)(d + (br ? ((int64_t)1 << 32) : 0));
  }
}
static void big_mul_u32(big *r, const big *a, uint32_t v) {
  uint64_t c = 0;
  for (int i = 0; i < NL; ++i) {
    c += (uint64_t)a->w[i] * v;
    r->w[i] = (uint32_t)c;
    c >>= 32;
  }
}
static uint32_t big_mod_u32(const big *a, uint32_t m) {
  uint64_t r = 0;
  for (int i = NL - 1; i >= 0; --i) r = ((r << 32) | a->w[i]) % m;
  return (uint32_t)r;
}
static int big_bitlen(const big *a) {
  for (int i = NL - 1; i >= 0; --i)
    if (a->w[i]) {
      int b = 32;
      while (!(a->w[i] >> (b - 1))) --b;
      return 32 * i + b;
    }
  return 0;
}
static int big_bit(const big *a, int pos) { return (a->w[pos / 32] >> (pos % 32)) & 1; }

/* Round a nonnegative multi-word integer to the nearest binary64, ties to
 * even (reading R5). */
static double big_to_double(const big *a) {
  int L = big_bitlen(a);
  if (L == 0) return 0.0;
  if (L <= 53) {
    uint64_t v = (uint64_t)a->w[0] | ((uint64_t)a->w[1] << 32);
    return (double)v; /* exact */
  }
  /* top 53 bits */
  uint64_t top = 0;
  for (int b = L - 1; b >= L - 53; --b) top = (top << 1) | (uint64_t)big_bit(a, b);
  int guard = big_bit(a, L - 54);
  int sticky = 0;
  for (int b = L - 55; b >= 0 && !sticky; --b) sticky = big_bit(a, b);
  if (guard && (sticky || (top & 1))) top += 1; /* may carry to 2^53: still exact */
  return ldexp((double)top, L - 53);
}

/* ------------------------------------------------------------------ */
/* Scheme II                                                           */
/* ------------------------------------------------------------------ */

static int gcd_i(int a, int b) {
  while (b) {
    int t = a % b;
    a = b;
    b = t;
  }
  return a;
}

/* Reading R4: the first nm entries of the greedy descending list of
 * pairwise-coprime integers starting at 256.  Returns the count found. */
int orc_moduli(int nm, int32_t *mods) {
  int cnt = 0;
  for (int x = 256; x >= 2 && cnt < nm; --x) {
    int ok = 1;
    for (int j = 0; j < cnt && ok; ++j) ok = gcd_i(x, mods[j]) == 1;
    if (ok) mods[cnt++] = x;
  }
  return cnt;
}

static void product_P(int nm, const int32_t *mods, big *P) {
  big_set_u32(P, 1);
  for (int l = 0; l < nm; ++l) big_mul_u32(P, P, (uint32_t)mods[l]);
}

/* floor(log2 P) for the first nm moduli. */
int orc_log2P_floor(int nm) {
  int32_t mods[32];
  orc_moduli(nm, mods);
  big P;
  product_P(nm, mods, &P);
  return big_bitlen(&P) - 1;
}

/* Reading R3: scaling exponent b. */
int orc_scale_bits_II(int nm, int64_t k, int is_complex) {
  int c = 0;
  while (((int64_t)1 << c) < k) ++c; /* ceil(log2 k), 0 for k <= 1 */
  int num = orc_log2P_floor(nm) - (is_complex ? 2 : 1) - c;
  /* floor division toward -inf */
  return num >= 0 ? num / 2 : -((-num + 1) / 2);
}

/* mathematical x mod m in [0, m), then the symmetric operand residue */
static int sym_residue(i128 x, int m) {
  int r = (int)(x % m);
  if (r < 0) r += m;
  if (r > (m - 1) / 2) r -= m;
  return r;
}

/* Eq. (5): integer scaling a' = trunc(a * 2^(b - E_i)) and symmetric
 * residues R[l][i][h] of a' modulo m_l.  X: rows x k real (stride 1) or,
 * when is_complex, interleaved (re, im) with part selecting 0 = re, 1 = im,
 * 2 = the 3M sum (a'_re + a'_im). */
void orc_residues_II(int64_t rows, int64_t k, const double *X, const int32_t *E, int b, int nm,
                     int is_complex, int part, int8_t *R) {
  int32_t mods[32];
  orc_moduli(nm, mods);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t h = 0; h < k; ++h) {
      i128 v;
      if (!is_complex) {
        v = scaled_trunc(X[i * k + h], b - E[i]);
      } else {
        i128 re = scaled_trunc(X[2 * (i * k + h)], b - E[i]);
        i128 im = scaled_trunc(X[2 * (i * k + h) + 1], b - E[i]);
        v = part == 0 ? re : part == 1 ? im : re + im;
      }
      for (int l = 0; l < nm; ++l) R[((int64_t)l * rows + i) * k + h] = (int8_t)sym_residue(v, mods[l]);
    }
}

/* Eqs. (6)-(7): per-modulus exact products and output residues in [0, m).
 * RA: nm x m x k, RB: nm x n x k (residues of Bt).  Out: nm x m x n. */
void orc_modprod_II(int64_t m, int64_t n, int64_t k, int nm, const int8_t *RA, const int8_t *RB,
                    uint8_t *Out) {
  int32_t mods[32];
  orc_moduli(nm, mods);
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j)
      for (int l = 0; l < nm; ++l) {
        const int8_t *a = RA + ((int64_t)l * m + i) * k;
        const int8_t *b = RB + ((int64_t)l * n + j) * k;
        int64_t acc = 0;
        for (int64_t h = 0; h < k; ++h) acc += (int64_t)a[h] * (int64_t)b[h];
        int64_t r = acc % mods[l];
        if (r < 0) r += mods[l];
        Out[((int64_t)l * m + i) * n + j] = (uint8_t)r;
      }
}

/* Table of the CRT weights of Eq. (8): T[l][r] = ((P/m_l) * q_l * r) mod P,
 * built by repeated modular addition. */
typedef struct {
  int nm;
  int32_t mods[32];
  big P, halfP_floor;
  big *T; /* nm x 256 */
} crt_ctx;

static int crt_init(crt_ctx *cx, int nm) {
  cx->nm = nm;
  orc_moduli(nm, cx->mods);
  product_P(nm, cx->mods, &cx->P);
  /* floor(P/2) */
  big h = cx->P;
  for (int i = 0; i < NL; ++i) h.w[i] = (h.w[i] >> 1) | (i + 1 < NL ? (h.w[i + 1] << 31) : 0);
  cx->halfP_floor = h;
  cx->T = malloc(sizeof(big) * 256 * (size_t)(nm > 0 ? nm : 1));
  if (!cx->T) return -1;
  for (int l = 0; l < nm; ++l) {
    int ml = cx->mods[l];
    big Pl; /* P / m_l as the product of the other moduli */
    big_set_u32(&Pl, 1);
    for (int j = 0; j < nm; ++j)
      if (j != l) big_mul_u32(&Pl, &Pl, (uint32_t)cx->mods[j]);
    int pm = (int)big_mod_u32(&Pl, (uint32_t)ml);
    int q = 0; /* modular inverse of P/m_l modulo m_l, by search */
    for (int c = 1; c < ml || (ml == 1 && c == 1); ++c)
      if ((pm * c) % ml == 1 % ml) {
        q = c;
        break;
      }
    big w;
    big_mul_u32(&w, &Pl, (uint32_t)q); /* (P/m_l) q_l < P */
    big_zero(&cx->T[l * 256 + 0]);
    for (int r = 1; r < 256; ++r) {
      big s;
      big_add(&s, &cx->T[l * 256 + r - 1], &w);
      if (big_cmp(&s, &cx->P) >= 0) big_sub(&s, &s, &cx->P);
      cx->T[l * 256 + r] = s;
    }
  }
  return 0;
}
static void crt_free(crt_ctx *cx) { free(cx->T); }

/* Eq. (8) with reading R5: the symmetric integer C' as a binary64 value
 * rounded to nearest (the integer itself is exact before the rounding). */
static double crt_value(const crt_ctx *cx, const uint8_t *res, int64_t stride) {
  big S;
  big_zero(&S);
  for (int l = 0; l < cx->nm; ++l) {
    big_add(&S, &S, &cx->T[l * 256 + res[(int64_t)l * stride]]);
    if (big_cmp(&S, &cx->P) >= 0) big_sub(&S, &S, &cx->P);
  }
  if (big_cmp(&S, &cx->halfP_floor) > 0) { /* S > P/2 -> S - P < 0 */
    big mag;
    big_sub(&mag, &cx->P, &S);
    return -big_to_double(&mag);
  }
  return big_to_double(&S);
}

/* Exposed for pinning: CRT of nm residue vectors (res: nm x cnt, each in
 * [0, m_l)) to binary64 values out[cnt]. */
int orc_crt(int nm, int64_t cnt, const uint8_t *res, double *out) {
  crt_ctx cx;
  if (crt_init(&cx, nm)) return -1;
  for (int64_t e = 0; e < cnt; ++e) out[e] = crt_value(&cx, res + e, cnt);
  crt_free(&cx);
  return 0;
}

/* Full Scheme II emulated real product (Eqs. 5-8, readings R3-R6).
 * A: m x k, Bt: n x k, C: m x n in/out (or Cf when out_f32). */
/* norm = 0: reading R3 (row-maximum exponents, one b); norm = 1: R9. */
int orc_emu_II_ex(int64_t m, int64_t n, int64_t k, int nm, int norm, double alpha, const double *A,
                  const double *Bt, double beta, double *C, float *Cf, int out_f32) {
  int32_t *E = malloc(sizeof(int32_t) * (m > 0 ? m : 1));
  int32_t *F = malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  int8_t *RA = malloc((size_t)(nm * m * k > 0 ? nm * m * k : 1));
  int8_t *RB = malloc((size_t)(nm * n * k > 0 ? nm * n * k : 1));
  uint8_t *O = malloc((size_t)(nm * m * n > 0 ? nm * m * n : 1));
  int rc = 0;
  crt_ctx cx;
  cx.T = NULL;
  if (norm ? (orc_norm_exponents(m, k, 1, A, E) || orc_norm_exponents(n, k, 1, Bt, F))
           : (orc_row_exponents(m, k, A, E) || orc_row_exponents(n, k, Bt, F))) {
    rc = -1;
    goto out;
  }
  {
    int bA, bB;
    if (norm) {
      orc_norm_halves_II(nm, &bA, &bB);
    } else {
      bA = bB = orc_scale_bits_II(nm, k, 0);
    }
    orc_residues_II(m, k, A, E, bA, nm, 0, 0, RA);
    orc_residues_II(n, k, Bt, F, bB, nm, 0, 0, RB);
    orc_modprod_II(m, n, k, nm, RA, RB, O);
    if (crt_init(&cx, nm)) {
      rc = -2;
      goto out;
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double v = crt_value(&cx, O + i * n + j, m * n);
        double r = ldexp(v, E[i] + F[j] - bA - bB);
        if (out_f32)
          Cf[i * n + j] = (float)blas_update(alpha, r, beta, beta == 0.0 ? 0.0 : (double)Cf[i * n + j]);
        else
          C[i * n + j] = blas_update(alpha, r, beta, beta == 0.0 ? 0.0 : C[i * n + j]);
      }
  }
out:
  if (cx.T) crt_free(&cx);
  free(E);
  free(F);
  free(RA);
  free(RB);
  free(O);
  return rc;
}

int orc_emu_II(int64_t m, int64_t n, int64_t k, int nm, double alpha, const double *A, const double *Bt,
               double beta, double *C, float *Cf, int out_f32) {
  return orc_emu_II_ex(m, n, k, nm, 0, alpha, A, Bt, beta, C, Cf, out_f32);
}

/* ------------------------------------------------------------------ */
/* 3M complex Scheme II (Sec. IV-B, Eq. 16)                            */
/* ------------------------------------------------------------------ */

/* Per-modulus 3M output residues: for modulus l,
 *   T1 = Are*Bre, T2 = Aim*Bim, T3 = Asum*Bsum (each mod m_l in [0, m_l)),
 *   Re = (T1 - T2) mod m_l, Im = (T3 - T1 - T2) mod m_l.
 * Inputs are the three residue sets of each operand (nm x rows x k). */
void orc_modprod_Z3M(int64_t m, int64_t n, int64_t k, int nm, const int8_t *Are, const int8_t *Aim,
                     const int8_t *Asum, const int8_t *Bre, const int8_t *Bim, const int8_t *Bsum,
                     uint8_t *ORe, uint8_t *OIm) {
  int32_t mods[32];
  orc_moduli(nm, mods);
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j)
      for (int l = 0; l < nm; ++l) {
        int64_t ml = mods[l], t[3];
        const int8_t *as[3] = {Are, Aim, Asum}, *bs[3] = {Bre, Bim, Bsum};
        for (int q = 0; q < 3; ++q) {
          const int8_t *a = as[q] + ((int64_t)l * m + i) * k;
          const int8_t *b = bs[q] + ((int64_t)l * n + j) * k;
          int64_t acc = 0;
          for (int64_t h = 0; h < k; ++h) acc += (int64_t)a[h] * (int64_t)b[h];
          t[q] = ((acc % ml) + ml) % ml;
        }
        int64_t re = ((t[0] - t[1]) % ml + ml) % ml;
        int64_t im = ((t[2] - t[0] - t[1]) % ml + 2 * ml) % ml;
        ORe[((int64_t)l * m + i) * n + j] = (uint8_t)re;
        OIm[((int64_t)l * m + i) * n + j] = (uint8_t)im;
      }
}

/* Complex BLAS update (reading R6 applied to complex numbers):
 *   t_re = alpha_re*r_re - alpha_im*r_im, t_im = alpha_re*r_im + alpha_im*r_re,
 * each as fma(x, y, -(u*v)) / fma(x, y, u*v); beta != 0 adds
 *   beta*c computed the same way, then one addition per component. */
static void zupdate(double ar, double ai, double rr, double ri, double br, double bi, double *cr,
                    double *ci) {
  double tr = fma(ar, rr, -(ai * ri));
  double ti = fma(ar, ri, ai * rr);
  if (br != 0.0 || bi != 0.0) {
    double ur = fma(br, *cr, -(bi * *ci));
    double ui = fma(br, *ci, bi * *cr);
    tr = tr + ur;
    ti = ti + ui;
  }
  *cr = tr;
  *ci = ti;
}

/* Full 3M complex emulated product.  A: m x k complex (interleaved re, im),
 * Bt: n x k complex (Bt = B^T, NOT conjugated), C: m x n complex in/out.
 * With out_f32 the result goes to Cf (m x n complex float, read when beta
 * != 0): the complex update is done in binary64 as for C, then each part is
 * rounded once more to binary32 (CGEMM). */
static int emu_Z3M_core(int64_t m, int64_t n, int64_t k, int nm, int norm, double alpha_re, double alpha_im,
                        const double *A, const double *Bt, double beta_re, double beta_im, double *C, float *Cf,
                        int out_f32) {
  int32_t *E = malloc(sizeof(int32_t) * (m > 0 ? m : 1));
  int32_t *F = malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  size_t sa = (size_t)(nm * m * k > 0 ? nm * m * k : 1), sb = (size_t)(nm * n * k > 0 ? nm * n * k : 1);
  size_t so = (size_t)(nm * m * n > 0 ? nm * m * n : 1);
  int8_t *A3 = malloc(3 * sa), *B3 = malloc(3 * sb);
  uint8_t *ORe = malloc(so), *OIm = malloc(so);
  int rc = 0;
  crt_ctx cx;
  cx.T = NULL;
  if (norm ? (orc_norm_exponents(m, k, 2, A, E) || orc_norm_exponents(n, k, 2, Bt, F))
           : (orc_row_exponents_z(m, k, A, E) || orc_row_exponents_z(n, k, Bt, F))) {
    rc = -1;
    goto out;
  }
  {
    int bA, bB;
    if (norm) {
      orc_norm_halves_II(nm, &bA, &bB);
    } else {
      bA = bB = orc_scale_bits_II(nm, k, 1);
    }
    for (int q = 0; q < 3; ++q) {
      orc_residues_II(m, k, A, E, bA, nm, 1, q, A3 + q * sa);
      orc_residues_II(n, k, Bt, F, bB, nm, 1, q, B3 + q * sb);
    }
    orc_modprod_Z3M(m, n, k, nm, A3, A3 + sa, A3 + 2 * sa, B3, B3 + sb, B3 + 2 * sb, ORe, OIm);
    if (crt_init(&cx, nm)) {
      rc = -2;
      goto out;
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double vr = crt_value(&cx, ORe + i * n + j, m * n);
        double vi = crt_value(&cx, OIm + i * n + j, m * n);
        double rr = ldexp(vr, E[i] + F[j] - bA - bB);
        double ri = ldexp(vi, E[i] + F[j] - bA - bB);
        double cr = 0.0, ci = 0.0;
        if (beta_re != 0.0 || beta_im != 0.0) {
          cr = out_f32 ? (double)Cf[2 * (i * n + j)] : C[2 * (i * n + j)];
          ci = out_f32 ? (double)Cf[2 * (i * n + j) + 1] : C[2 * (i * n + j) + 1];
        }
        zupdate(alpha_re, alpha_im, rr, ri, beta_re, beta_im, &cr, &ci);
        if (out_f32) {
          Cf[2 * (i * n + j)] = (float)cr;
          Cf[2 * (i * n + j) + 1] = (float)ci;
        } else {
          C[2 * (i * n + j)] = cr;
          C[2 * (i * n + j) + 1] = ci;
        }
      }
  }
out:
  if (cx.T) crt_free(&cx);
  free(E);
  free(F);
  free(A3);
  free(B3);
  free(ORe);
  free(OIm);
  return rc;
}

int orc_emu_Z3M(int64_t m, int64_t n, int64_t k, int nm, double alpha_re, double alpha_im,
                const double *A, const double *Bt, double beta_re, double beta_im, double *C) {
  return emu_Z3M_core(m, n, k, nm, 0, alpha_re, alpha_im, A, Bt, beta_re, beta_im, C, NULL, 0);
}

/* CGEMM by the 3M method: A, Bt complex double (the complex64 inputs widened
 * exactly), Cf complex float in/out. */
int orc_emu_C3M(int64_t m, int64_t n, int64_t k, int nm, double alpha_re, double alpha_im,
                const double *A, const double *Bt, double beta_re, double beta_im, float *Cf) {
  return emu_Z3M_core(m, n, k, nm, 0, alpha_re, alpha_im, A, Bt, beta_re, beta_im, NULL, Cf, 1);
}

/* 3M with the norm-based scaling of R9; out_f32 selects Cf (CGEMM). */
int orc_emu_Z3M_norm(int64_t m, int64_t n, int64_t k, int nm, double alpha_re, double alpha_im,
                     const double *A, const double *Bt, double beta_re, double beta_im, double *C, float *Cf,
                     int out_f32) {
  return emu_Z3M_core(m, n, k, nm, 1, alpha_re, alpha_im, A, Bt, beta_re, beta_im, C, Cf, out_f32);
}

/* ------------------------------------------------------------------ */
/* Double-double reference product (accuracy reference, not the method) */
/* ------------------------------------------------------------------ */

/* Compensated dot product (Ogita-Rump-Oishi Dot2): TwoProduct via fma and
 * TwoSum accumulation.  Result (hi, lo) with hi + lo ~ sum_h x_h*y_h to about
 * k^2 * 2^-106 relative to sum_h |x_h y_h|. */
static void dot2(const double *x, int64_t sx, const double *y, int64_t sy, int64_t k, double sign_odd,
                 double *hi, double *lo) {
  double s = 0.0, c = 0.0;
  for (int64_t h = 0; h < k; ++h) {
    double a = x[h * sx], b = y[h * sy];
    if (sign_odd != 0.0 && (h & 1)) a = -a;
    double p = a * b;
    double e = fma(a, b, -p);
    double t = s + p;
    double z = t - s;
    double err = (s - (t - z)) + (p - z);
    s = t;
    c += err + e;
  }
  double t = s + c;
  *lo = c - (t - s);
  *hi = t;
}

/* Real: Cref = A * B with A m x k, Bt n x k. */
void orc_dd_gemm(int64_t m, int64_t n, int64_t k, const double *A, const double *Bt, double *hi,
                 double *lo) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) dot2(A + i * k, 1, Bt + j * k, 1, k, 0.0, hi + i * n + j, lo + i * n + j);
}

/* Complex: A m x k, Bt n x k interleaved complex.  The real part is the dot
 * product of (a_re, a_im) with (b_re, -b_im) over 2k interleaved terms; the
 * imaginary part pairs (a_re, a_im) with (b_im, b_re). */
void orc_dd_zgemm(int64_t m, int64_t n, int64_t k, const double *A, const double *Bt, double *hi,
                  double *lo) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      const double *a = A + 2 * i * k, *b = Bt + 2 * j * k;
      dot2(a, 1, b, 1, 2 * k, 1.0, hi + 2 * (i * n + j), lo + 2 * (i * n + j));
      /* imaginary: sum a_re*b_im + a_im*b_re, i.e. x = a, y = swapped b */
      double s = 0.0, c = 0.0;
      for (int64_t h = 0; h < k; ++h) {
        double xs[2] = {a[2 * h], a[2 * h + 1]}, ys[2] = {b[2 * h + 1], b[2 * h]};
        for (int q = 0; q < 2; ++q) {
          double p = xs[q] * ys[q];
          double e = fma(xs[q], ys[q], -p);
          double t = s + p;
          double z = t - s;
          double err = (s - (t - z)) + (p - z);
          s = t;
          c += err + e;
        }
      }
      double t = s + c;
      lo[2 * (i * n + j) + 1] = c - (t - s);
      hi[2 * (i * n + j) + 1] = t;
    }
}

/* ------------------------------------------------------------------ */
/* Scheme I on FP8 (E4M3) slices (reading R7)                          */
/* ------------------------------------------------------------------ */

/* Balanced base-32 digits of x = trunc(a * 2^(5p-1-E)): from the lowest
 * digit up, d = x mod 32 taken in [-16, 15], x = (x - d) / 32; the remaining
 * x is the leading digit.  D: p x rows x k int16. */
void orc_split_F8(int64_t rows, int64_t k, const double *X, const int32_t *E, int p, int16_t *D) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t h = 0; h < k; ++h) {
      i128 x = scaled_trunc(X[i * k + h], 5 * p - 1 - E[i]);
      for (int t = p - 1; t >= 1; --t) {
        int r = (int)(x % 32);
        if (r < 0) r += 32;
        if (r >= 16) r -= 32;
        D[((int64_t)t * rows + i) * k + h] = (int16_t)r;
        x = (x - r) / 32;
      }
      D[i * k + h] = (int16_t)x;
    }
}

/* K_c for FP32-exact accumulation: every |d_i d_j| <= 256, so |C_s| grows by
 * at most (s+1)*256 per unit of K; largest multiple of 256 keeping all
 * partial sums within 2^24. */
int64_t orc_chunk_len_F8(int p) {
  int64_t worst = (int64_t)p * 256;
  int64_t lim = ((int64_t)1 << 24) / worst;
  return (lim / 256) * 256;
}

/* Full emulated product with E4M3 slices (reading R7), as orc_emu_I. */
int orc_emu_F8(int64_t m, int64_t n, int64_t k, int p, double alpha, const double *A, const double *Bt,
               double beta, double *C, float *Cf, int out_f32) {
  int32_t *E = malloc(sizeof(int32_t) * (m > 0 ? m : 1));
  int32_t *F = malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  int16_t *DA = malloc(sizeof(int16_t) * (size_t)(p * m * k > 0 ? p * m * k : 1));
  int16_t *DB = malloc(sizeof(int16_t) * (size_t)(p * n * k > 0 ? p * n * k : 1));
  int rc = 0;
  if (orc_row_exponents(m, k, A, E) || orc_row_exponents(n, k, Bt, F)) {
    rc = -1;
    goto out;
  }
  orc_split_F8(m, k, A, E, p, DA);
  orc_split_F8(n, k, Bt, F, p, DB);
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      i128 S = 0;
      for (int s = 0; s < p; ++s) {
        int64_t Cs = 0;
        for (int t = 0; t <= s; ++t) {
          const int16_t *a = DA + ((int64_t)t * m + i) * k;
          const int16_t *b = DB + ((int64_t)(s - t) * n + j) * k;
          for (int64_t h = 0; h < k; ++h) Cs += (int64_t)a[h] * (int64_t)b[h];
        }
        S += (i128)Cs << (5 * (p - 1 - s));
      }
      double r = ldexp(i128_to_double(S), E[i] + F[j] - 8 - 5 * (p - 1));
      if (out_f32)
        Cf[i * n + j] = (float)blas_update(alpha, r, beta, beta == 0.0 ? 0.0 : (double)Cf[i * n + j]);
      else
        C[i * n + j] = blas_update(alpha, r, beta, beta == 0.0 ? 0.0 : C[i * n + j]);
    }
out:
  free(E);
  free(F);
  free(DA);
  free(DB);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Scheme I complex, 4M (reading R8)                                   */
/* ------------------------------------------------------------------ */

/* T_s for one output: sum_{t<=s} <X_t, Y_{s-t}> over k, exact. */
static int64_t tri_sum(const int16_t *DX, int64_t rx, int64_t nx, const int16_t *DY, int64_t ry, int64_t ny,
                       int64_t k, int s) {
  int64_t acc = 0;
  for (int t = 0; t <= s; ++t) {
    const int16_t *a = DX + ((int64_t)t * nx + rx) * k;
    const int16_t *b = DY + ((int64_t)(s - t) * ny + ry) * k;
    for (int64_t h = 0; h < k; ++h) acc += (int64_t)a[h] * (int64_t)b[h];
  }
  return acc;
}

/* A: m x k complex, Bt: n x k complex (B^T, not conjugated), both
 * interleaved (re, im).  f8 selects the slices: 0 = INT8 bytes (R1), 1 =
 * E4M3 digits (R7).  C: m x n complex (interleaved) in/out; with out_f32 the
 * result goes to Cf (m x n complex float, interleaved), each component
 * rounded once more to binary32 (CGEMM).  Returns 0, or -1 on non-finite
 * input. */
int orc_emu_Z4M_I(int64_t m, int64_t n, int64_t k, int p, int f8, double alpha_re, double alpha_im,
                  const double *A, const double *Bt, double beta_re, double beta_im, double *C, float *Cf,
                  int out_f32) {
  const int beta_bits = f8 ? 5 : 8;
  const int escale = f8 ? -8 - 5 * (p - 1) : -14 - 8 * (p - 1);
  size_t mk = (size_t)(m * k > 0 ? m * k : 1), nk = (size_t)(n * k > 0 ? n * k : 1);
  int32_t *E = malloc(sizeof(int32_t) * (m > 0 ? m : 1));
  int32_t *F = malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  double *Ar = malloc(sizeof(double) * mk), *Ai = malloc(sizeof(double) * mk);
  double *Br = malloc(sizeof(double) * nk), *Bi = malloc(sizeof(double) * nk), *Bn = malloc(sizeof(double) * nk);
  int16_t *DAr = malloc(sizeof(int16_t) * p * mk), *DAi = malloc(sizeof(int16_t) * p * mk);
  int16_t *DBr = malloc(sizeof(int16_t) * p * nk), *DBi = malloc(sizeof(int16_t) * p * nk);
  int16_t *DBn = malloc(sizeof(int16_t) * p * nk);
  int rc = 0;
  if (orc_row_exponents_z(m, k, A, E) || orc_row_exponents_z(n, k, Bt, F)) {
    rc = -1;
    goto out;
  }
  for (int64_t q = 0; q < m * k; ++q) {
    Ar[q] = A[2 * q];
    Ai[q] = A[2 * q + 1];
  }
  for (int64_t q = 0; q < n * k; ++q) {
    Br[q] = Bt[2 * q];
    Bi[q] = Bt[2 * q + 1];
    Bn[q] = -Bt[2 * q + 1];
  }
  if (f8) {
    orc_split_F8(m, k, Ar, E, p, DAr);
    orc_split_F8(m, k, Ai, E, p, DAi);
    orc_split_F8(n, k, Br, F, p, DBr);
    orc_split_F8(n, k, Bi, F, p, DBi);
    orc_split_F8(n, k, Bn, F, p, DBn);
  } else {
    orc_split_I(m, k, Ar, E, p, DAr);
    orc_split_I(m, k, Ai, E, p, DAi);
    orc_split_I(n, k, Br, F, p, DBr);
    orc_split_I(n, k, Bi, F, p, DBi);
    orc_split_I(n, k, Bn, F, p, DBn);
  }
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) {
      i128 Sre = 0, Sim = 0;
      for (int s = 0; s < p; ++s) {
        const int64_t tre = tri_sum(DAr, i, m, DBr, j, n, k, s) + tri_sum(DAi, i, m, DBn, j, n, k, s);
        const int64_t tim = tri_sum(DAr, i, m, DBi, j, n, k, s) + tri_sum(DAi, i, m, DBr, j, n, k, s);
        Sre += (i128)tre << (beta_bits * (p - 1 - s));
        Sim += (i128)tim << (beta_bits * (p - 1 - s));
      }
      const double rr = ldexp(i128_to_double(Sre), E[i] + F[j] + escale);
      const double ri = ldexp(i128_to_double(Sim), E[i] + F[j] + escale);
      double cr = 0.0, ci = 0.0;
      if (beta_re != 0.0 || beta_im != 0.0) {
        cr = out_f32 ? (double)Cf[2 * (i * n + j)] : C[2 * (i * n + j)];
        ci = out_f32 ? (double)Cf[2 * (i * n + j) + 1] : C[2 * (i * n + j) + 1];
      }
      zupdate(alpha_re, alpha_im, rr, ri, beta_re, beta_im, &cr, &ci);
      if (out_f32) {
        Cf[2 * (i * n + j)] = (float)cr;
        Cf[2 * (i * n + j) + 1] = (float)ci;
      } else {
        C[2 * (i * n + j)] = cr;
        C[2 * (i * n + j) + 1] = ci;
      }
    }
out:
  free(E);
  free(F);
  free(Ar);
  free(Ai);
  free(Br);
  free(Bi);
  free(Bn);
  free(DAr);
  free(DAi);
  free(DBr);
  free(DBi);
  free(DBn);
  return rc;
}
