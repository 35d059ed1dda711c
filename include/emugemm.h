/*
 * emugemm.h -- C ABI of the GB300 (sm_103a) emulated-GEMM library.
 *
 * The library computes C = alpha * A * B + beta * C for FP64, FP32 and
 * complex128 matrices on the INT8 tensor cores, with the two Ozaki schemes
 * of the EmuGEMM paper (Lu, Maeder, Luisier, Ziogas):
 *
 *   Scheme I  (Sec. II-C-1, Eqs. 1-3; fused kernel of Algorithm 1, Sec. III)
 *     Each row of A and each column of B is scaled by a power of two to its
 *     maximum exponent and cut into p INT8 slices (signed leading slice,
 *     unsigned tails, beta = 8 bits each).  All p(p+1)/2 slice products with
 *     i + j < p are formed exactly in INT32 and combined by the shift-reduce
 *     of Eq. (3).  Here the shift-reduce is exact: the partial sums are
 *     combined as integers and rounded once to binary64.
 *
 *   Scheme II (Sec. II-C-2, Eqs. 4-8; fused kernel of Sec. IV-A)
 *     A and B are scaled to integers, reduced modulo N pairwise-coprime
 *     moduli m_l <= 256 (256, 255, 253, 251, ...), multiplied with one
 *     integer GEMM per modulus, reduced modulo m_l and reconstructed by the
 *     Chinese Remainder Theorem (Eq. 8).  Complex input uses the 3M method
 *     (Eq. 16).  On sm_103a the per-modulus GEMMs run by default on the bf16
 *     tensor cores (tcgen05): symmetric residues are exact bf16 values and
 *     FP32 sums of up to 960 of their products are exact integers, so each
 *     960-deep K segment is reduced modulo m_l as it leaves the accumulator.
 *     That engine uses two kernels, like the paper's Sec. IV design: the
 *     residue GEMM writes one residue byte per output and modulus (Eq. 7),
 *     and a second kernel forms the CRT sum, the inverse scaling and the
 *     BLAS update.  EMU_II_ENGINE=mma selects the INT8 mma.sync kernel
 *     instead, which keeps the residues on chip and does the CRT in the
 *     same kernel (same results, k <= EMU_K_MAX_II).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named A, B, C, X, or ending in _dev are DEVICE pointers on the
 *    handle's device.  They are owned by the caller; the library reads or
 *    writes them only inside the stream-ordered work it enqueues and never
 *    keeps them after the call returns.  Pointers ending in _host are host
 *    pointers, read or written before the call returns.
 *  - layout (EMU_ROW_MAJOR / EMU_COL_MAJOR) applies to A, B and C together.
 *    Row-major: element (i, j) of an r x c matrix X with leading dimension
 *    ldx is X[i * ldx + j], ldx >= c.  Column-major: X[i + j * ldx],
 *    ldx >= r.  A is m x k, B is k x n, C is m x n.
 *  - Complex matrices are arrays of interleaved (re, im) doubles
 *    (cuDoubleComplex layout); leading dimensions count complex elements.
 *    alpha and beta of emu_zgemm are host arrays {re, im}.
 *  - beta == 0 means C is not read (NaN in C is ignored).
 *  - All work is enqueued on `stream` (0 = legacy default stream) and the
 *    call returns without synchronising.  Errors visible on the host are
 *    returned at once and nothing is enqueued.  Errors found on the device
 *    (non-finite input, a bounded wait that timed out) are recorded in the
 *    handle's device status word; emu_get_status synchronises the stream
 *    and returns them.  When the status word reports an error the contents
 *    of C are unspecified.  No kernel traps.
 *  - A handle owns workspace and is not thread safe: calls that share a
 *    handle must be ordered (same stream, or synchronised by the caller).
 *  - m, n or k equal to 0 is valid: with k == 0 the product is zero and
 *    C = beta * C (alpha ignored); with m == 0 or n == 0 nothing is done.
 *  - Environment (read once per process; results do not depend on it):
 *    EMU_II_ENGINE=mma runs Scheme II on the INT8 mma.sync kernel instead of
 *    the bf16 tcgen05 one; EMU_F8_ENGINE=mma runs E4M3 slices on the warp
 *    level instead of tcgen05; EMU_II_CLUSTER=2 runs the bf16 Scheme II
 *    residue GEMM on CTA pairs (256 x 256 tiles, tcgen05.mma.cta_group::2)
 *    instead of single CTAs (128 x 256 tiles); EMU_FAULT=alloc makes every
 *    library-owned workspace allocation fail and EMU_FAULT=launch every
 *    fused GEMM launch of a product fail with EMU_ERR_CUDA (host-side fault
 *    injection; nothing is run on the device in its place).
 */
#ifndef EMUGEMM_H
#define EMUGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct emu_handle_s *emu_handle_t;
typedef void *emu_stream_t; /* a cudaStream_t */

typedef enum { EMU_ROW_MAJOR = 0, EMU_COL_MAJOR = 1 } emu_layout_t;

/* EMU_SCHEME_I_F8: Scheme I on the FP8 tensor cores -- the paper's
 * interleaved layout and fused triangular kernel with E4M3 slices (beta = 5,
 * balanced base-32 digits, all products exact, FP32 accumulation kept exact
 * by draining every K_c), the FP8 formulation Sec. VII names as future work.
 * p_or_nm is the number of E4M3 slices (5 bits each: p = 11 gives 54 bits). */
/* EMU_SCHEME_II_NORM: Scheme II with a data-dependent bound for the
 * exactness condition after Eq. 8 instead of the worst case: by
 * Cauchy-Schwarz, sum_h |a'_ih||b'_hj| <= ||a'_i||_2 ||b'_j||_2, so each row
 * of A (column of B) is scaled by the exponent of its 2-norm (computed
 * exactly, independent of summation order) and both operands get the same
 * floor((floor(log2 P) - 1)/2) bits; inputs whose rows are not flat keep up to
 * log2(k)/2 more bits per operand at the same number of moduli.  p_or_nm is
 * the number of moduli; real, 3M complex, FP64 and FP32. */
typedef enum { EMU_SCHEME_I = 1, EMU_SCHEME_II = 2, EMU_SCHEME_I_F8 = 3, EMU_SCHEME_II_NORM = 4 } emu_scheme_t;

typedef enum {
  EMU_OK = 0,
  EMU_ERR_INVALID_ARG = 1, /* bad pointer, size, leading dimension or enum */
  EMU_ERR_UNSUPPORTED = 2, /* p / N / k outside the supported range        */
  EMU_ERR_NONFINITE = 3,   /* an input held NaN or +-inf (device-detected) */
  EMU_ERR_CUDA = 4,        /* a CUDA runtime or driver call failed         */
  EMU_ERR_ALLOC = 5,       /* device memory could not be allocated         */
  EMU_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up           */
  EMU_ERR_TOL_NOT_MET = 7  /* auto precision: tolerance not met at p_max   */
} emu_status_t;

/* Supported ranges. */
#define EMU_P_MIN 1          /* Scheme I slices                         */
#define EMU_P_MAX 12
#define EMU_NM_MIN 1         /* Scheme II moduli                        */
#define EMU_NM_MAX 20
#define EMU_K_MAX_II 131071  /* Scheme II on the INT8 engine (EMU_II_ENGINE=mma): |products| <= 2^14, INT32 exact */

/* ------------------------------------------------------------------ */
/* Handle, status, workspace                                           */
/* ------------------------------------------------------------------ */

/* Create a handle bound to CUDA device `device` (made current inside every
 * call).  Allocates a small device status word.  Errors: EMU_ERR_CUDA,
 * EMU_ERR_ALLOC, EMU_ERR_INVALID_ARG (h == NULL). */
emu_status_t emu_create(emu_handle_t *h, int device);

/* Destroy a handle: synchronises its device, frees library-owned workspace,
 * cached graphs and the status word.  NULL is accepted. */
emu_status_t emu_destroy(emu_handle_t h);

/* Synchronise `stream`, read and clear the device status word.  Returns
 * EMU_OK, EMU_ERR_NONFINITE, EMU_ERR_TIMEOUT or EMU_ERR_CUDA. */
emu_status_t emu_get_status(emu_handle_t h, emu_stream_t stream);

/* Failure-path self-test: launches one block whose mbarrier wait can never
 * be satisfied (nothing arrives on it).  The wait is bounded exactly like the
 * waits of the GEMM kernels, here by limit_cycles (clamped to [1e3, 2e9]
 * clock cycles); when it gives up the kernel records EMU_ERR_TIMEOUT in the
 * status word and returns, leaving the context usable.  emu_get_status then
 * reports EMU_ERR_TIMEOUT.  (The library's own waits give up after ~1 s.)
 * Host-side fault injection: with the environment variable EMU_FAULT=alloc
 * every library-owned workspace allocation fails with EMU_ERR_ALLOC; with
 * EMU_FAULT=launch the fused GEMM launch of every emu_dgemm / emu_sgemm /
 * emu_zgemm / emu_cgemm call fails with EMU_ERR_CUDA ("unspecified launch
 * failure") after the scan and split were enqueued, and C is not written. */
emu_status_t emu_selftest_wait(emu_handle_t h, int64_t limit_cycles, emu_stream_t stream);

/* Human-readable name of a status code (static string). */
const char *emu_status_string(emu_status_t s);

/* The CUDA runtime's description of the error behind the calling thread's
 * most recent EMU_ERR_CUDA from a launch or a tensor-map encoding ("no
 * error" if there was none); a static string. */
const char *emu_last_cuda_error(void);

/* Bytes of device workspace one call needs (is_complex selects the complex
 * layouts: three residue sets per operand for the Scheme II 3M method, the
 * real embedding plus the slices of the 2K-deep product for Scheme I 4M). */
emu_status_t emu_workspace_size(emu_scheme_t scheme, int64_t m, int64_t n, int64_t k, int p_or_nm,
                                int is_complex, size_t *bytes_host);

/* Give the handle a caller-owned workspace (device pointer, 256-byte
 * aligned).  Calls that need more than `bytes` return EMU_ERR_ALLOC instead
 * of allocating.  Passing NULL returns to library-owned workspace, which is
 * grown with cudaMallocAsync on the call's stream when needed.
 * CUDA graphs: emu_dgemm, emu_sgemm, emu_zgemm, emu_cgemm and the step
 * entry points may be captured on their stream once the workspace is large
 * enough for the call (after an uncaptured call of the same shape, or with
 * a caller-owned workspace); a call that would have to grow the
 * library-owned workspace while its stream is capturing returns
 * EMU_ERR_ALLOC and enqueues nothing.  emu_dgemm_host, emu_dgemm_auto(_II)
 * and emu_get_status synchronise and cannot be captured. */
emu_status_t emu_set_workspace(emu_handle_t h, void *workspace_dev, size_t bytes);

/* Tracing: when enabled, every call records CUDA events on its stream around
 * each kernel phase (exponent scan, split, fused GEMM, other) and counts the
 * kernels it launches.  emu_trace_read synchronises the recorded events and
 * returns the accumulated device milliseconds per phase (ms_host[4]: scan,
 * split, gemm, other -- on the bf16 Scheme II engine "gemm" is the residue
 * GEMM and "other" the CRT kernel), the number of GEMM launches and of all kernel
 * launches since the last read, then clears the counters.  Not available
 * while a stream is being captured into a CUDA graph.  Independently of
 * this switch, the host-side launches of each phase sit in an NVTX range
 * named emu.scan, emu.split, emu.gemm or emu.other (for profilers). */
emu_status_t emu_trace_enable(emu_handle_t h, int enable);
emu_status_t emu_trace_read(emu_handle_t h, double *ms_host, int64_t *gemm_launches_host,
                            int64_t *kernel_launches_host);

/* ------------------------------------------------------------------ */
/* Emulated GEMM                                                       */
/* ------------------------------------------------------------------ */

/* FP64 C = alpha*A*B + beta*C.  scheme = EMU_SCHEME_I or EMU_SCHEME_I_F8
 * with p_or_nm = p in [EMU_P_MIN, EMU_P_MAX] slices, or EMU_SCHEME_II with
 * p_or_nm = N in [EMU_NM_MIN, EMU_NM_MAX] moduli (k <= EMU_K_MAX_II when the
 * environment selects the INT8 engine with EMU_II_ENGINE=mma; the default
 * bf16 tcgen05 engine reduces every 960-deep segment modulo m and takes any k).
 * Sec. II-C. */
emu_status_t emu_dgemm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                       double alpha, const double *A, int64_t lda, const double *B, int64_t ldb,
                       double beta, double *C, int64_t ldc, emu_scheme_t scheme, int p_or_nm,
                       emu_stream_t stream);

/* FP32 C = alpha*A*B + beta*C.  The inputs are widened to binary64 exactly,
 * the method runs as in emu_dgemm, and each result is rounded once more to
 * binary32 (the paper's SGEMM emulation, Sec. III-B, "FP32 or FP64 output"). */
emu_status_t emu_sgemm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                       float alpha, const float *A, int64_t lda, const float *B, int64_t ldb,
                       float beta, float *C, int64_t ldc, emu_scheme_t scheme, int p_or_nm,
                       emu_stream_t stream);

/* complex128 C = alpha*A*B + beta*C.  A, B, C are interleaved (re, im)
 * arrays; lda, ldb, ldc count complex elements; alpha_host and beta_host
 * are host arrays {re, im}.  One power-of-two scale per row of A / column of
 * B covers both parts.
 *  - EMU_SCHEME_II, p_or_nm = N moduli: the 3M method (Sec. IV-B, Eq. 16):
 *    per modulus T1 = Re*Re, T2 = Im*Im, T3 = Sum*Sum, Re(C') = T1 - T2,
 *    Im(C') = T3 - T1 - T2 (mod m_l), one CRT per part.
 *  - EMU_SCHEME_I / EMU_SCHEME_I_F8, p_or_nm = p slices: the 4M formulation
 *    (the paper's Scheme I CGEMM/ZGEMM, Sec. VI): the four real triangle
 *    sums of Eq. 2, the Im*Im term from the slices of -Im B, combined exactly
 *    before one rounding per part -- Scheme I on the real matrices [Re A, Im A]
 *    and [[Re B, Im B], [-Im B, Re B]].  Workspace: emu_workspace_size with
 *    is_complex = 1 (the embedding of A and B, 16 (M + 2N) K bytes, plus the
 *    slices of the 2K-deep real product).
 * beta == 0: C is not read.  Errors as emu_dgemm. */
emu_status_t emu_zgemm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                       const double *alpha_host, const double *A, int64_t lda, const double *B,
                       int64_t ldb, const double *beta_host, double *C, int64_t ldc,
                       emu_scheme_t scheme, int p_or_nm, emu_stream_t stream);

/* complex64 C = alpha*A*B + beta*C, as emu_zgemm: EMU_SCHEME_I /
 * EMU_SCHEME_I_F8 (4M, p_or_nm = p) or EMU_SCHEME_II (3M, p_or_nm = N
 * moduli).  Inputs widened to binary64 exactly, the complex update done in
 * binary64, each part rounded once more to binary32 (the paper's CGEMM
 * emulation, Sec. VI).  alpha_host, beta_host: {re, im}. */
emu_status_t emu_cgemm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                       const float *alpha_host, const float *A, int64_t lda, const float *B,
                       int64_t ldb, const float *beta_host, float *C, int64_t ldc,
                       emu_scheme_t scheme, int p_or_nm, emu_stream_t stream);

/* emu_dgemm on host-resident matrices: A_host, B_host, C_host are host
 * memory (pinned, for the copies to overlap the computation; pageable
 * memory works, but then each copy completes before the next step is
 * queued).  Scheme I (EMU_SCHEME_I, EMU_SCHEME_I_F8) scales per row of A and
 * per column of B (Sec. III-A), so the product is cut along the rows of C
 * (of the row-major view: columns of C for EMU_COL_MAJOR) into up to four
 * chunks of at least 1024 rows: B is copied to the device, scanned and
 * split once, then each chunk's rows of A (and of C when beta != 0) are
 * copied on a copy stream while the compute stream scans, splits and
 * multiplies the chunk before and the copy stream returns the finished rows
 * of C -- the result is bit-identical to emu_dgemm on device copies.
 * Scheme II (EMU_SCHEME_II, EMU_SCHEME_II_NORM) scales per row and column
 * as well and runs the same way on the default bf16 tcgen05 engine (B's
 * residues once, then each chunk of A through the residue GEMM and the
 * CRT); the INT8 Scheme II engine and k = 0 copy the operands whole around
 * emu_dgemm.  The handle owns the
 * device staging (8 (m k + k n + m n) bytes, grown on demand by cudaMalloc)
 * and the copy stream, so calls on one handle must not overlap.  The call
 * returns once C_host holds the result (it synchronises `stream`).
 * Arguments, layouts and return codes otherwise as emu_dgemm. */
emu_status_t emu_dgemm_host(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                            double alpha, const double *A_host, int64_t lda, const double *B_host,
                            int64_t ldb, double beta, double *C_host, int64_t ldc,
                            emu_scheme_t scheme, int p_or_nm, emu_stream_t stream);

/* Allocation-free Scheme I DGEMM.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory while they
 * run -- programs that reserve all device memory up front in their own pool,
 * latency-critical code that cannot afford the implicit synchronisation of
 * cudaMalloc / cudaFree, and plugins whose host forbids allocation.  It
 * computes exactly what emu_dgemm(..., EMU_SCHEME_I, p, stream) computes (the
 * same kernels, bit-identical results) without a handle, and calls no
 * cudaMalloc, cudaFree or other allocating routine: its scratch is a fixed
 * file-scope device array of EMU_NOALLOC_SCRATCH_BYTES that every GPU which
 * loads the library holds until the process exits.
 *  - Runs on the current CUDA device.  The first call in a CUDA context of
 *    a device looks up the array's device address (cudaGetSymbolAddress) and
 *    caches it with the context's unique ID; make that first call before any
 *    stream capture on that device.  A call in a different context (for
 *    example after cudaDeviceReset re-created the primary context) looks the
 *    address up again, so that call, too, belongs outside a capture.
 *  - Products whose workspace (emu_workspace_size for Scheme I) exceeds
 *    EMU_NOALLOC_SCRATCH_BYTES are rejected with EMU_ERR_UNSUPPORTED
 *    (e.g. m = n = k = 2048 fits for p <= 7).
 *  - All calls share the array and it keeps the last call's contents; each
 *    call clears what must start at zero.  Calls whose work overlaps on the
 *    GPU (unordered streams) race on the array and give wrong results.
 *  - status_dev (device int, optional): device-detected errors are OR-ed
 *    into it as bit flags (1 = non-finite input, 2 = a bounded wait timed
 *    out); the caller zeroes it and reads it after synchronising.  NULL
 *    discards them.
 *  - Arguments, layouts and return codes otherwise as emu_dgemm. */
#define EMU_NOALLOC_SCRATCH_BYTES (64ll << 20)
emu_status_t emu_dgemm_noalloc(emu_layout_t layout, int64_t m, int64_t n, int64_t k, double alpha,
                               const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                               double *C, int64_t ldc, int p, int *status_dev, emu_stream_t stream);

/* ------------------------------------------------------------------ */
/* Steps of the path, exported for verification and ablation           */
/* ------------------------------------------------------------------ */

/* Layout of the split outputs (Eq. 11, "interleaved" layout): an operand
 * with `rows` reduction vectors of length k becomes an int8 matrix of
 * emu_split_rows(rows) rows and emu_split_cols_I(k, p) columns, row-major,
 * K contiguous.  Row r, K-chunk c (32 wide), slice t occupies bytes
 * [(c*p + t)*32, (c*p + t)*32 + 32).  Slice 0 is two's-complement signed,
 * slices t >= 1 are unsigned bytes.  Rows >= `rows` and K >= k are zero.
 * emu_split_rows rounds up to a multiple of 128, emu_split_cols_I(k, p) is
 * p * (k rounded up to 32).  Scheme II uses planes: plane l (modulus m_l) is
 * a matrix of emu_split_rows(rows) x emu_split_cols_II(k) int8 symmetric
 * residues, emu_split_cols_II(k) = k rounded up to 128. */
int64_t emu_split_rows(int64_t rows);
int64_t emu_split_cols_I(int64_t k, int p);
int64_t emu_split_cols_II(int64_t k);

/* Scheme I split of one operand (Eq. 1 + Eq. 11).  operand = 0: the rows
 * of the m x k matrix X (the A operand); operand = 1: the columns of the
 * k x n matrix X (the B operand).  `rows` is m or n.  Writes the
 * interleaved slices to hat_dev (emu_split_rows(rows) * emu_split_cols_I(k,
 * p) bytes) and the exponents E (smallest E with max |x| < 2^E, 0 for a zero
 * vector) to exp_dev (int32[rows]).  Non-finite input sets the status word. */
emu_status_t emu_split_I(emu_handle_t h, emu_layout_t layout, int operand, int64_t rows, int64_t k,
                         const double *X, int64_t ldx, int p, int8_t *hat_dev, int32_t *exp_dev,
                         emu_stream_t stream);

/* As emu_split_I for EMU_SCHEME_I_F8: the same interleaved layout holding
 * E4M3 bytes of the balanced base-32 digits of x = trunc(x * 2^(5p-1-E)). */
emu_status_t emu_split_F8(emu_handle_t h, emu_layout_t layout, int operand, int64_t rows, int64_t k,
                          const double *X, int64_t ldx, int p, int8_t *hat_dev, int32_t *exp_dev,
                          emu_stream_t stream);

/* Scheme II split of one operand (Eq. 5): residues of trunc(x * 2^(b - E))
 * for the first nm moduli, b = emu_scale_bits_II(nm, k_total, 0).  Writes
 * nm planes to res_dev (nm * emu_split_rows(rows) * emu_split_cols_II(k)
 * bytes) and exponents to exp_dev.  k_total is the K of the product whose
 * scaling is wanted (normally k). */
emu_status_t emu_split_II(emu_handle_t h, emu_layout_t layout, int operand, int64_t rows, int64_t k,
                          int64_t k_total, const double *X, int64_t ldx, int nm, int8_t *res_dev,
                          int32_t *exp_dev, emu_stream_t stream);

/* Unfused ("naive") Scheme I: the exact INT32 partials C_s of Eq. (2),
 * s = 0..p-1, written to Cs_dev as p row-major m x n int32 matrices
 * (Cs_dev[(s*m + i)*n + j]).  Requires k <= emu_chunk_len_I(p) so that every
 * C_s fits in INT32; A, B and layout as in emu_dgemm.  This is the INT32
 * round trip that the fused kernel avoids (Eq. 9); it shares the fused
 * kernel's main loop. */
emu_status_t emu_partials_I(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                            const double *A, int64_t lda, const double *B, int64_t ldb, int p,
                            int32_t *Cs_dev, emu_stream_t stream);

/* As emu_partials_I for EMU_SCHEME_I_F8: the FP32 accumulators of the E4M3
 * triangle converted to int32 (exact), p row-major m x n matrices;
 * k <= emu_chunk_len_F8(p). */
emu_status_t emu_partials_F8(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                             const double *A, int64_t lda, const double *B, int64_t ldb, int p,
                             int32_t *Cs_dev, emu_stream_t stream);

/* Unfused ("naive") Scheme I epilogue, Eq. (3): reads the p partials written
 * by emu_partials_I (f8 = 0) or emu_partials_F8 (f8 = 1) and writes
 *   C_ij = alpha * RN(sum_s Cs[s][i][j] * 2^(b (p-1-s))) * 2^(E_i + F_j + e) + beta * C_ij
 * with b = 8, e = -14 - 8(p-1) (INT8) or b = 5, e = -8 - 5(p-1) (E4M3); S is
 * formed exactly and rounded once (nearest, ties to even), as in the fused
 * kernels.  EA_dev: m row exponents of A, FB_dev: n column exponents of B, as
 * returned by emu_split_I / emu_split_F8 (operand 0 and 1).  C_dev:
 * row-major m x n, ldc >= n; not read when beta == 0.  Together with
 * emu_partials_I this is the INT32 round trip the fused kernel avoids
 * (Eq. 9); results are bit-identical to emu_dgemm when k <= K_c.
 * EMU_ERR_INVALID_ARG for bad sizes or null pointers. */
emu_status_t emu_shift_reduce_I(emu_handle_t h, int64_t m, int64_t n, int p, int f8, const int32_t *Cs_dev,
                                const int32_t *EA_dev, const int32_t *FB_dev, double alpha, double beta,
                                double *C_dev, int64_t ldc, emu_stream_t stream);

/* Paper-design Scheme II output (Sec. IV-A): per-modulus INT8 residues
 * C'_l = (A'_l B'_l) mod m_l in [0, m_l), as nm row-major m x n uint8
 * matrices (R_dev[(l*m + i)*n + j]).  The CRT is left to the caller. */
emu_status_t emu_residues_II(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                             const double *A, int64_t lda, const double *B, int64_t ldb, int nm,
                             uint8_t *R_dev, emu_stream_t stream);

/* Method constants computed by the library's host code. */
int64_t emu_chunk_len_I(int p);              /* K_c: INT32-exact K range of Eq. (2) */
int64_t emu_chunk_len_F8(int p);             /* K_c: FP32-exact K range, E4M3 slices */
int emu_moduli(int nm, int32_t *mods_host); /* first nm moduli; returns count      */
int emu_scale_bits_II(int nm, int64_t k, int is_complex); /* Scheme II exponent b    */

/* ------------------------------------------------------------------ */
/* Grouped (batched) emulated DGEMM                                    */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t m, n, k;
  double alpha, beta;
  const double *A; /* device */
  int64_t lda;
  const double *B; /* device */
  int64_t ldb;
  double *C; /* device */
  int64_t ldc;
} emu_gemm_desc_t;

/* `count` independent Scheme I products with p slices (row-major, the
 * descriptors are host memory).  Each product falls into a shape bucket (p
 * and log2 classes of sqrt(m n) and of k) and runs in that bucket's tuned
 * configuration: output tiles of 64 x 32, 32 x 32 or 32 x 64 and the
 * triangle's slice pairs B-slice-major or A-slice-major (64 x 32,
 * B-slice-major where the handle holds no tuning).  The products are
 * ordered by GEMM work per operand element and cut into up to three stages
 * (at 15 % and 50 % of the batch's GEMM work; one stage below 8 products).
 * Per stage: one grouped exponent scan, one grouped split, then one
 * persistent grouped GEMM launch per configuration in use over its
 * (problem, tile) work list, balanced longest-first over the CTAs.  Each
 * stage's GEMM launches run on parallel branches of one CUDA graph beside
 * the next stages' scan and split; the graph is captured once and replayed
 * while the descriptors and tunings stay identical.  The paper has no
 * batched interface; the tile model follows Table I. */
emu_status_t emu_dgemm_grouped(emu_handle_t h, int count, const emu_gemm_desc_t *descs_host, int p,
                               emu_stream_t stream);

/* Same products, one emu_dgemm call per problem (the launch-loop baseline). */
emu_status_t emu_dgemm_grouped_loop(emu_handle_t h, int count, const emu_gemm_desc_t *descs_host,
                                    int p, emu_stream_t stream);

/* Autotune the configuration per shape bucket on this problem list (data
 * as given).  A configuration is a tile shape (64 x 32, 32 x 32 or 32 x 64
 * outputs per CTA) and a slice-pair order of the triangle of Eq. (2)
 * (B-slice-major or A-slice-major): indices 0-2 are the three shapes in
 * B-slice-major order, 3-5 the same shapes A-slice-major.  Tuned twice,
 * with the batch cut into three stages and as one stage, keeping the
 * faster outcome and its stage setting.  Each time: the whole batch is
 * timed (CUDA events, 5 graph replays) in each single configuration and in
 * the current choices, the fastest being the starting point; each bucket's
 * products are timed alone in every configuration, the fastest being the
 * bucket's candidate; the whole batch with all candidates replaces the
 * starting point if faster, else the candidates are tried one bucket at a
 * time on the whole batch (kept if the batch gets 0.5 % faster).  The
 * choices are stored in the handle and, if `path` is non-NULL, written to
 * that cache file ("p<p>_s<i>_k<j>": configuration index per bucket,
 * "p<p>_stages": 1 or 3).  *timed_host receives the number of (sub-)batch
 * configurations timed.  Synchronises `stream`; the C arrays are written. */
emu_status_t emu_tune_grouped(emu_handle_t h, int count, const emu_gemm_desc_t *descs_host, int p,
                              const char *path, int *timed_host, emu_stream_t stream);

/* Load a tuning cache written by emu_tune_grouped. */
emu_status_t emu_load_tuning(emu_handle_t h, const char *path);

/* ------------------------------------------------------------------ */
/* Learned slice-count selector                                        */
/* ------------------------------------------------------------------ */

/* MLP 66 -> 64 -> 64 -> 8 (ReLU, softmax over p = 3..10), FP32, 8968
 * parameters in the packed order W1[64][66], b1[64], W2[64][64], b2[64],
 * W3[8][64], b3[8].  The paper has no selector (it lacks automatic dynamic
 * precision, Sec. VII); this is the library's own. */
#define EMU_SEL_IN 66
#define EMU_SEL_HID 64
#define EMU_SEL_OUT 8
#define EMU_SEL_P0 3
#define EMU_SEL_NM0 6 /* Scheme II selector: classes N = 6, 8, .., 20 */
#define EMU_SEL_NPARAM 8968

/* Features of one product (device output float[66]): 32-bin histogram of
 * d = E_i - e(a_ij) (exponent deficit of each element of A against its row
 * maximum, e = frexp exponent) in bins of 3 exponents, bin = min(d/3, 31),
 * zeros in bin 31, normalised to sum 1; the same for the columns of B;
 * log2(k)/16 and -log10(tol)/16.  A, B device,
 * layout as emu_dgemm; at most `sample` rows of A and columns of B are read
 * (evenly spaced; 0 = all). */
emu_status_t emu_sel_features(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                              const double *A, int64_t lda, const double *B, int64_t ldb, double tol,
                              int64_t sample, float *feat_dev, emu_stream_t stream);

/* Forward pass for `batch` feature rows X_dev[batch][66] -> probabilities
 * P_dev[batch][8]; params_dev holds the packed parameters.  When act_dev is
 * non-NULL the hidden activations (batch x 128 floats) are saved for the
 * backward pass. */
emu_status_t emu_sel_forward(emu_handle_t h, int64_t batch, const float *params_dev,
                             const float *X_dev, float *P_dev, float *act_dev, emu_stream_t stream);

/* Backward pass of the mean cross-entropy loss against integer labels
 * y_dev[batch] in [0, 8): writes dL/dparams to grad_dev (8968 floats,
 * overwritten) and the loss to loss_dev (one float). */
emu_status_t emu_sel_backward(emu_handle_t h, int64_t batch, const float *params_dev,
                              const float *X_dev, const float *act_dev, const float *P_dev,
                              const int32_t *y_dev, float *grad_dev, float *loss_dev,
                              emu_stream_t stream);

/* One Adam step (step >= 1) over the 8968 parameters; m_dev and v_dev are
 * the moment buffers (zero-initialised by the caller). */
emu_status_t emu_sel_adam(emu_handle_t h, float *params_dev, const float *grad_dev, float *m_dev,
                          float *v_dev, int step, float lr, float beta1, float beta2, float eps,
                          emu_stream_t stream);

/* Install trained parameters (host array of 8968 floats) in the handle. */
emu_status_t emu_sel_load(emu_handle_t h, const float *params_host);

/* Install trained parameters of the Scheme II selector (same network,
 * classes N = EMU_SEL_NM0 + 2c moduli, c = 0..7, for EMU_SCHEME_II_NORM). */
emu_status_t emu_sel_load_II(emu_handle_t h, const float *params_host);

/* Double-double reference of sampled output entries (the selector's judge):
 * for the `count` (i, j) pairs in idx_dev (int32 pairs), ref_dev receives
 * (hi, lo) of sum_h a_ih b_hj computed with error-free transformations in
 * FP64, and absab_dev receives sum_h |a_ih||b_hj|. */
emu_status_t emu_probe_dd(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                          const double *A, int64_t lda, const double *B, int64_t ldb, int count,
                          const int32_t *idx_dev, double *ref_dev, double *absab_dev,
                          emu_stream_t stream);

/* Auto precision: C = alpha*A*B with the smallest p the selector predicts
 * for max_ij |C - AB|_ij / (|A||B|)_ij <= tol: the smallest class whose
 * cumulative predicted probability reaches 0.8, and EMU_P_MAX for the
 * open-ended top class "10 or more".  The result is checked on `probe`
 * sampled entries against emu_probe_dd; on a miss p is raised to
 * max(p + 1, the bound-based p), then to EMU_P_MAX, and the product is
 * recomputed.  Without loaded selector weights the bound-based p is used.
 * Synchronises `stream` (the probe decides the next step); *p_used receives
 * the p of the returned result.  There is no beta: C is overwritten.
 * Returns EMU_ERR_TOL_NOT_MET (C holds the EMU_P_MAX result) if even
 * EMU_P_MAX misses on the probed entries. */
emu_status_t emu_dgemm_auto(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                            double alpha, const double *A, int64_t lda, const double *B,
                            int64_t ldb, double *C, int64_t ldc, double tol, int probe,
                            int *p_used_host, emu_stream_t stream);

/* Auto precision with Scheme II (norm-based scaling, EMU_SCHEME_II_NORM):
 * as emu_dgemm_auto with N moduli in place of p -- class c means N = 6 + 2c,
 * the top class means EMU_NM_MAX; on a probe miss N is raised to
 * max(N + 2, the bound-based N), then to EMU_NM_MAX.  *nm_used_host receives
 * the N of the returned result; EMU_ERR_TOL_NOT_MET if EMU_NM_MAX misses. */
emu_status_t emu_dgemm_auto_II(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                               double alpha, const double *A, int64_t lda, const double *B,
                               int64_t ldb, double *C, int64_t ldc, double tol, int probe,
                               int *nm_used_host, emu_stream_t stream);

/* Bound-based number of moduli for EMU_SCHEME_II_NORM (host): the smallest
 * N in 6, 8, .., 20 with 2^(-h(N) + spread + ceil(log2(k)/2) + 3) <= tol,
 * h(N) the shared scale bits and spread as in emu_bound_p (20 if none
 * does).  A heuristic from the per-term truncation error, not a guarantee. */
emu_status_t emu_bound_nm(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                          const double *A, int64_t lda, const double *B, int64_t ldb, double tol,
                          int *nm_host, emu_stream_t stream);

/* Bound-based slice count for tolerance tol from the exponent statistics
 * (host): smallest p in [3, 10] whose worst-case truncation bound
 * 2^(-8p+3) * 2^(spread) * k meets tol, where spread is the upper edge of the
 * largest exponent-deficit bin seen in 64 sampled rows/columns (10 if none
 * does).  Written to *p_host. */
emu_status_t emu_bound_p(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k,
                         const double *A, int64_t lda, const double *B, int64_t ldb, double tol,
                         int *p_host, emu_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* EMUGEMM_H */
