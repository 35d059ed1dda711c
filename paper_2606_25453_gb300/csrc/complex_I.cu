// complex_I.cu -- Scheme I complex GEMM (the 4M formulation the paper uses
// for its Scheme I CGEMM / ZGEMM, Sec. VI).
//
// The four real products are one real Scheme I product of the real embedding
//     Ae = [Re A, Im A]                        (M x 2K)
//     Be = column 2j: [Re B_j; -Im B_j], column 2j+1: [Im B_j; Re B_j]   (2K x 2N)
// whose output row i holds (Re C_ij, Im C_ij) interleaved, i.e. exactly the
// complex layout of C.  The row maximum of Ae is the complex row maximum of A
// and the column maxima of Be are the complex column maxima of B, so one
// power-of-two scale per complex row / column covers both parts, and the
// exact triangle sums of the real and imaginary parts are rounded once each
// (the exact shift-reduce of the real path).  The embedding costs one pass
// over A and B (about 3x their bytes written), small next to the 4MNK
// tensor-core products.  Column-major calls are NOT mapped onto the
// transposed product here: that would move the negated operand from Im B to
// Im A and change the truncated triangle.  The embedding reads either layout
// directly and the result reaches C through the combine kernel.
#include "emu_internal.h"
#include "emu_handle.h"

namespace emu {
namespace {

// Ae[r][h] = Re A(r, h), Ae[r][K + h] = Im A(r, h).  Element (r, h) of the
// complex source is at X[(r ld + h)] (kcontig) or X[(h ld + r)].  32 x 32
// tiles through shared memory so that both the reads and the writes are
// coalesced for either source layout.
template <typename T>
__global__ void embed_A_kernel(const T* __restrict__ X, int64_t ld, bool kcontig, int64_t rows, int64_t K,
                               double* __restrict__ Ae) {
  __shared__ double tre[32][33], tim[32][33];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32, h0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int q = ty; q < 32; q += 8) {
    // kcontig: lanes along h; strided: lanes along r
    const int64_t r = kcontig ? r0 + q : r0 + tx, h = kcontig ? h0 + tx : h0 + q;
    double re = 0.0, im = 0.0;
    if (r < rows && h < K) {
      const T* p = X + 2 * (kcontig ? r * ld + h : h * ld + r);
      re = static_cast<double>(p[0]);
      im = static_cast<double>(p[1]);
    }
    if (kcontig) {
      tre[q][tx] = re;
      tim[q][tx] = im;
    } else {
      tre[tx][q] = re;
      tim[tx][q] = im;
    }
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int64_t r = r0 + q, h = h0 + tx;
    if (r < rows && h < K) {
      Ae[r * 2 * K + h] = tre[q][tx];
      Ae[r * 2 * K + K + h] = tim[q][tx];
    }
  }
}

// Rows of Be^T (2N x 2K, K-contiguous): row 2j = [Re B_j, -Im B_j],
// row 2j+1 = [Im B_j, Re B_j], B_j the j-th column of B (element (h, j) at
// X[(j ld + h)] when kcontig, else X[(h ld + j)]).
template <typename T>
__global__ void embed_B_kernel(const T* __restrict__ X, int64_t ld, bool kcontig, int64_t cols, int64_t K,
                               double* __restrict__ Bt) {
  __shared__ double tre[32][33], tim[32][33];
  const int64_t j0 = static_cast<int64_t>(blockIdx.y) * 32, h0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    const int64_t j = kcontig ? j0 + q : j0 + tx, h = kcontig ? h0 + tx : h0 + q;
    double re = 0.0, im = 0.0;
    if (j < cols && h < K) {
      const T* p = X + 2 * (kcontig ? j * ld + h : h * ld + j);
      re = static_cast<double>(p[0]);
      im = static_cast<double>(p[1]);
    }
    if (kcontig) {
      tre[q][tx] = re;
      tim[q][tx] = im;
    } else {
      tre[tx][q] = re;
      tim[tx][q] = im;
    }
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int64_t j = j0 + q, h = h0 + tx;
    if (j < cols && h < K) {
      double* even = Bt + (2 * j) * 2 * K;
      double* odd = even + 2 * K;
      even[h] = tre[q][tx];
      even[K + h] = -tim[q][tx];
      odd[h] = tim[q][tx];
      odd[K + h] = tre[q][tx];
    }
  }
}

// C = alpha * R + beta * C for complex alpha, beta (the complex BLAS update:
// t = fma(a_re, r_re, -(a_im r_im)) + i fma(a_re, r_im, a_im r_re), the same
// form for beta * C when beta != 0, one addition per part; C is not read
// when beta == 0).  R: rows x cols complex, row pitch cols; C row-major
// (element (i, j) at 2 (i ldc + j)) or column-major (2 (j ldc + i)); T =
// double or float output (float: each part rounded once more).
template <typename T>
__global__ void zcombine_kernel(const double* __restrict__ R, int64_t rows, int64_t cols, double ar, double ai,
                                double br, double bi, T* __restrict__ C, int64_t ldc, bool colmajor) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t i = idx / cols, j = idx % cols;
  const double rr = R[2 * idx], ri = R[2 * idx + 1];
  double tr = __fma_rn(ar, rr, -__dmul_rn(ai, ri));
  double ti = __fma_rn(ar, ri, __dmul_rn(ai, rr));
  T* p = C + 2 * (colmajor ? j * ldc + i : i * ldc + j);
  if (br != 0.0 || bi != 0.0) {
    const double cr = static_cast<double>(p[0]), ci = static_cast<double>(p[1]);
    tr = __dadd_rn(tr, __fma_rn(br, cr, -__dmul_rn(bi, ci)));
    ti = __dadd_rn(ti, __fma_rn(br, ci, __dmul_rn(bi, cr)));
  }
  p[0] = static_cast<T>(tr);
  p[1] = static_cast<T>(ti);
}

size_t al256c(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t workspace_complex_I(int64_t M, int64_t N, int64_t K, int p) {
  const size_t emb = al256c(sizeof(double) * static_cast<size_t>(M) * 2 * K) +
                     al256c(sizeof(double) * static_cast<size_t>(2 * N) * 2 * K);
  const size_t tmp = al256c(sizeof(double) * static_cast<size_t>(M) * 2 * N);
  return emb + tmp + plan_I(M, 2 * N, 2 * K, p).bytes;
}

template <typename T>
emu_status_t run_complex_I(emu_handle_s* h, emu_layout_t layout, int64_t M, int64_t N, int64_t K, const T* A,
                           int64_t lda, const T* B, int64_t ldb, int p, bool f8, const double* alpha,
                           const double* beta, T* C, int64_t ldc, cudaStream_t st) {
  const bool colmajor = layout == EMU_COL_MAJOR;
  uint8_t* ws = nullptr;
  emu_status_t s = handle_workspace(h, workspace_complex_I(M, N, K, p), st, &ws);
  if (s != EMU_OK) return s;
  double* Ae = reinterpret_cast<double*>(ws);
  double* Bt = reinterpret_cast<double*>(ws + al256c(sizeof(double) * static_cast<size_t>(M) * 2 * K));
  double* R = reinterpret_cast<double*>(reinterpret_cast<uint8_t*>(Bt) +
                                        al256c(sizeof(double) * static_cast<size_t>(2 * N) * 2 * K));
  uint8_t* ws_I = reinterpret_cast<uint8_t*>(R) + al256c(sizeof(double) * static_cast<size_t>(M) * 2 * N);
  // row-major: rows of A and columns of B are read K-contiguous / strided;
  // column-major the other way round
  const dim3 blk(32, 8);
  trace_begin(h, PH_SPLIT, st);
  embed_A_kernel<T><<<dim3(static_cast<unsigned>((K + 31) / 32), static_cast<unsigned>((M + 31) / 32)), blk, 0,
                      st>>>(A, lda, !colmajor, M, K, Ae);
  embed_B_kernel<T><<<dim3(static_cast<unsigned>((K + 31) / 32), static_cast<unsigned>((N + 31) / 32)), blk, 0,
                      st>>>(B, ldb, colmajor, N, K, Bt);
  trace_end(h, PH_SPLIT, st, 2);
  if (cudaGetLastError() != cudaSuccess) return EMU_ERR_CUDA;
  View e{};
  e.M = M;
  e.N = 2 * N;
  e.A = Ae;
  e.ldA = 2 * K;
  e.a_kcontig = true;
  e.B = Bt;
  e.ldB = 2 * K;
  e.b_kcontig = true;
  const bool direct =
      !colmajor && alpha[0] == 1.0 && alpha[1] == 0.0 && beta[0] == 0.0 && beta[1] == 0.0;
  if (direct) {
    // (Re, Im) pairs land straight in C: a real M x 2N matrix of row pitch 2 ldc
    return run_scheme_I<double>(h, e, 2 * K, p, 1.0, 0.0, C, 2 * ldc, sizeof(T) == 8 ? OUT_F64 : OUT_F32,
                                nullptr, st, ws_I, f8);
  }
  s = run_scheme_I<double>(h, e, 2 * K, p, 1.0, 0.0, R, 2 * N, OUT_F64, nullptr, st, ws_I, f8);
  if (s != EMU_OK) return s;
  const int64_t tot = M * N;
  zcombine_kernel<T><<<static_cast<unsigned>((tot + 255) / 256), 256, 0, st>>>(
      R, M, N, alpha[0], alpha[1], beta[0], beta[1], C, ldc, colmajor);
  return cudaGetLastError() == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}
template emu_status_t run_complex_I<double>(emu_handle_s*, emu_layout_t, int64_t, int64_t, int64_t,
                                            const double*, int64_t, const double*, int64_t, int, bool,
                                            const double*, const double*, double*, int64_t, cudaStream_t);
template emu_status_t run_complex_I<float>(emu_handle_s*, emu_layout_t, int64_t, int64_t, int64_t, const float*,
                                           int64_t, const float*, int64_t, int, bool, const double*,
                                           const double*, float*, int64_t, cudaStream_t);

}  // namespace emu
