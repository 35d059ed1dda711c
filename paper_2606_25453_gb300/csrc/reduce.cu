// reduce.cu -- the unfused Scheme I epilogue (Eq. 3) as its own kernel: the
// second half of the "naive" pipeline that writes the INT32 partials of
// Eq. (2) to HBM (emu_partials_I / emu_partials_F8) and reads them back.  The
// fused kernels do the same arithmetic in their epilogue without the round
// trip; this entry point exists to measure that difference.
#include "emu_internal.h"
#include "emu_handle.h"

namespace emu {
namespace {

// C_ij = blas_update(alpha, RN(S) 2^(E_i + F_j + escale), beta, C_ij) with
// S = sum_s Cs[s][i][j] 2^(bits (p - 1 - s)) formed exactly in 128 bits.
__global__ void shift_reduce_kernel(const int32_t* __restrict__ Cs, int64_t m, int64_t n, int p, int bits,
                                    int escale, const int32_t* __restrict__ EA, const int32_t* __restrict__ FB,
                                    double alpha, double beta, double* __restrict__ C, int64_t ldc) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= m * n) return;
  const int64_t i = idx / n, j = idx % n;
  __int128 S = 0;
  for (int s = 0; s < p; ++s) S = (S << bits) + static_cast<__int128>(Cs[s * m * n + idx]);
  const double r = scale2(i128_to_double_rn(S), EA[i] + FB[j] + escale);
  double* cp = C + i * ldc + j;
  *cp = blas_update(alpha, r, beta, beta != 0.0 ? *cp : 0.0);
}

}  // namespace
}  // namespace emu

extern "C" emu_status_t emu_shift_reduce_I(emu_handle_t h, int64_t m, int64_t n, int p, int f8,
                                           const int32_t* Cs, const int32_t* EA, const int32_t* FB,
                                           double alpha, double beta, double* C, int64_t ldc,
                                           emu_stream_t stream) {
  if (!h || m < 0 || n < 0 || (m * n > 0 && (!Cs || !EA || !FB || !C)) || ldc < (n > 1 ? n : 1))
    return EMU_ERR_INVALID_ARG;
  if (p < EMU_P_MIN || p > EMU_P_MAX) return EMU_ERR_UNSUPPORTED;
  if (m == 0 || n == 0) return EMU_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return EMU_ERR_CUDA;
  const int bits = f8 ? 5 : 8;
  const int escale = f8 ? -8 - 5 * (p - 1) : -14 - 8 * (p - 1);
  const int64_t tot = m * n;
  emu::shift_reduce_kernel<<<static_cast<unsigned>((tot + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      Cs, m, n, p, bits, escale, EA, FB, alpha, beta, C, ldc);
  return cudaGetLastError() == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}
