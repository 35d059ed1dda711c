// host_api.cu -- emulated DGEMM on host-resident matrices, with the copies
// to and from the device overlapping the computation.
//
// Scheme I (INT8 or E4M3 slices) scales per row of A and per column of B
// (Sec. III-A), so the product can be cut along the rows of A without
// changing a single bit of the result: B (the K x N operand of the row-major
// view) is copied, scanned and split once; the rows of A then go in chunks,
// each chunk's copy to the device, exponent scan, split and fused GEMM
// running on the compute stream while a copy stream brings in the next
// chunks and takes the finished rows of C back.  Scheme II scales per row
// of A and per column of B as well, and runs the same way on the bf16
// tcgen05 engine (B split once, then each chunk of A through the residue
// GEMM and the CRT); k = 0, the INT8 Scheme II engine and products below
// 2048 rows copy the operands whole around emu_dgemm.
#include <algorithm>

#include "emu_handle.h"
#include "emu_internal.h"

namespace emu {
namespace {

constexpr int kMaxChunks = 4;

struct HostIO {
  void* dev = nullptr;  // staging of the row-major view: A (M x K), B (K x N), C (M x N), compact
  size_t dev_bytes = 0;
  cudaStream_t copy = nullptr;
  cudaEvent_t ev_start = nullptr, ev_b = nullptr, ev_done = nullptr;
  cudaEvent_t ev_a[kMaxChunks] = {}, ev_c[kMaxChunks] = {};
};

HostIO* hostio_of(emu_handle_s* h) {
  if (!h->hostio) h->hostio = new HostIO();
  return static_cast<HostIO*>(h->hostio);
}

void hostio_free_sync(HostIO* io) {
  if (io->copy) cudaStreamDestroy(io->copy);
  for (cudaEvent_t e : {io->ev_start, io->ev_b, io->ev_done})
    if (e) cudaEventDestroy(e);
  for (int c = 0; c < kMaxChunks; ++c) {
    if (io->ev_a[c]) cudaEventDestroy(io->ev_a[c]);
    if (io->ev_c[c]) cudaEventDestroy(io->ev_c[c]);
  }
  io->copy = nullptr;
  io->ev_start = io->ev_b = io->ev_done = nullptr;
  for (int c = 0; c < kMaxChunks; ++c) io->ev_a[c] = io->ev_c[c] = nullptr;
}

emu_status_t hostio_setup(HostIO* io, size_t bytes) {
  if (!io->copy) {  // all or nothing: a partial set is released again
    bool ok = cudaStreamCreateWithFlags(&io->copy, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&io->ev_start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&io->ev_b, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&io->ev_done, cudaEventDisableTiming) == cudaSuccess;
    for (int c = 0; ok && c < kMaxChunks; ++c)
      ok = cudaEventCreateWithFlags(&io->ev_a[c], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&io->ev_c[c], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      hostio_free_sync(io);
      return EMU_ERR_CUDA;
    }
  }
  if (bytes > io->dev_bytes) {
    // every earlier call waited for its copies and kernels before returning,
    // so nothing in flight still uses the old staging buffer
    if (io->dev) cudaFree(io->dev);
    io->dev = nullptr;
    io->dev_bytes = 0;
    if (cudaMalloc(&io->dev, bytes) != cudaSuccess) {
      cudaGetLastError();
      return EMU_ERR_ALLOC;
    }
    io->dev_bytes = bytes;
  }
  return EMU_OK;
}

// Rows [r0, r0 + rows) of a row-major matrix with `cols` doubles per row,
// between a buffer of pitch ld_src and one of pitch ld_dst (elements).
cudaError_t copy_rows(double* dst, int64_t ld_dst, const double* src, int64_t ld_src, int64_t r0, int64_t rows,
                      int64_t cols, cudaMemcpyKind kind, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  // compact rows on both sides: one linear copy (a little steadier than the
  // pitched form at n = 8192: 260.7 against 262.4 ms per end-to-end call)
  if (ld_dst == cols && ld_src == cols)
    return cudaMemcpyAsync(dst + r0 * ld_dst, src + r0 * ld_src, static_cast<size_t>(rows * cols) * sizeof(double),
                           kind, st);
  return cudaMemcpy2DAsync(dst + r0 * ld_dst, static_cast<size_t>(ld_dst) * sizeof(double), src + r0 * ld_src,
                           static_cast<size_t>(ld_src) * sizeof(double), static_cast<size_t>(cols) * sizeof(double),
                           static_cast<size_t>(rows), kind, st);
}

}  // namespace

void hostio_release(emu_handle_s* h) {
  auto* io = static_cast<HostIO*>(h->hostio);
  if (!io) return;
  if (io->dev) cudaFree(io->dev);
  hostio_free_sync(io);
  delete io;
  h->hostio = nullptr;
}

}  // namespace emu

using namespace emu;

namespace {

// The whole product on the staging buffers: view A (M x K), B (K x N) and C
// (M x N, rows of C in the caller's memory at pitch ldc).
emu_status_t host_gemm(emu_handle_s* h, HostIO* io, const View& v, int64_t k, double alpha, double beta,
                       double* C_host, int64_t ldc, emu_scheme_t scheme, int p, cudaStream_t st) {
  const int64_t M = v.M, N = v.N;
  double* dA = static_cast<double*>(io->dev);
  double* dB = dA + M * k;
  double* dC = dB + k * N;
  const auto* A_host = static_cast<const double*>(v.A);
  const auto* B_host = static_cast<const double*>(v.B);
  cudaStream_t cs = io->copy;
  // the copy stream starts after the caller's earlier work on `st`
  if (cudaEventRecord(io->ev_start, st) != cudaSuccess || cudaStreamWaitEvent(cs, io->ev_start, 0) != cudaSuccess)
    return EMU_ERR_CUDA;
  const bool sI = (scheme == EMU_SCHEME_I || scheme == EMU_SCHEME_I_F8) && k > 0;
  // Scheme II in chunks on the bf16 tcgen05 engine (the INT8 engine takes
  // the whole product)
  const bool sII = (scheme == EMU_SCHEME_II || scheme == EMU_SCHEME_II_NORM) && k > 0 && ii_engine_tc();
  const int nch = (sI || sII) ? static_cast<int>(std::min<int64_t>(kMaxChunks, std::max<int64_t>(1, M / 1024))) : 1;
  // chunk rows: a multiple of the split's row padding, so that each chunk's
  // slices start on a padded row of the whole split
  const int64_t R = split_rows((M + nch - 1) / nch);
  bool ok = copy_rows(dB, N, B_host, v.ldB, 0, k, N, cudaMemcpyHostToDevice, cs) == cudaSuccess &&
            cudaEventRecord(io->ev_b, cs) == cudaSuccess;
  for (int c = 0; ok && c < nch; ++c) {
    const int64_t r0 = c * R, rows = std::min(R, M - r0);
    ok = copy_rows(dA, k, A_host, v.ldA, r0, rows, k, cudaMemcpyHostToDevice, cs) == cudaSuccess &&
         (beta == 0.0 || copy_rows(dC, N, C_host, ldc, r0, rows, N, cudaMemcpyHostToDevice, cs) == cudaSuccess) &&
         cudaEventRecord(io->ev_a[c], cs) == cudaSuccess;
  }
  if (!ok) return EMU_ERR_CUDA;
  emu_status_t s = EMU_OK;
  if (sII) {
    // B's scan and split once (phase 1), then each chunk of A through the
    // rest of the product (phase 2) on a workspace laid out for R rows
    const bool norm = scheme == EMU_SCHEME_II_NORM;
    View vb{R, N, dA, std::max<int64_t>(k, 1), true, dB, N, false};
    if (cudaStreamWaitEvent(st, io->ev_b, 0) != cudaSuccess) return EMU_ERR_CUDA;
    s = run_scheme_II<double>(h, vb, k, p, 1, alpha, 0.0, beta, 0.0, dC, N, II_F64, nullptr, st, norm, 1, R);
    if (s != EMU_OK) return s;
    for (int c = 0; c < nch; ++c) {
      const int64_t r0 = c * R, rows = std::min(R, M - r0);
      View vc{rows, N, dA + r0 * k, k, true, dB, N, false};
      if (cudaStreamWaitEvent(st, io->ev_a[c], 0) != cudaSuccess) return EMU_ERR_CUDA;
      s = run_scheme_II<double>(h, vc, k, p, 1, alpha, 0.0, beta, 0.0, dC + r0 * N, N, II_F64, nullptr, st, norm, 2,
                                R);
      if (s != EMU_OK) return s;
      if (cudaEventRecord(io->ev_c[c], st) != cudaSuccess || cudaStreamWaitEvent(cs, io->ev_c[c], 0) != cudaSuccess ||
          copy_rows(C_host, ldc, dC, N, r0, rows, N, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
        return EMU_ERR_CUDA;
    }
  } else if (!sI) {
    // whole operands around emu_dgemm on the row-major view
    if (cudaStreamWaitEvent(st, io->ev_a[0], 0) != cudaSuccess) return EMU_ERR_CUDA;
    s = emu_dgemm(h, EMU_ROW_MAJOR, M, N, k, alpha, dA, std::max<int64_t>(k, 1), dB, N, beta, dC, N, scheme, p, st);
    if (s != EMU_OK) return s;
    if (cudaEventRecord(io->ev_c[0], st) != cudaSuccess || cudaStreamWaitEvent(cs, io->ev_c[0], 0) != cudaSuccess ||
        copy_rows(C_host, ldc, dC, N, 0, M, N, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
      return EMU_ERR_CUDA;
  } else {
    const bool f8 = scheme == EMU_SCHEME_I_F8;
    Plan pl = plan_I(M, N, k, p);
    uint8_t* ws = nullptr;
    s = handle_workspace(h, pl.bytes, st, &ws);
    if (s != EMU_OK) return s;
    auto* maxA = reinterpret_cast<unsigned long long*>(ws + pl.off_maxA);
    auto* maxB = reinterpret_cast<unsigned long long*>(ws + pl.off_maxB);
    auto* EA = reinterpret_cast<int32_t*>(ws + pl.off_EA);
    auto* FB = reinterpret_cast<int32_t*>(ws + pl.off_FB);
    auto* hatA = reinterpret_cast<int8_t*>(ws + pl.off_hatA);
    auto* hatB = reinterpret_cast<int8_t*>(ws + pl.off_hatB);
    if (cudaStreamWaitEvent(st, io->ev_b, 0) != cudaSuccess) return EMU_ERR_CUDA;
    launch_scan<double>(dB, N, false, N, k, 1, maxB, h->status, st);
    launch_split_I<double>(dB, N, false, N, k, p, maxB, hatB, FB, st, f8);
    for (int c = 0; c < nch; ++c) {
      const int64_t r0 = c * R, rows = std::min(R, M - r0);
      if (cudaStreamWaitEvent(st, io->ev_a[c], 0) != cudaSuccess) return EMU_ERR_CUDA;
      launch_scan<double>(dA + r0 * k, k, true, rows, k, 1, maxA + r0, h->status, st);
      launch_split_I<double>(dA + r0 * k, k, true, rows, k, p, maxA + r0, hatA + r0 * pl.cols, EA + r0, st, f8);
      s = scheme_I_gemm(h, hatA + r0 * pl.cols, split_rows(rows), hatB, pl.rows_b, pl.cols, rows, N, k, p, EA + r0,
                        FB, alpha, beta, dC + r0 * N, N, OUT_F64, nullptr, st, f8);
      if (s != EMU_OK) return s;
      if (cudaEventRecord(io->ev_c[c], st) != cudaSuccess || cudaStreamWaitEvent(cs, io->ev_c[c], 0) != cudaSuccess ||
          copy_rows(C_host, ldc, dC, N, r0, rows, N, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
        return EMU_ERR_CUDA;
    }
  }
  if (cudaEventRecord(io->ev_done, cs) != cudaSuccess || cudaStreamWaitEvent(st, io->ev_done, 0) != cudaSuccess)
    return EMU_ERR_CUDA;
  return EMU_OK;
}

}  // namespace

extern "C" {

emu_status_t emu_dgemm_host(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, double alpha,
                            const double* A_host, int64_t lda, const double* B_host, int64_t ldb, double beta,
                            double* C_host, int64_t ldc, emu_scheme_t scheme, int p_or_nm, emu_stream_t stream) {
  emu_status_t s = gemm_common(h, layout, m, n, k, A_host, lda, B_host, ldb, C_host, ldc, scheme, p_or_nm);
  if (s != EMU_OK) return s;
  View v;
  normalize(layout, m, n, A_host, lda, B_host, ldb, &v);
  if (v.M == 0 || v.N == 0) return EMU_OK;
  HostIO* io = hostio_of(h);
  s = hostio_setup(io, sizeof(double) * static_cast<size_t>(v.M * k + k * v.N + v.M * v.N));
  if (s != EMU_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = host_gemm(h, io, v, k, alpha, beta, C_host, ldc, scheme, p_or_nm, st);
  // C is in the caller's memory when the call returns; on an error nothing
  // may still be copying from or into the caller's buffers either
  const cudaError_t e1 = cudaStreamSynchronize(io->copy);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (s != EMU_OK) return s;
  return e1 == cudaSuccess && e2 == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
}

}  // extern "C"
