// emu_handle.h -- the library handle and host-side planning helpers shared
// by the C ABI translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/emugemm.h"

struct emu_handle_s {
  int device = 0;
  int num_sms = 0;
  int* status = nullptr;  // device status word (bit flags, see emu_device.cuh)
  void* ws = nullptr;     // workspace
  size_t ws_bytes = 0;
  bool ws_user = false;   // caller-owned workspace
  void* grouped = nullptr;   // grouped-GEMM plan cache (grouped.cu)
  void* selector = nullptr;  // selector state (select.cu)
  void* trace = nullptr;     // per-phase timing state (trace.cu), null when off
  void* hostio = nullptr;    // host-buffer entry point's staging and copy stream (host_api.cu)
};

namespace emu {

// Byte offsets of one call's workspace regions.
struct Plan {
  int64_t rows_a, rows_b, cols;
  size_t off_maxA, off_maxB, off_EA, off_FB, off_hatA, off_hatB, bytes;
  size_t off_accA = 0, off_accB = 0, off_nEA = 0, off_nEB = 0;  // Scheme II norm-based scaling
  size_t off_scratch = 0;                                        // Scheme II tcgen05 residue slots
};
Plan plan_I(int64_t m, int64_t n, int64_t k, int p);
Plan plan_II(int64_t m, int64_t n, int64_t k, int nm, int nsets, int es);
bool ii_engine_tc();

// Row-major view of a product (see normalize in api.cu).
struct View {
  int64_t M, N;
  const void* A;
  int64_t ldA;
  bool a_kcontig;
  const void* B;
  int64_t ldB;
  bool b_kcontig;
};
void normalize(emu_layout_t layout, int64_t m, int64_t n, const void* A, int64_t lda, const void* B,
               int64_t ldb, View* v);
bool check_lds(emu_layout_t layout, int64_t m, int64_t n, int64_t k, int64_t lda, int64_t ldb, int64_t ldc);

emu_status_t handle_workspace(emu_handle_s* h, size_t bytes, cudaStream_t st, uint8_t** out);

// Argument checks shared by the emulated GEMM entry points; sets the
// handle's device (api.cu).
emu_status_t gemm_common(emu_handle_t h, emu_layout_t layout, int64_t m, int64_t n, int64_t k, const void* A,
                         int64_t lda, const void* B, int64_t ldb, const void* C, int64_t ldc, emu_scheme_t scheme,
                         int p_or_nm);

// Scheme II on the row-major view (api.cu).  phase: 0 the whole product;
// 1 only B's scan and split; 2 the rest, with B's split from an earlier
// phase-1 call on the same workspace.  plan_rows: the rows of A the
// workspace is laid out for (at least v.M; 0 means v.M), the same in the
// phase-1 and phase-2 calls of one product.
template <typename T>
emu_status_t run_scheme_II(emu_handle_s* h, const View& v, int64_t k, int nm, int cw, double ar, double ai,
                           double br, double bi, void* C, int64_t ldc, int out_mode, uint8_t* residues,
                           cudaStream_t st, bool norm = false, int phase = 0, int64_t plan_rows = 0);

// The fused Scheme I GEMM on operands already split (api.cu).
emu_status_t scheme_I_gemm(emu_handle_s* h, const int8_t* hatA, int64_t rows_a, const int8_t* hatB, int64_t rows_b,
                           int64_t cols, int64_t M, int64_t N, int64_t k, int p, const int32_t* EA,
                           const int32_t* FB, double alpha, double beta, void* C, int64_t ldc, int out_mode,
                           int32_t* partials, cudaStream_t st, bool f8);

// C = beta * C for products with k == 0 (beta == 0 writes zeros, C is not read).
template <typename T>
void launch_scale_c(T* C, int64_t ldc, int64_t M, int64_t N, double beta, cudaStream_t st);

// Tracing phases and hooks (no-ops unless tracing is enabled).
enum TracePhase : int { PH_SCAN = 0, PH_SPLIT = 1, PH_GEMM = 2, PH_OTHER = 3 };
void trace_begin(emu_handle_s* h, int phase, cudaStream_t st);
void trace_end(emu_handle_s* h, int phase, cudaStream_t st, int kernels);
void trace_release(emu_handle_s* h);
void handle_release_extras(emu_handle_s* h);

template <typename T>
emu_status_t run_scheme_I(emu_handle_s* h, const View& v, int64_t k, int p, double alpha, double beta,
                          void* C, int64_t ldc, int out_mode, int32_t* partials, cudaStream_t st,
                          uint8_t* ws_override, bool f8 = false);

// Scheme I complex (4M) through the real embedding; T = double (ZGEMM) or
// float (CGEMM) for both the inputs and C.  alpha, beta: {re, im}.
size_t workspace_complex_I(int64_t M, int64_t N, int64_t K, int p);
template <typename T>
emu_status_t run_complex_I(emu_handle_s* h, emu_layout_t layout, int64_t M, int64_t N, int64_t K, const T* A,
                           int64_t lda, const T* B, int64_t ldb, int p, bool f8, const double* alpha,
                           const double* beta, T* C, int64_t ldc, cudaStream_t st);

}  // namespace emu
