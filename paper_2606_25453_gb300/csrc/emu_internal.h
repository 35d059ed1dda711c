// emu_internal.h -- declarations shared by the library's translation units
// (host launchers, layout helpers, method tables passed to kernels).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "emu_device.cuh"

namespace emu {

constexpr int kMaxModuli = 20;  // Scheme II moduli supported
constexpr int kCrtLimbs = 5;     // P < 2^160 for up to 20 moduli
constexpr int kSplitRowAlign = 128;

// Layout of split outputs (see the C ABI header).
inline int64_t split_rows(int64_t rows) { return (rows + kSplitRowAlign - 1) / kSplitRowAlign * kSplitRowAlign; }
inline int64_t split_cols_I(int64_t k, int p) { return (k + 31) / 32 * 32 * p; }
inline int64_t split_cols_II(int64_t k) { return (k + 127) / 128 * 128; }

// Scheme II tables, passed by value to kernels.
// Residues of the scaled integers a' (|a'| < 2^80) are taken from their
// 16-bit digits: a' = sum_j d_j 2^(16 j), a' mod m = sum_j d_j (2^(16 j) mod m)
// mod m, the last reduction in single precision (the sum stays below 2^26).
constexpr int kResDigits = 5;
constexpr int kResDigitsF = 6;
struct ModTables {
  uint32_t mods[kMaxModuli];
  int32_t off[kMaxModuli];                 // m - 1 - floor((m - 1)/2): symmetric residues lie in [-off, m - 1 - off]
  float inv[kMaxModuli];                   // 1/m rounded to nearest
  float offinv[kMaxModuli];                // off/m rounded to nearest
  float offhinv[kMaxModuli];               // (off + 1/2)/m rounded to nearest
  int32_t pow16[kMaxModuli][kResDigits];   // symmetric residue of 2^(16 j) mod m
  // binary32 form for the bf16 planes: 14-bit digits (six cover 2^84)
  float pow14f[kMaxModuli][kResDigitsF];   // symmetric residue of 2^(14 j) mod m
  float mf[kMaxModuli], offf[kMaxModuli];  // m and off as binary32
};

// CRT tables of Eq. (8) for a given number of moduli.
struct CrtTables {
  uint32_t w[kMaxModuli][kCrtLimbs];  // (P/m_l) * q_l, little-endian 32-bit limbs
  uint32_t P[kCrtLimbs];
  uint32_t Phalf[kCrtLimbs];          // floor(P/2)
  double invP;                        // 1/P rounded (quotient estimate only)
  float wP[kMaxModuli];               // w_l / P rounded to binary32 (quotient estimate only)
  int nm;
};

// Host-side method constants (api.cu).
int host_moduli(int nm, int32_t* out);
int64_t host_chunk_len_I(int p);
int64_t host_chunk_len_F8(int p);
int host_scale_bits_II(int nm, int64_t k, int is_complex);
void host_mod_tables(int nm, ModTables* t);
void host_crt_tables(int nm, CrtTables* t);

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_scan(const T* X, int64_t ld, bool kcontig, int64_t rows, int64_t k, int cw,
                 unsigned long long* maxbits, int* status, cudaStream_t st);
template <typename T>
void launch_split_I(const T* X, int64_t ld, bool kcontig, int64_t rows, int64_t k, int p,
                    const unsigned long long* maxbits, int8_t* hat, int32_t* E, cudaStream_t st,
                    bool f8 = false);
template <typename T>
void launch_split_II(const T* X, int64_t ld, bool kcontig, int64_t rows, int64_t k, int nm, int b,
                     int cw, const ModTables& tabs, const unsigned long long* maxbits, int8_t* res,
                     int32_t* E, cudaStream_t st, const int32_t* Ein = nullptr, bool bf16 = false);
// Norm-based Scheme II scaling: E[r] with ||x_r||_2 < 2^E[r], computed
// exactly (maxbits from launch_scan; acc: 2 rows words of scratch).
template <typename T>
void launch_norm(const T* X, int64_t ld, bool kcontig, int64_t rows, int64_t k, int cw,
                 const unsigned long long* maxbits, unsigned long long* acc, int32_t* E, cudaStream_t st);
void host_norm_halves_II(int nm, int* hA, int* hB);

// Output modes of the Scheme I kernel.
enum GemmOut : int { OUT_F64 = 0, OUT_F32 = 1, OUT_PARTIALS = 2 };

struct GemmIArgs {
  const CUtensorMap* descA;  // host copies, passed to the kernel by value
  const CUtensorMap* descB;
  int M, N;
  int nk32;     // number of 32-wide K-chunks
  int kc32;     // fold interval in K-chunks (K_c / 32)
  const int32_t* EA;
  const int32_t* FB;
  double alpha, beta;
  void* C;
  int64_t ldc;
  int32_t* partials;
  int* status;
  int num_sms;
};
cudaError_t launch_gemm_I(int p, int out_mode, const GemmIArgs& a, cudaStream_t st, bool f8 = false);
// Scheme I on E4M3 slices with tcgen05 / TMEM (128 x 32 output tiles).
cudaError_t launch_gemm_f8tc(int p, int out_mode, const GemmIArgs& a, cudaStream_t st);

// Scheme II kernel modes.
enum GemmIIOut : int { II_F64 = 0, II_F32 = 1, II_RESIDUES = 2, II_Z3M = 3, II_C3M = 4 };

struct GemmIIArgs {
  const CUtensorMap* descA;
  const CUtensorMap* descB;
  int M, N;
  int nk32;
  int rowsA_pad, rowsB_pad;  // plane heights in the stacked residue matrices
  int nm;
  int escale;                 // -2b
  const int32_t* EA;
  const int32_t* FB;
  double alpha_re, alpha_im, beta_re, beta_im;
  void* C;
  int64_t ldc;
  uint8_t* residues;
  int* status;
  int num_sms;
  int cluster;       // tcgen05 kernel: CTAs per GEMM tile (2: a CTA pair, cta_group::2; 1: one CTA)
  uint8_t* scratch;  // tcgen05 kernel: the residue planes
};
cudaError_t launch_gemm_II(int out_mode, const GemmIIArgs& a, const ModTables& mt,
                           const CrtTables& ct, cudaStream_t st);
// Scheme II on bf16 residue planes with tcgen05 / TMEM (256 x 256 tiles on
// CTA pairs, or 128 x 256 on single CTAs; modulus-major), then the CRT
// kernel; modes II_F64, II_F32, II_Z3M, II_C3M.  GemmIIArgs::scratch: gemm_II_tc_residue_bytes(M, N, nm, complex,
// cluster) bytes of device memory for the residue planes.  part: 1 launches
// the residue GEMM, 2 the CRT kernel (after the residue GEMM on the same
// stream), 3 both.
cudaError_t launch_gemm_II_tc(int out_mode, const GemmIIArgs& a, const ModTables& mt,
                              const CrtTables& ct, cudaStream_t st, int part = 3);
int gemm_II_tc_tile_m();
int gemm_II_tc_tile_n();
size_t gemm_II_tc_residue_bytes(int64_t M, int64_t N, int nm, bool is_complex, int cluster);
int gemm_II_tc_cluster();

// Tensor map for a row-major byte matrix [rows][cols] read in boxes of
// box_bytes x box_rows: 32-byte boxes with 32-byte swizzling, or 128-byte
// boxes with 128-byte swizzling.
bool make_tmap_i8(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows,
                  uint32_t box_rows, uint32_t box_bytes = 32);

}  // namespace emu
