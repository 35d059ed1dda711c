// gemm_f8tc.cu -- Scheme I on E4M3 slices with the 5th-generation tensor
// cores (tcgen05.mma kind::f8f6f4), accumulators in tensor memory.
//
// The paper's Blackwell design keeps the p accumulators of the triangular
// schedule (Eq. 2, Algorithm 1) in TMEM and issues one MMA per slice pair.
// Here the p accumulators of a 128 x 32 output tile sit side by side in TMEM
// (accumulator s at columns [32 s, 32 s + 32)), so for a fixed A slice i the
// whole row of the triangle is ONE wide MMA:
//     D[:, 32 i : 32 P] += A'_i x [B'_0 | B'_1 | ... | B'_{P-1-i}]
// (the B slices of a K-chunk are contiguous in shared memory, and B'_j lands
// in the columns of accumulator i + j).  A K-chunk therefore costs about P
// tensor-core instructions (N split at 256) instead of P(P+1)/2.
//
// Roles (320 threads): warps 0-7 drain TMEM into exact 128-bit sums and write
// C (warp w: tile rows 32 (w % 4) .. +31, one per lane, columns 16 (w / 4)
// .. +15); warp 8 lane 0 issues the TMA loads; warp 9 owns the TMEM
// allocation and lane 0 issues the MMAs.
//
// The A slices of a K-chunk travel as 128-byte rows (four slices per TMA box,
// 128-byte swizzle; the MMA of slice 4g+u starts 32 u bytes into the row), so
// one L2 request carries four slices instead of one.  Each CTA loads its own
// operands from this GPU's memory (no cluster sharing: pairs of CTAs that
// shared the A slices by multicast measured within 1.5 % of single CTAs at
// n = 8192, p = 12).  Slices are balanced
// base-32 digits stored as E4M3 bytes, so every product is exact and the FP32
// accumulators stay exact integers while |sum| <= 2^24: they are drained
// every K_c (the E4M3 chunk bound) and at the end of each tile.  All waits are
// bounded; a timeout sets the status word, raises an abort flag for the other
// roles, and the TMEM is still released.
#include <cstdlib>

#include "emu_internal.h"
#include "tc_core.cuh"

namespace emu {
namespace {

constexpr int kBM = 128, kBN = 32;
constexpr int kThreadsTC = 320;
constexpr int kEpiThreads = 256;
constexpr int kProducerWarp = 8, kMmaWarp = 9;
constexpr uint32_t kTmemCols = 512;

template <int P>
struct CfgTC {
  // A: slices in groups of four, each group one 128-byte-wide TMA box per row
  // (the four 32-byte slice blocks of a K-chunk are adjacent in the
  // interleaved layout), 128-byte swizzle: 128 rows x 128 B per group.
  // B: one 32-row x 32-byte box per slice, slices stacked along N.
  static constexpr int kGroups = (P + 3) / 4;
  static constexpr int kBlkAg = kBM * 128;  // one group of A slices
  static constexpr int kBlkB = kBN * 32;    // one slice of B
  static constexpr int kStageBytes = kGroups * kBlkAg + P * kBlkB;
  static constexpr int kRaw = 196608 / kStageBytes;
  static constexpr int kStages = kRaw < 2 ? 2 : (kRaw > 6 ? 6 : kRaw);
  // at least 116 KB so that a single CTA (holding all 512 TMEM columns) runs per SM
  static constexpr int kSmemUsed = kStages * kStageBytes + 1024 + 256;
  static constexpr int kSmem = kSmemUsed < 118784 ? 118784 : kSmemUsed;
  static_assert(P * kBN <= static_cast<int>(kTmemCols), "accumulators must fit in TMEM");
  static_assert(kStageBytes % 1024 == 0, "stages must keep the 1024-byte swizzle alignment");
};

struct KParamsTC {
  CUtensorMap tA;  // box: 128 B x 128 rows, 128-byte swizzle
  CUtensorMap tB;  // box: 32 B x 32 rows
  int M, N, nk32, kc32, tiles_m, tiles_n;
  const int32_t* EA;
  const int32_t* FB;
  int escale;
  double alpha, beta;
  void* C;
  int64_t ldc;
  int32_t* partials;  // non-null: write the p accumulators (exact int32) instead of C (k <= K_c)
  int* status;
};

// ---------------------------------------------------------------- PTX wrappers
// Shared-memory matrix descriptor of a K-major operand block [rows][32 B]
// with the 32-byte swizzle TMA wrote: 8-row atoms 256 B apart (SBO), version
// 1, layout type 6 (32-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_k32(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);         // start address
  d |= static_cast<uint64_t>(1u) << 16;                        // leading byte offset (unused)
  d |= static_cast<uint64_t>((256u >> 4) & 0x3FFFu) << 32;     // stride byte offset: 8 rows x 32 B
  d |= static_cast<uint64_t>(1u) << 46;                        // descriptor version
  d |= static_cast<uint64_t>(6u) << 61;                        // 32-byte swizzle
  return d;
}

// Instruction descriptor: E4M3 x E4M3 -> F32, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4)                                  // D format F32
         | (0u << 7) | (0u << 10)                   // A, B format E4M3
         | (static_cast<uint32_t>(N >> 3) << 17)    // N / 8
         | (static_cast<uint32_t>(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void umma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane, as integers (the
// accumulators hold exact integers of magnitude <= 2^24).
__device__ __forceinline__ void tmem_ld8_int(uint32_t taddr, int32_t* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __float2int_rn(__uint_as_float(r[i]));
}

// Fold digits S0 .. S1-1 of the P accumulators of 8 columns (base 2^5
// Horner scheme) in 64-bit integers -- at most six digits, so the partial
// stays below 2^50 -- and add the partial into S at its weight
// 2^(5 (P - S1)).
template <int P, int S0, int S1>
__device__ __forceinline__ void fold_range(uint32_t taddr, __int128* S) {
  long long acc[8];
#pragma unroll
  for (int s = S0; s < S1; ++s) {
    int32_t v[8];
    tmem_ld8_int(taddr + static_cast<uint32_t>(s * kBN), v);
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = (s == S0) ? static_cast<long long>(v[c]) : acc[c] * 32 + v[c];
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) S[c] += static_cast<__int128>(acc[c]) << (5 * (P - S1));
}

// Add the P accumulators of 16 columns, sum_s C_s 2^(5 (P - 1 - s)), to S.
template <int P>
__device__ __forceinline__ void drain16(uint32_t taddr, __int128* S) {
  constexpr int H = (P + 1) / 2;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    fold_range<P, 0, H>(taddr + 8u * h, S + 8 * h);
    if constexpr (H < P) fold_range<P, H, P>(taddr + 8u * h, S + 8 * h);
  }
}

__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int& tm, int& tn) {
  constexpr int G = 8;
  int per_group = G * tiles_n;
  int g = tile / per_group;
  int first = g * G;
  int gsz = tiles_m - first < G ? tiles_m - first : G;
  int in = tile - g * per_group;
  tm = first + in % gsz;
  tn = in / gsz;
}

template <int P, int OUT>
__global__ void __launch_bounds__(kThreadsTC, 1) gemm_f8tc_kernel(const __grid_constant__ KParamsTC kp) {
  using Cfg = CfgTC<P>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* empty = full + Cfg::kStages;
  uint64_t* acc_full = empty + Cfg::kStages;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cid = static_cast<int>(blockIdx.x);
  const int ncl = static_cast<int>(gridDim.x);
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiThreads);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {  // the whole warp allocates the tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // the CTA walks tiles of 128 rows x 32 columns
  const int ntiles = kp.tiles_m * kp.tiles_n;
  const int my_tiles = cid < ntiles ? (ntiles - 1 - cid) / ncl + 1 : 0;
  const int drains_per_tile = (kp.nk32 + kp.kc32 - 1) / kp.kc32;

  if (warp == kProducerWarp) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      tma_prefetch_desc(&kp.tA);
      tma_prefetch_desc(&kp.tB);
      const uint32_t total = static_cast<uint32_t>(my_tiles) * static_cast<uint32_t>(kp.nk32);
      bool ok = true;
      for (uint32_t j = 0; j < total; ++j) {
        const uint32_t stage = j % Cfg::kStages;
        // the stage is free once the MMAs that read it have completed
        if (j >= static_cast<uint32_t>(Cfg::kStages) &&
            !wait_or_abort(&empty[stage], ((j / Cfg::kStages) & 1u) ^ 1u, abort_flag, kp.status)) {
          ok = false;
          break;
        }
        const int tt = static_cast<int>(j / kp.nk32);
        const int tile = cid + tt * ncl;
        // every other wave of tiles walks K backwards, starting on the chunks
        // the previous wave read last (still in L2); the sums are exact, so
        // their order does not matter
        const int kk = (tt & 1) ? kp.nk32 - 1 - static_cast<int>(j % kp.nk32) : static_cast<int>(j % kp.nk32);
        int tm, tn;
        tile_coords(tile, kp.tiles_m, kp.tiles_n, tm, tn);
        mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
        uint8_t* sA = smem + stage * Cfg::kStageBytes;
        uint8_t* sB = sA + Cfg::kGroups * Cfg::kBlkAg;
        // A: slices 4g .. 4g+3 of the chunk in one 128-byte box (a group that
        // runs past slice P-1 reads the next chunk's slices, or the zero fill
        // past the last chunk; the MMAs never use them)
#pragma unroll
        for (int g = 0; g < Cfg::kGroups; ++g)
          tma_load_2d(sA + g * Cfg::kBlkAg, &kp.tA, &full[stage], (kk * P + 4 * g) * 32, tm * kBM);
#pragma unroll
        for (int t = 0; t < P; ++t)
          tma_load_2d(sB + t * Cfg::kBlkB, &kp.tB, &full[stage], (kk * P + t) * 32, tn * kBN);
      }
      (void)ok;
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t it = 0, drain = 0;
      const uint32_t total = static_cast<uint32_t>(my_tiles) * static_cast<uint32_t>(kp.nk32);
      // A barrier probe stalls this thread until shared memory answers,
      // which under full tensor-core load takes long enough to drain the MMA
      // queue if the queue holds only the short MMAs at the end of a chunk.
      // So the next chunk's barrier is probed early in the current chunk,
      // right after the wide MMAs of the first rows are queued, and the wait
      // at the next chunk is skipped when that probe already saw the data.
      constexpr int kProbeRow = P >= 4 ? 2 : 0;
      bool ready = false;
      bool stop = false;
      for (int t = 0; t < my_tiles && !stop; ++t) {
        for (int kk = 0; kk < kp.nk32; ++kk, ++it) {
          const bool chunk_first = (kk % kp.kc32) == 0;
          if (chunk_first && drain > 0) {  // the epilogue must have emptied the accumulators
            if (!wait_or_abort(acc_empty, (drain - 1) & 1u, abort_flag, kp.status)) {
              stop = true;
              break;
            }
            tc_fence_after();
          }
          const uint32_t stage = it % Cfg::kStages;
          if (!ready && !wait_or_abort(&full[stage], (it / Cfg::kStages) & 1u, abort_flag, kp.status)) {
            stop = true;
            break;
          }
          ready = false;
          tc_fence_after();
          const uint32_t sA = base + stage * Cfg::kStageBytes;
          const uint32_t sB = sA + Cfg::kGroups * Cfg::kBlkAg;
#pragma unroll
          for (int i = 0; i < P; ++i) {
            const uint64_t adesc = smem_desc_k128(sA + (i >> 2) * Cfg::kBlkAg + (i & 3) * 32);
            // columns [32 i, 32 P) += A'_i x [B'_0 .. B'_{P-1-i}], N split at 256
#pragma unroll
            for (int q = 0; q * 256 < (P - i) * kBN; ++q) {
              const int n = (P - i) * kBN - q * 256 < 256 ? (P - i) * kBN - q * 256 : 256;
              const uint64_t bdesc = smem_desc_k32(sB + q * 256 * 32);
              const uint32_t acc = (chunk_first && i == 0) ? 0u : 1u;
              umma_e4m3(tmem + static_cast<uint32_t>(i * kBN + q * 256), adesc, bdesc, idesc_e4m3(kBM, n), acc);
            }
            if (i == kProbeRow && it + 1 < total)
              ready = mbar_test_wait(&full[(it + 1) % Cfg::kStages], ((it + 1) / Cfg::kStages) & 1u);
          }
          // the stage is free once these MMAs finish
          umma_commit(&empty[stage]);
          if ((kk + 1) % kp.kc32 == 0 || kk + 1 == kp.nk32) {
            umma_commit(acc_full);  // accumulators ready for the epilogue
            ++drain;
          }
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- epilogue (warps 0-3)
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows) and columns
    // 16 (w / 4) .. +15 of every accumulator
    const int row_in_tile = (warp & 3) * 32 + lane;
    const int c0 = (warp >> 2) * 16;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + static_cast<uint32_t>(c0);
    uint32_t drain = 0;
    bool stop = false;
    for (int t = 0; t < my_tiles && !stop; ++t) {
      const int tile = cid + t * ncl;
      int tm, tn;
      tile_coords(tile, kp.tiles_m, kp.tiles_n, tm, tn);
      __int128 S[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) S[c] = 0;
      for (int d = 0; d < drains_per_tile; ++d, ++drain) {
        if (!wait_or_abort(acc_full, drain & 1u, abort_flag, kp.status)) {
          stop = true;
          break;
        }
        tc_fence_after();
        if (kp.partials) {
          // unfused output: accumulator s of this thread's 16 columns to
          // partials[s][row][col] (one drain per tile, since k <= K_c)
          const int prow = tm * kBM + row_in_tile;
#pragma unroll 1
          for (int s = 0; s < P; ++s) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              int32_t v[8];
              tmem_ld8_int(lane_base + static_cast<uint32_t>(s * kBN + 8 * hh), v);
              if (prow < kp.M) {
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                  const int col = tn * kBN + c0 + 8 * hh + c;
                  if (col < kp.N)
                    kp.partials[(static_cast<int64_t>(s) * kp.M + prow) * kp.N + col] = v[c];
                }
              }
            }
          }
        } else {
          drain16<P>(lane_base, S);
        }
        tc_fence_before();
        mbar_arrive(acc_empty);
      }
      if (stop) break;
      if (kp.partials) continue;
      const int row = tm * kBM + row_in_tile;
      if (row < kp.M) {
        const int erow = kp.EA[row] + kp.escale;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int col = tn * kBN + c0 + c;
          if (col >= kp.N) continue;
          double dv = i128_to_double_rn(S[c]);
          double r = scale2(dv, erow + kp.FB[col]);
          if (OUT == OUT_F64) {
            double* cp = static_cast<double*>(kp.C) + static_cast<int64_t>(row) * kp.ldc + col;
            *cp = blas_update(kp.alpha, r, kp.beta, kp.beta != 0.0 ? *cp : 0.0);
          } else {
            float* cp = static_cast<float*>(kp.C) + static_cast<int64_t>(row) * kp.ldc + col;
            *cp = static_cast<float>(
                blas_update(kp.alpha, r, kp.beta, kp.beta != 0.0 ? static_cast<double>(*cp) : 0.0));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

template <int P, int OUT>
cudaError_t launch_tc(const GemmIArgs& a, cudaStream_t st, bool partials) {
  using Cfg = CfgTC<P>;
  cudaError_t e =
      cudaFuncSetAttribute(gemm_f8tc_kernel<P, OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  if (e != cudaSuccess) return e;
  KParamsTC kp;
  kp.tA = *a.descA;
  kp.tB = *a.descB;
  kp.M = a.M;
  kp.N = a.N;
  kp.nk32 = a.nk32;
  kp.kc32 = a.kc32;
  kp.tiles_m = (a.M + kBM - 1) / kBM;
  kp.tiles_n = (a.N + kBN - 1) / kBN;
  kp.EA = a.EA;
  kp.FB = a.FB;
  kp.escale = -8 - 5 * (P - 1);
  kp.alpha = a.alpha;
  kp.beta = a.beta;
  kp.C = a.C;
  kp.ldc = a.ldc;
  kp.partials = partials ? a.partials : nullptr;
  kp.status = a.status;
  const int ntiles = kp.tiles_m * kp.tiles_n;
  if (ntiles == 0 || kp.nk32 == 0) return cudaSuccess;
  const int grid = ntiles < a.num_sms ? ntiles : a.num_sms;
  gemm_f8tc_kernel<P, OUT><<<grid, kThreadsTC, Cfg::kSmem, st>>>(kp);
  return cudaGetLastError();
}

}  // namespace

int gemm_f8tc_tile_m() { return kBM; }
int gemm_f8tc_tile_n() { return kBN; }

cudaError_t launch_gemm_f8tc(int p, int out_mode, const GemmIArgs& a, cudaStream_t st) {
#define EMU_TC(PP)                                                \
  case PP:                                                        \
    return out_mode == OUT_F32 ? launch_tc<PP, OUT_F32>(a, st, false)     \
                               : launch_tc<PP, OUT_F64>(a, st, out_mode == OUT_PARTIALS);
  switch (p) {
    EMU_TC(1) EMU_TC(2) EMU_TC(3) EMU_TC(4) EMU_TC(5) EMU_TC(6)
    EMU_TC(7) EMU_TC(8) EMU_TC(9) EMU_TC(10) EMU_TC(11) EMU_TC(12)
    default:
      return cudaErrorInvalidValue;
  }
#undef EMU_TC
}

}  // namespace emu
