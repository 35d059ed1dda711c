// gemm_I.cu -- fused Scheme I kernel (Algorithm 1, Sec. III-B).
//
// One persistent CTA per SM walks the output tiles.  A producer streams the
// interleaved slices (Eq. 11) of A-hat and B-hat into a multi-stage
// shared-memory ring with TMA (one 32-byte-wide box per slice, 32-byte
// swizzle, completion on an mbarrier).  Eight math warps each own a
// 16 x 16 output patch and, per 32-wide K-chunk, load all p A-slice
// fragments with ldmatrix, then stream the B slices and issue the triangular
// schedule of Eq. (2): acc[i+j] += A'_i B'_j for i + j < p, p(p+1) INT8
// mma.sync per chunk (signed leading / unsigned tail variants).  The p INT32
// accumulators live in registers (the GB300 INT8 path is the warp-level
// mma.sync, so this is the paper's register-resident regime).
//
// Every K_c elements (the INT32-exact range of Eq. 2) the accumulators are
// drained into an exact 128-bit integer S = sum_s C_s 256^(p-1-s).  The
// epilogue rounds S once to binary64 (shift-reduce of Eq. 3 without any
// rounding beyond the final one), applies 2^(E_i + F_j - 14 - 8(p-1)) and
// the BLAS update, and stores C.  No partial product reaches global memory
// (OUT_PARTIALS, the unfused ablation, writes the INT32 C_s instead).
//
// The same kernel runs the E4M3 engine (F8): slices are balanced base-32
// digits in E4M3 bytes, the MMA is the FP8 mma.sync with FP32 accumulators
// (exact below 2^24, drained every K_c of that engine), beta = 5.
#include "emu_internal.h"
#include "gemm_I_core.cuh"

namespace emu {

namespace {

constexpr int kBM = 64, kBN = 32;
constexpr int kCW = 8;  // math warps (4 along M x 2 along N)
// INT8 engine: a ninth, dedicated producer warp issues the TMA loads (the
// INT8 kernels fit in 168 registers, the limit with 3 warps on one SM
// sub-partition).  E4M3 engine: no ninth warp -- thread 0 issues the loads
// kStages - 1 iterations ahead -- so each thread may use 255 registers.
template <bool F8>
constexpr int threads_of() { return F8 ? kCW * 32 : (kCW + 1) * 32; }
constexpr int kBlkA = kBM * 32, kBlkB = kBN * 32;

template <int P>
struct CfgI {
  static constexpr int kStageBytes = P * (kBlkA + kBlkB);
  static constexpr int kRaw = 163840 / kStageBytes;
  static constexpr int kStages = kRaw < 2 ? 2 : (kRaw > 8 ? 8 : kRaw);
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 2 * kStages * 8 + 64;
};

struct KParamsI {
  CUtensorMap tA;
  CUtensorMap tB;
  int M, N, nk32, kc32, tiles_m, tiles_n;
  const int32_t* EA;
  const int32_t* FB;
  int escale;
  double alpha, beta;
  void* C;
  int64_t ldc;
  int32_t* partials;
  int* status;
};

__device__ __forceinline__ void tile_coords(int tile, int tiles_m, int tiles_n, int& tm, int& tn) {
  constexpr int G = 8;  // group of tile rows for L2 reuse
  int per_group = G * tiles_n;
  int g = tile / per_group;
  int first = g * G;
  int gsz = tiles_m - first < G ? tiles_m - first : G;
  int in = tile - g * per_group;
  tm = first + in % gsz;
  tn = in / gsz;
}

// Issue the TMA loads of pipeline iteration j (tile of this CTA, K-chunk).
template <int P>
__device__ __forceinline__ void issue_loads(const KParamsI& kp, uint8_t* smem, uint64_t* full, uint32_t j) {
  using Cfg = CfgI<P>;
  const uint32_t stage = j % Cfg::kStages;
  const int t = static_cast<int>(j / kp.nk32);
  const int tile = blockIdx.x + t * gridDim.x;
  // every other wave of tiles walks K backwards: it starts on the chunks the
  // previous wave read last, which are still in L2 (the sums are exact, so
  // their order does not matter)
  const int kk = (t & 1) ? kp.nk32 - 1 - static_cast<int>(j % kp.nk32) : static_cast<int>(j % kp.nk32);
  int tm, tn;
  tile_coords(tile, kp.tiles_m, kp.tiles_n, tm, tn);
  mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
  uint8_t* sA = smem + stage * Cfg::kStageBytes;
  uint8_t* sB = sA + P * kBlkA;
#pragma unroll
  for (int t = 0; t < P; ++t) tma_load_2d(sA + t * kBlkA, &kp.tA, &full[stage], (kk * P + t) * 32, tm * kBM);
#pragma unroll
  for (int t = 0; t < P; ++t) tma_load_2d(sB + t * kBlkB, &kp.tB, &full[stage], (kk * P + t) * 32, tn * kBN);
}

template <int P, int OUT, bool F8>
__global__ void __launch_bounds__(threads_of<F8>(), 1) gemm_I_kernel(const __grid_constant__ KParamsI kp) {
  using Cfg = CfgI<P>;
  using Acc = typename Engine<F8>::Acc;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* empty = full + Cfg::kStages;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kCW);
    }
    fence_mbar_init();
  }
  __syncthreads();

  const int ntiles = kp.tiles_m * kp.tiles_n;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - static_cast<int>(blockIdx.x)) / gridDim.x + 1 : 0;
  const uint32_t total = static_cast<uint32_t>(my_tiles) * static_cast<uint32_t>(kp.nk32);
  if constexpr (!F8) {
    if (warp == kCW) {  // dedicated producer warp
      if (lane == 0) {
        tma_prefetch_desc(&kp.tA);
        tma_prefetch_desc(&kp.tB);
        for (uint32_t j = 0; j < total; ++j) {
          if (j >= static_cast<uint32_t>(Cfg::kStages) &&
              !mbar_wait_bounded(&empty[j % Cfg::kStages], ((j / Cfg::kStages) & 1u) ^ 1u)) {
            set_status(kp.status, ST_TIMEOUT);
            return;
          }
          issue_loads<P>(kp, smem, full, j);
        }
      }
      return;
    }
  }
  const bool producer = F8 && threadIdx.x == 0;  // inline producer of the E4M3 engine
  if (producer) {
    tma_prefetch_desc(&kp.tA);
    tma_prefetch_desc(&kp.tB);
    for (uint32_t j = 0; j < total && j + 1 < static_cast<uint32_t>(Cfg::kStages); ++j) issue_loads<P>(kp, smem, full, j);
  }

  const int wm = warp >> 1, wn = warp & 1;
  const uint32_t a_off = swz32(wm * 16 + (lane & 15), lane >> 4);
  const uint32_t b_off = swz32(wn * 16 + (lane & 7) + ((lane >> 4) << 3), (lane >> 3) & 1);
  uint32_t it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int tm, tn;
    tile_coords(tile, kp.tiles_m, kp.tiles_n, tm, tn);
    Acc acc[P][2][4];
    __int128 S[2][4];
#pragma unroll
    for (int s = 0; s < P; ++s)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[s][nt][q] = 0;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) S[nt][q] = 0;

    int since_fold = 0;
    for (int kk = 0; kk < kp.nk32; ++kk, ++it) {
      // keep the ring kStages - 1 iterations ahead: reuse a slot once every warp released it
      if (producer) {
        const uint32_t j = it + Cfg::kStages - 1;
        if (j < total) {
          if (j >= static_cast<uint32_t>(Cfg::kStages) &&
              !mbar_wait_bounded(&empty[j % Cfg::kStages], ((j / Cfg::kStages) & 1u) ^ 1u)) {
            set_status(kp.status, ST_TIMEOUT);
            return;
          }
          issue_loads<P>(kp, smem, full, j);
        }
      }
      const uint32_t stage = it % Cfg::kStages;
      const uint32_t par = (it / Cfg::kStages) & 1u;
      if (!mbar_wait_bounded(&full[stage], par)) {
        set_status(kp.status, ST_TIMEOUT);
        return;
      }
      const uint32_t sA = base + stage * Cfg::kStageBytes;
      const uint32_t sB = sA + P * kBlkA;
      uint32_t af[P][4];
#pragma unroll
      for (int i = 0; i < P; ++i) ldsm_x4(sA + i * kBlkA + a_off, af[i][0], af[i][1], af[i][2], af[i][3]);
      TriAll<P, kBlkB, F8>::run(acc, af, sB, b_off);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[stage]);
      if (OUT != OUT_PARTIALS && ++since_fold == kp.kc32) {
        fold<P, F8>(acc, S);
        since_fold = 0;
      }
    }

    const int row0 = tm * kBM + wm * 16 + (lane >> 2);
    const int col0 = tn * kBN + wn * 16 + (lane & 3) * 2;
    if (OUT == OUT_PARTIALS) {
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int row = row0 + (q >> 1) * 8, col = col0 + nt * 8 + (q & 1);
          if (row < kp.M && col < kp.N) {
#pragma unroll
            for (int s = 0; s < P; ++s)
              kp.partials[(static_cast<int64_t>(s) * kp.M + row) * kp.N + col] =
                  static_cast<int32_t>(Engine<F8>::to_int(acc[s][nt][q]));
          }
        }
      continue;
    }
    fold<P, F8>(acc, S);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int row = row0 + (q >> 1) * 8, col = col0 + nt * 8 + (q & 1);
        if (row < kp.M && col < kp.N) {
          double d = i128_to_double_rn(S[nt][q]);
          double r = scale2(d, kp.EA[row] + kp.FB[col] + kp.escale);
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

template <int P, int OUT, bool F8>
cudaError_t launch_p(const GemmIArgs& a, cudaStream_t st) {
  using Cfg = CfgI<P>;
  cudaError_t e = cudaFuncSetAttribute(gemm_I_kernel<P, OUT, F8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem);
  if (e != cudaSuccess) return e;
  KParamsI kp;
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
  kp.escale = F8 ? -8 - 5 * (P - 1) : -14 - 8 * (P - 1);
  kp.alpha = a.alpha;
  kp.beta = a.beta;
  kp.C = a.C;
  kp.ldc = a.ldc;
  kp.partials = a.partials;
  kp.status = a.status;
  int ntiles = kp.tiles_m * kp.tiles_n;
  if (ntiles == 0) return cudaSuccess;
  int grid = ntiles < a.num_sms ? ntiles : a.num_sms;
  gemm_I_kernel<P, OUT, F8><<<grid, threads_of<F8>(), Cfg::kSmem, st>>>(kp);
  return cudaGetLastError();
}

}  // namespace

int gemm_I_tile_m() { return kBM; }
int gemm_I_tile_n() { return kBN; }

cudaError_t launch_gemm_I(int p, int out_mode, const GemmIArgs& a, cudaStream_t st, bool f8) {
#define EMU_P(PP)                                                                       \
  case PP:                                                                              \
    if (f8) {                                                                           \
      if (out_mode == OUT_F64) return launch_p<PP, OUT_F64, true>(a, st);               \
      if (out_mode == OUT_F32) return launch_p<PP, OUT_F32, true>(a, st);               \
      return launch_p<PP, OUT_PARTIALS, true>(a, st);                                   \
    }                                                                                   \
    if (out_mode == OUT_F64) return launch_p<PP, OUT_F64, false>(a, st);                \
    if (out_mode == OUT_F32) return launch_p<PP, OUT_F32, false>(a, st);                \
    return launch_p<PP, OUT_PARTIALS, false>(a, st);
  switch (p) {
    EMU_P(1) EMU_P(2) EMU_P(3) EMU_P(4) EMU_P(5) EMU_P(6)
    EMU_P(7) EMU_P(8) EMU_P(9) EMU_P(10) EMU_P(11) EMU_P(12)
    default:
      return cudaErrorInvalidValue;
  }
#undef EMU_P
}

}  // namespace emu
