// gemm_II.cu -- fused Scheme II kernel (Sec. IV) with the CRT in the epilogue.
//
// Same persistent TMA/mbarrier skeleton as the Scheme I kernel.  For every
// output tile the K loop runs once per modulus m_l over that modulus's
// residue planes (Eq. 6) with a single INT32 accumulator set; at the end of
// each modulus the accumulator is reduced modulo m_l in registers (Eq. 7)
// and immediately folded into a multi-word CRT sum S += w_l * r_l with
// w_l = (P/m_l) q_l (Eq. 8).  After the last modulus S is reduced modulo P,
// lifted to the symmetric range, rounded once to binary64 and scaled back
// (inverse scaling after Eq. 8).  Unlike the paper, which writes the INT8
// residues to global memory and runs a separate CRT kernel (Sec. IV-C),
// no per-modulus result leaves the chip.
//
// Complex input (II_Z3M) uses the 3M method of Sec. IV-B (Eq. 16): per
// modulus three K loops (re*re, im*im, sum*sum) reuse one accumulator, T1
// and T2 are kept as residues in registers, and Re = T1 - T2,
// Im = T3 - T1 - T2 (mod m_l) feed two CRT sums.
// II_RESIDUES writes the per-modulus residues (the paper's kernel output).
#include <type_traits>

#include "crt_core.cuh"
#include "emu_internal.h"

namespace emu {

namespace {

constexpr int kBM = 64, kBN = 32;
constexpr int kCW = 8;
constexpr int kThreads = (kCW + 1) * 32;
constexpr int kKS = 4;  // 32-wide K-chunks per pipeline stage
constexpr int kBlkA = kBM * 32, kBlkB = kBN * 32;
constexpr int kStageBytes = kKS * (kBlkA + kBlkB);
constexpr int kStages = 8;
constexpr int kSmem = kStages * kStageBytes + 1024 + 2 * kStages * 8 + 64;

struct KParamsII {
  CUtensorMap tA;
  CUtensorMap tB;
  int M, N, nst, tiles_m, tiles_n;  // nst: pipeline stages per plane (K / 128)
  int rowsA_pad, rowsB_pad, nm;
  const int32_t* EA;
  const int32_t* FB;
  int escale;
  double alpha_re, alpha_im, beta_re, beta_im;
  void* C;
  int64_t ldc;
  uint8_t* residues;
  int* status;
};

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

__device__ __forceinline__ uint32_t modpos(int32_t v, uint32_t m) {
  int32_t r = v % static_cast<int32_t>(m);
  return static_cast<uint32_t>(r < 0 ? r + static_cast<int32_t>(m) : r);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_II_kernel(const __grid_constant__ KParamsII kp, const __grid_constant__ CrtTables ct,
                   const __grid_constant__ ModTables mt) {
  constexpr bool CPLX = MODE == II_Z3M || MODE == II_C3M;  // 3M complex, f64 or f32 output
  constexpr int NSET = CPLX ? 3 : 1;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kCW);
    }
    fence_mbar_init();
  }
  __syncthreads();
  const int ntiles = kp.tiles_m * kp.tiles_n;
  const int nm = kp.nm;

  if (warp == kCW) {
    if (lane == 0) {
      tma_prefetch_desc(&kp.tA);
      tma_prefetch_desc(&kp.tB);
      uint32_t it = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int tm, tn;
        tile_coords(tile, kp.tiles_m, kp.tiles_n, tm, tn);
        for (int l = 0; l < nm; ++l)
          for (int set = 0; set < NSET; ++set) {
            const int ya = (set * nm + l) * kp.rowsA_pad + tm * kBM;
            const int yb = (set * nm + l) * kp.rowsB_pad + tn * kBN;
            for (int ks = 0; ks < kp.nst; ++ks, ++it) {
              const uint32_t stage = it % kStages;
              const uint32_t par = (it / kStages) & 1u;
              if (it >= static_cast<uint32_t>(kStages) && !mbar_wait_bounded(&empty[stage], par ^ 1u)) {
                set_status(kp.status, ST_TIMEOUT);
                return;
              }
              mbar_arrive_expect_tx(&full[stage], kStageBytes);
              uint8_t* sA = smem + stage * kStageBytes;
              uint8_t* sB = sA + kKS * kBlkA;
#pragma unroll
              for (int c = 0; c < kKS; ++c)
                tma_load_2d(sA + c * kBlkA, &kp.tA, &full[stage], (ks * kKS + c) * 32, ya);
#pragma unroll
              for (int c = 0; c < kKS; ++c)
                tma_load_2d(sB + c * kBlkB, &kp.tB, &full[stage], (ks * kKS + c) * 32, yb);
            }
          }
      }
    }
    return;
  }

  const int wm = warp >> 1, wn = warp & 1;
  const uint32_t a_off = swz32(wm * 16 + (lane & 15), lane >> 4);
  const uint32_t b_off = swz32(wn * 16 + (lane & 7) + ((lane >> 4) << 3), (lane >> 3) & 1);
  uint32_t it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int tm, tn;
    tile_coords(tile, kp.tiles_m, kp.tiles_n, tm, tn);
    const int row0 = tm * kBM + wm * 16 + (lane >> 2);
    const int col0 = tn * kBN + wn * 16 + (lane & 3) * 2;
    uint32_t Sre[8][kSL];
    uint32_t Sim[CPLX ? 8 : 1][kSL];
#pragma unroll
    for (int e = 0; e < 8; ++e)
#pragma unroll
      for (int i = 0; i < kSL; ++i) {
        Sre[e][i] = 0;
        if (CPLX) Sim[e][i] = 0;
      }
    uint32_t t1[CPLX ? 8 : 1], t2[CPLX ? 8 : 1];
    for (int l = 0; l < nm; ++l) {
      const uint32_t m = mt.mods[l];
      for (int set = 0; set < NSET; ++set) {
        // two accumulator sets (even / odd K-chunks) give the tensor pipe
        // four independent MMA chains per warp; summed before the reduction
        // (exact: the total is the same INT32-bounded sum)
        int32_t acc[2][4], acc2[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[nt][q] = acc2[nt][q] = 0;
        for (int ks = 0; ks < kp.nst; ++ks, ++it) {
          const uint32_t stage = it % kStages;
          const uint32_t par = (it / kStages) & 1u;
          if (!mbar_wait_bounded(&full[stage], par)) {
            set_status(kp.status, ST_TIMEOUT);
            return;
          }
          const uint32_t sA = base + stage * kStageBytes;
          const uint32_t sB = sA + kKS * kBlkA;
#pragma unroll
          for (int c = 0; c < kKS; ++c) {
            uint32_t af[4], bf[4];
            ldsm_x4(sA + c * kBlkA + a_off, af[0], af[1], af[2], af[3]);
            ldsm_x4(sB + c * kBlkB + b_off, bf[0], bf[1], bf[2], bf[3]);
            if (c & 1) {
              mma_i8<true, true>(acc2[0], af, bf);
              mma_i8<true, true>(acc2[1], af, bf + 2);
            } else {
              mma_i8<true, true>(acc[0], af, bf);
              mma_i8<true, true>(acc[1], af, bf + 2);
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[stage]);
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[nt][q] += acc2[nt][q];
        // Eq. (7): residue in [0, m) per element, then CRT accumulation
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int nt = e >> 2, q = e & 3;
          uint32_t r = modpos(acc[nt][q], m);
          if (MODE == II_RESIDUES) {
            int row = row0 + (q >> 1) * 8, col = col0 + nt * 8 + (q & 1);
            if (row < kp.M && col < kp.N)
              kp.residues[(static_cast<int64_t>(l) * kp.M + row) * kp.N + col] = static_cast<uint8_t>(r);
          } else if (CPLX) {
            if (set == 0) {
              t1[e] = r;
            } else if (set == 1) {
              t2[e] = r;
            } else {
              uint32_t re = (t1[e] + m - t2[e]) % m;
              uint32_t im = (r + 2 * m - t1[e] - t2[e]) % m;
              crt_acc(Sre[e], ct.w[l], re);
              crt_acc(Sim[e], ct.w[l], im);
            }
          } else {
            crt_acc(Sre[e], ct.w[l], r);
          }
        }
      }
    }
    if (MODE == II_RESIDUES) continue;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int nt = e >> 2, q = e & 3;
      int row = row0 + (q >> 1) * 8, col = col0 + nt * 8 + (q & 1);
      if (row >= kp.M || col >= kp.N) continue;
      const int sc = kp.EA[row] + kp.FB[col] + kp.escale;
      double rr = scale2(crt_finish(Sre[e], ct), sc);
      if (CPLX) {
        // complex update in binary64; complex64 output rounds each part once more
        using TO = typename std::conditional<MODE == II_C3M, float, double>::type;
        double ri = scale2(crt_finish(Sim[e], ct), sc);
        TO* cp = static_cast<TO*>(kp.C) + 2 * (static_cast<int64_t>(row) * kp.ldc + col);
        double tr = __fma_rn(kp.alpha_re, rr, -__dmul_rn(kp.alpha_im, ri));
        double ti = __fma_rn(kp.alpha_re, ri, __dmul_rn(kp.alpha_im, rr));
        if (kp.beta_re != 0.0 || kp.beta_im != 0.0) {
          double cr = static_cast<double>(cp[0]), ci = static_cast<double>(cp[1]);
          double ur = __fma_rn(kp.beta_re, cr, -__dmul_rn(kp.beta_im, ci));
          double ui = __fma_rn(kp.beta_re, ci, __dmul_rn(kp.beta_im, cr));
          tr = __dadd_rn(tr, ur);
          ti = __dadd_rn(ti, ui);
        }
        cp[0] = static_cast<TO>(tr);
        cp[1] = static_cast<TO>(ti);
      } else if (MODE == II_F64) {
        double* cp = static_cast<double*>(kp.C) + static_cast<int64_t>(row) * kp.ldc + col;
        *cp = blas_update(kp.alpha_re, rr, kp.beta_re, kp.beta_re != 0.0 ? *cp : 0.0);
      } else {
        float* cp = static_cast<float*>(kp.C) + static_cast<int64_t>(row) * kp.ldc + col;
        *cp = static_cast<float>(
            blas_update(kp.alpha_re, rr, kp.beta_re, kp.beta_re != 0.0 ? static_cast<double>(*cp) : 0.0));
      }
    }
  }
}

template <int MODE>
cudaError_t launch_mode(const GemmIIArgs& a, const ModTables& mt, const CrtTables& ct,
                        cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(gemm_II_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmem);
  if (e != cudaSuccess) return e;
  KParamsII kp;
  kp.tA = *a.descA;
  kp.tB = *a.descB;
  kp.M = a.M;
  kp.N = a.N;
  kp.nst = (a.nk32 + kKS - 1) / kKS;
  kp.tiles_m = (a.M + kBM - 1) / kBM;
  kp.tiles_n = (a.N + kBN - 1) / kBN;
  kp.rowsA_pad = a.rowsA_pad;
  kp.rowsB_pad = a.rowsB_pad;
  kp.nm = a.nm;
  kp.EA = a.EA;
  kp.FB = a.FB;
  kp.escale = a.escale;
  kp.alpha_re = a.alpha_re;
  kp.alpha_im = a.alpha_im;
  kp.beta_re = a.beta_re;
  kp.beta_im = a.beta_im;
  kp.C = a.C;
  kp.ldc = a.ldc;
  kp.residues = a.residues;
  kp.status = a.status;
  int ntiles = kp.tiles_m * kp.tiles_n;
  if (ntiles == 0) return cudaSuccess;
  int grid = ntiles < a.num_sms ? ntiles : a.num_sms;
  gemm_II_kernel<MODE><<<grid, kThreads, kSmem, st>>>(kp, ct, mt);
  return cudaGetLastError();
}

}  // namespace

int gemm_II_kchunk() { return kKS * 32; }

cudaError_t launch_gemm_II(int out_mode, const GemmIIArgs& a, const ModTables& mt,
                           const CrtTables& ct, cudaStream_t st) {
  switch (out_mode) {
    case II_F64:
      return launch_mode<II_F64>(a, mt, ct, st);
    case II_F32:
      return launch_mode<II_F32>(a, mt, ct, st);
    case II_RESIDUES:
      return launch_mode<II_RESIDUES>(a, mt, ct, st);
    case II_Z3M:
      return launch_mode<II_Z3M>(a, mt, ct, st);
    case II_C3M:
      return launch_mode<II_C3M>(a, mt, ct, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace emu
