// gemm_I_core.cuh -- per-warp pieces of the fused Scheme I main loop shared
// by the single-product and the grouped kernels: the triangular slice-pair
// schedule of Eq. (2) on a 16 x 16 warp patch, and the exact drain of the p
// INT32 accumulator sets into 128-bit integers (Eq. 3 without rounding).
#pragma once
#include "emu_device.cuh"

namespace emu {

template <int I, int J>
__device__ __forceinline__ void mma_slice(int32_t* d, const uint32_t* a, const uint32_t* b) {
  mma_i8<I == 0, J == 0>(d, a, b);
}

// acc[s] += A'_i B'_j for all i + j = s < P, for one B slice j (static).
template <int P, int J, int I = 0>
struct TriRow {
  __device__ __forceinline__ static void run(int32_t (*acc)[2][4], const uint32_t (*af)[4],
                                             const uint32_t* bf) {
    if constexpr (I + J < P) {
      mma_slice<I, J>(acc[I + J][0], af[I], bf);
      mma_slice<I, J>(acc[I + J][1], af[I], bf + 2);
      TriRow<P, J, I + 1>::run(acc, af, bf);
    }
  }
};

template <int P, int BLKB, int J = 0>
struct TriAll {
  __device__ __forceinline__ static void run(int32_t (*acc)[2][4], const uint32_t (*af)[4],
                                             uint32_t sB, uint32_t b_off) {
    if constexpr (J < P) {
      uint32_t bf[4];
      ldsm_x4(sB + J * BLKB + b_off, bf[0], bf[1], bf[2], bf[3]);
      TriRow<P, J>::run(acc, af, bf);
      TriAll<P, BLKB, J + 1>::run(acc, af, sB, b_off);
    }
  }
};

template <int P>
__device__ __forceinline__ void fold(int32_t (*acc)[2][4], __int128 (*S)[4]) {
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __int128 t = acc[0][nt][q];
#pragma unroll
      for (int s = 1; s < P; ++s) t = t * 256 + acc[s][nt][q];
      S[nt][q] += t;
#pragma unroll
      for (int s = 0; s < P; ++s) acc[s][nt][q] = 0;
    }
}

}  // namespace emu
