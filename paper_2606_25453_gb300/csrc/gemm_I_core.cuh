// gemm_I_core.cuh -- per-warp pieces of the fused Scheme I main loop shared
// by the single-product and the grouped kernels: the triangular slice-pair
// schedule of Eq. (2) on a 16 x 16 warp patch (in two orders: B-slice-major
// and A-slice-major), and the exact drain of the p accumulator sets into
// 128-bit integers (Eq. 3 without rounding).
//
// Two slice engines share the code: INT8 slices (beta = 8, signed leading /
// unsigned tail bytes, int32 accumulators, INT8 mma.sync) and E4M3 slices
// (beta = 5, balanced base-32 digits, FP32 accumulators that stay exact
// below 2^24, FP8 mma.sync).
#pragma once
#include "emu_device.cuh"

namespace emu {

template <bool F8>
struct Engine;
template <>
struct Engine<false> {
  using Acc = int32_t;
  static constexpr int kBeta = 8;
  template <int I, int J>
  __device__ __forceinline__ static void mma(Acc* d, const uint32_t* a, const uint32_t* b) {
    mma_i8<I == 0, J == 0>(d, a, b);
  }
  __device__ __forceinline__ static long long to_int(Acc v) { return v; }
};
template <>
struct Engine<true> {
  using Acc = float;
  static constexpr int kBeta = 5;
  template <int I, int J>
  __device__ __forceinline__ static void mma(Acc* d, const uint32_t* a, const uint32_t* b) {
    mma_e4m3(d, a, b);
  }
  __device__ __forceinline__ static long long to_int(Acc v) { return __float2ll_rn(v); }  // exact integer
};

// acc[s] += A'_i B'_j for all i + j = s < P, for one B slice j (static).
template <int P, bool F8, int J, int I = 0>
struct TriRow {
  using Acc = typename Engine<F8>::Acc;
  __device__ __forceinline__ static void run(Acc (*acc)[2][4], const uint32_t (*af)[4], const uint32_t* bf) {
    if constexpr (I + J < P) {
      Engine<F8>::template mma<I, J>(acc[I + J][0], af[I], bf);
      Engine<F8>::template mma<I, J>(acc[I + J][1], af[I], bf + 2);
      TriRow<P, F8, J, I + 1>::run(acc, af, bf);
    }
  }
};

template <int P, int BLKB, bool F8, int J = 0>
struct TriAll {
  using Acc = typename Engine<F8>::Acc;
  __device__ __forceinline__ static void run(Acc (*acc)[2][4], const uint32_t (*af)[4], uint32_t sB, uint32_t b_off) {
    if constexpr (J < P) {
      uint32_t bf[4];
      ldsm_x4(sB + J * BLKB + b_off, bf[0], bf[1], bf[2], bf[3]);
      TriRow<P, F8, J>::run(acc, af, bf);
      TriAll<P, BLKB, F8, J + 1>::run(acc, af, sB, b_off);
    }
  }
};

// The same triangle in A-slice-major order: the P B-slice fragments are
// loaded first, then row i of the triangle (acc[i + j] += A'_i B'_j for
// j < P - i) is issued as one run of MMAs.  More registers (4 P for the
// fragments) against fewer shared-memory loads between MMAs of one slice
// pair row; which order is faster depends on p and the tile, so the grouped
// autotuner chooses.
template <int P, bool F8, int I, int J = 0>
struct TriRowA {
  using Acc = typename Engine<F8>::Acc;
  __device__ __forceinline__ static void run(Acc (*acc)[2][4], const uint32_t (*af)[4], const uint32_t (*bf)[4]) {
    if constexpr (I + J < P) {
      Engine<F8>::template mma<I, J>(acc[I + J][0], af[I], bf[J]);
      Engine<F8>::template mma<I, J>(acc[I + J][1], af[I], bf[J] + 2);
      TriRowA<P, F8, I, J + 1>::run(acc, af, bf);
    }
  }
};

template <int P, bool F8, int I = 0>
struct TriRowsA {
  using Acc = typename Engine<F8>::Acc;
  __device__ __forceinline__ static void run(Acc (*acc)[2][4], const uint32_t (*af)[4], const uint32_t (*bf)[4]) {
    if constexpr (I < P) {
      TriRowA<P, F8, I>::run(acc, af, bf);
      TriRowsA<P, F8, I + 1>::run(acc, af, bf);
    }
  }
};

template <int P, int BLKB, bool F8>
struct TriAllByA {
  using Acc = typename Engine<F8>::Acc;
  __device__ __forceinline__ static void run(Acc (*acc)[2][4], const uint32_t (*af)[4], uint32_t sB, uint32_t b_off) {
    uint32_t bf[P][4];
#pragma unroll
    for (int j = 0; j < P; ++j) ldsm_x4(sB + j * BLKB + b_off, bf[j][0], bf[j][1], bf[j][2], bf[j][3]);
    TriRowsA<P, F8>::run(acc, af, bf);
  }
};

// S += sum_s C_s * 2^(beta (P-1-s)) exactly, then clear the accumulators.
template <int P, bool F8>
__device__ __forceinline__ void fold(typename Engine<F8>::Acc (*acc)[2][4], __int128 (*S)[4]) {
  constexpr int kBase = 1 << Engine<F8>::kBeta;
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __int128 t = Engine<F8>::to_int(acc[0][nt][q]);
#pragma unroll
      for (int s = 1; s < P; ++s) t = t * kBase + Engine<F8>::to_int(acc[s][nt][q]);
      S[nt][q] += t;
#pragma unroll
      for (int s = 0; s < P; ++s) acc[s][nt][q] = 0;
    }
}

}  // namespace emu
