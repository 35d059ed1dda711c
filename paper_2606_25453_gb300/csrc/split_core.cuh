// split_core.cuh -- per-element Scheme I slicing shared by the dense and
// the grouped split kernels: two's-complement INT8 bytes, balanced base-32
// E4M3 digits, and the packing of four consecutive K elements into one
// 32-bit word per slice.
#pragma once
#include "emu_device.cuh"

namespace emu {

// Bytes of the 8P-bit two's complement of x = sign * (mag << lsh).
template <int P>
__device__ __forceinline__ void slice_digits(uint64_t bits, int E, uint32_t* out) {
  ScaledInt s = scaled_trunc_bits(bits, 8 * P - 1 - E);
  bool neg = (bits >> 63) != 0;
  if (P <= 8) {
    uint64_t v = s.lsh < 64 ? (s.mag << s.lsh) : 0ull;  // < 2^(8P-1) <= 2^63
    if (neg) v = ~v + 1ull;
#pragma unroll
    for (int t = 0; t < P; ++t) out[t] = static_cast<uint32_t>((v >> (8 * (P - 1 - t))) & 0xFFu);
  } else {
    unsigned __int128 v = s.lsh < 128 ? (static_cast<unsigned __int128>(s.mag) << s.lsh)
                                      : static_cast<unsigned __int128>(0);
    if (neg) v = ~v + static_cast<unsigned __int128>(1);
#pragma unroll
    for (int t = 0; t < P; ++t) out[t] = static_cast<uint32_t>((v >> (8 * (P - 1 - t))) & 0xFFu);
  }
}

__device__ __forceinline__ int exp_from_maxbits(const unsigned long long* maxbits, int64_t r,
                                                int64_t rows) {
  if (r >= rows) return 0;
  uint64_t mb = maxbits[r];
  if (mb >= 0x7FF0000000000000ull) return 0;  // non-finite: flagged by the scan
  return frexp_exp_bits(mb);
}

// Bit pattern (binary64) of an element: binary32 sources are widened exactly.
__device__ __forceinline__ uint64_t elem_bits(double x) { return dbits(x); }
__device__ __forceinline__ uint64_t elem_bits(float x) { return dbits(static_cast<double>(x)); }

// Elements h0 .. h0+3 (h0 a multiple of 4) of a K-contiguous vector starting
// at `row`, as binary64 bit patterns; zero past k and for a padding vector
// (live false).  `vec`: the vector starts on a 16-byte boundary, so the four
// elements are one (binary32) or two (binary64) aligned 16-byte loads
// whenever all four lie inside.
template <typename T>
__device__ __forceinline__ void load4_kcontig(const T* row, int64_t h0, int64_t k, bool live, bool vec,
                                              uint64_t* bits) {
  if (live && vec && h0 + 3 < k) {
    const uint4* pv = reinterpret_cast<const uint4*>(row + h0);
    if constexpr (sizeof(T) == 8) {
      const uint4 v0 = __ldg(pv), v1 = __ldg(pv + 1);
      bits[0] = (static_cast<uint64_t>(v0.y) << 32) | v0.x;
      bits[1] = (static_cast<uint64_t>(v0.w) << 32) | v0.z;
      bits[2] = (static_cast<uint64_t>(v1.y) << 32) | v1.x;
      bits[3] = (static_cast<uint64_t>(v1.w) << 32) | v1.z;
    } else {
      const uint4 v = __ldg(pv);
      bits[0] = elem_bits(__uint_as_float(v.x));
      bits[1] = elem_bits(__uint_as_float(v.y));
      bits[2] = elem_bits(__uint_as_float(v.z));
      bits[3] = elem_bits(__uint_as_float(v.w));
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) bits[q] = (live && h0 + q < k) ? elem_bits(__ldg(row + h0 + q)) : 0ull;
}

// Fill tile[32][133] with 32 K-strided vectors r0 .. r0+31 x 128 elements
// hbase .. hbase+127 (element (r, h) at X[h ld + r]; zero outside rows x k),
// element hl of vector rl at column (hl mod 4) 33 + hl / 4, by all 256
// threads of the block.  With `vec` (X on a 16-byte boundary, ld a multiple
// of 16 bytes) each thread reads 16 contiguous bytes: 16 / sizeof(T)
// consecutive vectors of one K row.
template <typename T>
__device__ __forceinline__ void fill_tile_strided(uint64_t (*tile)[133], const T* X, int64_t ld, int64_t rows,
                                                  int64_t k, int64_t r0, int64_t hbase, bool vec) {
  constexpr int V = 16 / static_cast<int>(sizeof(T));  // vectors per 16-byte load
  constexpr int LPR = 32 / V;                           // threads per K row
#pragma unroll 4
  for (int it = 0; it < 32 * 128 / V / 256; ++it) {
    const int i = threadIdx.x + it * 256;
    const int rl = (i % LPR) * V, hl = i / LPR;
    const int64_t r = r0 + rl, h = hbase + hl;
    const int col = (hl & 3) * 33 + (hl >> 2);
    const T* p = X + h * ld + r;
    if (vec && h < k && r + V <= rows) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
      if constexpr (sizeof(T) == 8) {
        tile[rl][col] = (static_cast<uint64_t>(v.y) << 32) | v.x;
        tile[rl + 1][col] = (static_cast<uint64_t>(v.w) << 32) | v.z;
      } else {
        tile[rl][col] = elem_bits(__uint_as_float(v.x));
        tile[rl + 1][col] = elem_bits(__uint_as_float(v.y));
        tile[rl + 2][col] = elem_bits(__uint_as_float(v.z));
        tile[rl + 3][col] = elem_bits(__uint_as_float(v.w));
      }
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j) tile[rl + j][col] = (r + j < rows && h < k) ? elem_bits(__ldg(p + j)) : 0ull;
    }
  }
}

// True when 16-byte loads of the vectors of X (leading dimension ld) are
// aligned: X on a 16-byte boundary and ld a multiple of 16 bytes.
template <typename T>
inline bool vec16_ok(const T* X, int64_t ld) {
  return (reinterpret_cast<uintptr_t>(X) & 15u) == 0 && (static_cast<uint64_t>(ld) * sizeof(T)) % 16 == 0;
}

// E4M3 bytes of two digits given as exact small integers in float: the
// conversion of a lands in the upper byte, that of b in the lower byte.
__device__ __forceinline__ uint32_t e4m3x2(float a, float b) {
  unsigned short r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(a), "f"(b));
  return static_cast<uint32_t>(r);
}

// Four consecutive K elements of one vector (their binary64 bits) -> for
// every slice t one 32-bit word holding the four slice bytes in K order
// (byte q = element q).
// E4M3 slices (beta = 5): balanced base-32 digits of x = sign * (mag << lsh),
// |x| < 2^(5P-1) <= 2^59 (leading digit in [-16, 16], the others in
// [-16, 15]), each encoded as its exact E4M3 byte.  Adding 16 * 32^t for
// every lower position t turns the balanced digits into plain base-32 digits
// of the biased value y, so all digits come from independent shifts:
// d_t = ((y >> 5(P-1-t)) & 31) - 16 for t >= 1, d_0 = y >> 5(P-1).  Each
// digit becomes an exact float through the 1.5 * 2^23 bit pattern (field f
// -> f - 16 in one OR and one FADD), and the hardware conversion packs two
// at a time.  INT8: the bytes of the two's complement (slice_digits).
template <int P, bool F8>
__device__ __forceinline__ void pack4(const uint64_t* bits, int E, uint32_t* word) {
  if (F8) {
    constexpr long long kBias = [] {
      long long b = 0;
      for (int t = 1; t < P; ++t) b = b * 32 + 16;
      return b;
    }();
    long long y[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const ScaledInt sc = scaled_trunc_bits(bits[q], 5 * P - 1 - E);
      long long x = static_cast<long long>(sc.lsh < 64 ? (sc.mag << sc.lsh) : 0ull);
      if ((bits[q] >> 63) != 0) x = -x;
      y[q] = x + kBias;
    }
#pragma unroll
    for (int t = 0; t < P; ++t) {
      float f[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (t == 0) {  // leading digit, in [-16, 16]
          const int d = static_cast<int>(y[q] >> (5 * (P - 1)));
          f[q] = __int_as_float(0x4B400000 + d) - 12582912.0f;
        } else {  // field in [0, 31], digit = field - 16
          const int fld = static_cast<int>((y[q] >> (5 * (P - 1 - t))) & 31);
          f[q] = __int_as_float(0x4B400000 | fld) - 12582928.0f;
        }
      }
      word[t] = e4m3x2(f[1], f[0]) | (e4m3x2(f[3], f[2]) << 16);
    }
  } else {
#pragma unroll
    for (int t = 0; t < P; ++t) word[t] = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t dg[P];
      slice_digits<P>(bits[q], E, dg);
#pragma unroll
      for (int t = 0; t < P; ++t) word[t] |= (dg[t] & 0xFFu) << (8 * q);
    }
  }
}

}  // namespace emu
