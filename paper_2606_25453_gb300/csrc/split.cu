// split.cu -- exponent scan and slice / residue packing (HBM-bound steps).
//
// Scan (Eq. 1 scale vectors; Scheme II scaling): for every reduction vector
// of an operand (row of A, column of B) the largest |x| is found by an
// unsigned max over the IEEE-754 bit patterns with the sign cleared (which
// orders finite magnitudes), so the scan does no floating-point arithmetic.
// Non-finite values have bit patterns >= 0x7FF0... and set the status word.
//
// Split I (Eq. 1, layout Eq. 11): x = trunc(a * 2^(8p-1-E)) taken exactly
// from the bits of a; the p bytes of the 8p-bit two's complement of x are
// the slices (leading slice signed, tails unsigned), written interleaved:
// row r, K-chunk c (32 wide), slice t at bytes [(c*p+t)*32, +32).
//
// Split I on E4M3 slices: the same layout with beta = 5 balanced base-32
// digits stored as exact E4M3 bytes (the FP8 formulation of Sec. VII).
//
// Split II (Eq. 5): a' = trunc(a * 2^(b-E)), symmetric residues modulo the
// moduli, one plane per modulus; complex input also writes the residues of
// a'_re + a'_im for the 3M product (Eq. 16).
#include "emu_internal.h"
#include "split_core.cuh"

namespace emu {

// ------------------------------------------------------------------ loads
template <typename T>
__device__ __forceinline__ uint64_t load_absbits(const T* p);
template <>
__device__ __forceinline__ uint64_t load_absbits<double>(const double* p) {
  return dbits(__ldg(p)) & 0x7FFFFFFFFFFFFFFFull;
}
template <>
__device__ __forceinline__ uint64_t load_absbits<float>(const float* p) {
  return dbits(static_cast<double>(__ldg(p))) & 0x7FFFFFFFFFFFFFFFull;  // exact widening
}
template <typename T>
__device__ __forceinline__ uint64_t load_bits(const T* p);
template <>
__device__ __forceinline__ uint64_t load_bits<double>(const double* p) {
  return dbits(__ldg(p));
}
template <>
__device__ __forceinline__ uint64_t load_bits<float>(const float* p) {
  return dbits(static_cast<double>(__ldg(p)));
}

// ------------------------------------------------------------------ scan
// Vector r, element h of operand X: kcontig -> X[(r*ld + h)*cw + part],
// else X[(h*ld + r)*cw + part]; cw = 2 for complex (both parts scanned).
// seg: elements of a vector per block row (K segment), chosen by the launcher.
template <typename T, bool KCONTIG>
__global__ void scan_kernel(const T* __restrict__ X, int64_t ld, int64_t rows, int64_t k, int cw, int64_t seg,
                            unsigned long long* __restrict__ maxbits, int* status) {
  if (KCONTIG) {
    // one warp per (row, K segment)
    int lane = threadIdx.x & 31;
    int64_t r = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    int64_t len = k * cw;
    int64_t h0 = static_cast<int64_t>(blockIdx.y) * seg;
    int64_t h1 = h0 + seg < len ? h0 + seg : len;
    const T* row = X + r * ld * cw;
    uint64_t mx = 0;
    for (int64_t h = h0 + lane; h < h1; h += 32) {
      uint64_t v = load_absbits(row + h);
      mx = v > mx ? v : mx;
    }
    for (int o = 16; o; o >>= 1) {
      uint64_t w = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = w > mx ? w : mx;
    }
    if (lane == 0 && h0 < h1) {
      atomicMax(maxbits + r, static_cast<unsigned long long>(mx));
      if (mx >= 0x7FF0000000000000ull) set_status(status, ST_NONFINITE);
    }
  } else {
    // block 32 x 8: lanes over vectors (coalesced), 8 row-groups over K
    int64_t r = static_cast<int64_t>(blockIdx.x) * 32 + threadIdx.x;
    int64_t h0 = static_cast<int64_t>(blockIdx.y) * seg;
    int64_t h1 = h0 + seg < k ? h0 + seg : k;
    uint64_t mx = 0;
    if (r < rows) {
      for (int64_t h = h0 + threadIdx.y; h < h1; h += blockDim.y) {
        const T* p = X + (h * ld + r) * cw;
        uint64_t v = load_absbits(p);
        mx = v > mx ? v : mx;
        if (cw == 2) {
          uint64_t w = load_absbits(p + 1);
          mx = w > mx ? w : mx;
        }
      }
    }
    __shared__ uint64_t red[8][32];
    red[threadIdx.y][threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.y == 0 && r < rows) {
      for (int q = 1; q < blockDim.y; ++q) mx = red[q][threadIdx.x] > mx ? red[q][threadIdx.x] : mx;
      if (h0 < h1) {
        atomicMax(maxbits + r, static_cast<unsigned long long>(mx));
        if (mx >= 0x7FF0000000000000ull) set_status(status, ST_NONFINITE);
      }
    }
  }
}

// The same scan with 16-byte loads, for operands whose vectors start on
// 16-byte boundaries (base and leading dimension aligned).  A uint4 holds
// S = 16 / sizeof(T) scalars, CV = S / cw vectors of the strided layout.
// Float magnitudes are compared on their own bit patterns and the largest
// is widened once (widening is exact and monotone, so the result is the
// same as that of the scalar scan).
template <typename T>
__device__ __forceinline__ uint64_t widen_absbits(uint64_t b);
template <>
__device__ __forceinline__ uint64_t widen_absbits<double>(uint64_t b) {
  return b;
}
template <>
__device__ __forceinline__ uint64_t widen_absbits<float>(uint64_t b) {
  return dbits(static_cast<double>(__uint_as_float(static_cast<uint32_t>(b))));
}
// |scalar j| of a uint4 as unsigned bits of T's width (sign cleared)
template <typename T>
__device__ __forceinline__ uint64_t lane_absbits(const uint4& v, int j) {
  if constexpr (sizeof(T) == 8) {
    const uint32_t lo = j == 0 ? v.x : v.z, hi = j == 0 ? v.y : v.w;
    return ((static_cast<uint64_t>(hi) << 32) | lo) & 0x7FFFFFFFFFFFFFFFull;
  } else {
    const uint32_t w = j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
    return w & 0x7FFFFFFFu;
  }
}

template <typename T>
__device__ __forceinline__ uint64_t scalar_absbits(T x) {
  if constexpr (sizeof(T) == 8)
    return dbits(x) & 0x7FFFFFFFFFFFFFFFull;
  else
    return __float_as_uint(x) & 0x7FFFFFFFu;
}

template <typename T, bool KCONTIG>
__global__ void scan_vec_kernel(const T* __restrict__ X, int64_t ld, int64_t rows, int64_t k, int cw, int64_t seg,
                                unsigned long long* __restrict__ maxbits, int* status) {
  constexpr int S = 16 / static_cast<int>(sizeof(T));
  if (KCONTIG) {
    // one warp per (row, segment of seg scalars); lane l loads uint4 l, l + 32, ...
    const int lane = threadIdx.x & 31;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const int64_t len = k * cw, h0 = static_cast<int64_t>(blockIdx.y) * seg;
    const int64_t h1 = h0 + seg < len ? h0 + seg : len;
    const T* row = X + r * ld * cw;
    const int64_t nv = (h1 - h0) / S;
    const uint4* pv = reinterpret_cast<const uint4*>(row + h0);
    uint64_t mx = 0;
#pragma unroll 4
    for (int64_t i = lane; i < nv; i += 32) {
      const uint4 v = __ldg(pv + i);
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const uint64_t a = lane_absbits<T>(v, j);
        mx = a > mx ? a : mx;
      }
    }
    for (int64_t h = h0 + nv * S + lane; h < h1; h += 32) {  // ragged end of the row
      const uint64_t a = scalar_absbits<T>(__ldg(row + h));
      mx = a > mx ? a : mx;
    }
    for (int o = 16; o; o >>= 1) {
      const uint64_t w = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = w > mx ? w : mx;
    }
    if (lane == 0 && h0 < h1) {
      mx = widen_absbits<T>(mx);
      atomicMax(maxbits + r, static_cast<unsigned long long>(mx));
      if (mx >= 0x7FF0000000000000ull) set_status(status, ST_NONFINITE);
    }
  } else {
    // block 32 x 8: lane x loads the CV vectors x*CV .. x*CV + CV - 1 of a
    // block of 32*CV vectors (512 contiguous bytes per warp and K row);
    // the 8 row-groups split a K segment of seg
    const int cv = S / cw;
    const int64_t rb = static_cast<int64_t>(blockIdx.x) * 32 * cv;
    const int64_t r = rb + static_cast<int64_t>(threadIdx.x) * cv;
    const int64_t h0 = static_cast<int64_t>(blockIdx.y) * seg;
    const int64_t h1 = h0 + seg < k ? h0 + seg : k;
    uint64_t mx[4] = {0, 0, 0, 0};
    if (r + cv <= rows) {
#pragma unroll 4
      for (int64_t h = h0 + threadIdx.y; h < h1; h += 8) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(X + (h * ld + r) * cw));
#pragma unroll
        for (int j = 0; j < S; ++j) {  // scalar j belongs to vector j / cw (cw is 1 or 2)
          const uint64_t a = lane_absbits<T>(v, j);
          if (cw == 2)
            mx[j >> 1] = a > mx[j >> 1] ? a : mx[j >> 1];
          else
            mx[j] = a > mx[j] ? a : mx[j];
        }
      }
    } else if (r < rows) {  // the last vectors of the operand: scalar loads
      for (int64_t h = h0 + threadIdx.y; h < h1; h += 8) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c < cv && r + c < rows) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              if (q < cw) {
                const uint64_t a = scalar_absbits<T>(__ldg(X + (h * ld + r + c) * cw + q));
                mx[c] = a > mx[c] ? a : mx[c];
              }
            }
          }
        }
      }
    }
    __shared__ uint64_t red[8][32 * 4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < cv) red[threadIdx.y][threadIdx.x * cv + c] = mx[c];
    __syncthreads();
    const int t = threadIdx.y * 32 + threadIdx.x;
    if (t < 32 * cv && rb + t < rows && h0 < h1) {
      uint64_t m = red[0][t];
      for (int q = 1; q < 8; ++q) m = red[q][t] > m ? red[q][t] : m;
      m = widen_absbits<T>(m);
      atomicMax(maxbits + rb + t, static_cast<unsigned long long>(m));
      if (m >= 0x7FF0000000000000ull) set_status(status, ST_NONFINITE);
    }
  }
}

// ------------------------------------------------------------------ norm scan
// Norm-based Scheme II scaling: e_r with ||x_r||_2 < 2^e_r, computed exactly
// so that the value does not depend on the summation order.  With E the
// frexp exponent of the row maximum and y = x 2^-E (|y| < 1), every square
// is rounded UP to an integer number of units 2^-64, the integers are summed
// (order-free, 128 bits), and e = E + ceil((bitlen(S) - 64) / 2).
// The value is below 2^64 (y^2 < 1): M^2 (106 bits at most) shifted right
// by s = -sh >= 1 with a sticky round-up, in 64-bit halves; a left shift
// (sh >= 0) only occurs for rows of subnormal numbers.
__device__ __forceinline__ uint64_t sq_ceil64(uint64_t bits, int Emax) {
  const uint64_t ab = bits & 0x7FFFFFFFFFFFFFFFull;
  if (ab == 0) return 0;
  const int ef = static_cast<int>(ab >> 52);
  uint64_t M = ab & ((uint64_t{1} << 52) - 1);
  int q;  // |x| = M 2^q
  if (ef == 0) {
    q = -1074;
  } else {
    M |= uint64_t{1} << 52;
    q = ef - 1075;
  }
  const uint64_t lo = M * M, hi = __umul64hi(M, M);
  const int sh = 2 * (q - Emax) + 64;
  if (sh >= 0) return lo << sh;  // then M^2 2^sh < 2^64, so hi = 0 and lo << sh is exact
  const int s = -sh;
  if (s >= 128) return 1;
  uint64_t r, sticky;
  if (s >= 64) {
    const int t = s - 64;
    r = hi >> t;
    sticky = lo | (t ? (hi << (64 - t)) : 0ull);
  } else {
    r = (hi << (64 - s)) | (lo >> s);
    sticky = lo << (64 - s);
  }
  return r + (sticky != 0 ? 1ull : 0ull);
}

// Exact 128-bit atomic add on (lo, hi) words.
__device__ __forceinline__ void atomic_add_u128(unsigned long long* acc, unsigned __int128 v) {
  const unsigned long long lo = static_cast<unsigned long long>(v), hi = static_cast<unsigned long long>(v >> 64);
  const unsigned long long old = atomicAdd(acc, lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(acc + 1, hi + carry);
}

__device__ __forceinline__ unsigned __int128 shfl_add_u128(unsigned __int128 v) {
  for (int o = 16; o; o >>= 1) {
    const unsigned long long lo = __shfl_xor_sync(0xffffffffu, static_cast<unsigned long long>(v), o);
    const unsigned long long hi = __shfl_xor_sync(0xffffffffu, static_cast<unsigned long long>(v >> 64), o);
    v += (static_cast<unsigned __int128>(hi) << 64) | lo;
  }
  return v;
}

// Same launch shapes as scan_kernel; acc: 2 words per row, zeroed first.
template <typename T, bool KCONTIG>
__global__ void norm_kernel(const T* __restrict__ X, int64_t ld, int64_t rows, int64_t k, int cw, int64_t seg,
                            const unsigned long long* __restrict__ maxbits, unsigned long long* __restrict__ acc) {
  if (KCONTIG) {
    const int lane = threadIdx.x & 31;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const uint64_t mb = maxbits[r];
    if (mb == 0 || mb >= 0x7FF0000000000000ull) return;  // zero row / non-finite (flagged by the scan)
    const int Emax = frexp_exp_bits(mb);
    const int64_t len = k * cw;
    const int64_t h0 = static_cast<int64_t>(blockIdx.y) * seg;
    const int64_t h1 = h0 + seg < len ? h0 + seg : len;
    const T* row = X + r * ld * cw;
    unsigned __int128 sum = 0;
#pragma unroll 4
    for (int64_t h = h0 + lane; h < h1; h += 32) sum += sq_ceil64(load_bits(row + h), Emax);
    sum = shfl_add_u128(sum);
    if (lane == 0 && sum) atomic_add_u128(acc + 2 * r, sum);
  } else {
    const int64_t r = static_cast<int64_t>(blockIdx.x) * 32 + threadIdx.x;
    const int64_t h0 = static_cast<int64_t>(blockIdx.y) * seg;
    const int64_t h1 = h0 + seg < k ? h0 + seg : k;
    if (r >= rows) return;
    const uint64_t mb = maxbits[r];
    if (mb == 0 || mb >= 0x7FF0000000000000ull) return;
    const int Emax = frexp_exp_bits(mb);
    unsigned __int128 sum = 0;
#pragma unroll 4
    for (int64_t h = h0 + threadIdx.y; h < h1; h += blockDim.y) {
      const T* p = X + (h * ld + r) * cw;
      sum += sq_ceil64(load_bits(p), Emax);
      if (cw == 2) sum += sq_ceil64(load_bits(p + 1), Emax);
    }
    if (sum) atomic_add_u128(acc + 2 * r, sum);
  }
}

__global__ void norm_finish_kernel(int64_t rows, const unsigned long long* __restrict__ maxbits,
                                   const unsigned long long* __restrict__ acc, int32_t* __restrict__ E) {
  const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const unsigned long long lo = acc[2 * r], hi = acc[2 * r + 1];
  const uint64_t mb = maxbits[r];
  if ((lo | hi) == 0 || mb >= 0x7FF0000000000000ull) {
    E[r] = 0;
    return;
  }
  const int L = hi ? 128 - __clzll(static_cast<long long>(hi)) : 64 - __clzll(static_cast<long long>(lo));
  const int d = L - 64;
  const int ep = d >= 0 ? (d + 1) / 2 : -((-d) / 2);  // ceil(d / 2)
  E[r] = frexp_exp_bits(mb) + ep;
}

// ------------------------------------------------------------------ split I
// K-contiguous source: one warp per (row, group of four 32-wide K-chunks);
// lane l handles h = 4l .. 4l+3 of the group and writes one 4-byte word per
// slice (lanes 8c .. 8c+7 fill the 32-byte block of chunk c).
template <typename T, int P, bool F8>
__global__ void split_I_kcontig(const T* __restrict__ X, int64_t ld, int64_t rows, int64_t k,
                                int64_t rows_pad, int64_t nchunks,
                                const unsigned long long* __restrict__ maxbits,
                                int8_t* __restrict__ hat, int32_t* __restrict__ E_out, bool vec) {
  const int lane = threadIdx.x & 31;
  const int64_t ngroups = (nchunks + 3) / 4;
  const int64_t w = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= rows_pad * ngroups) return;
  const int64_t r = w / ngroups, g = w % ngroups;
  const int64_t c = g * 4 + (lane >> 3);  // chunk of this lane
  if (c >= nchunks) return;
  const int64_t h0 = c * 32 + (lane & 7) * 4;
  const int E = exp_from_maxbits(maxbits, r, rows);
  uint64_t bits[4];
  load4_kcontig(X + (r < rows ? r : 0) * ld, h0, k, r < rows, vec, bits);
  uint32_t word[P];
  pack4<P, F8>(bits, E, word);
  uint8_t* row = reinterpret_cast<uint8_t*>(hat) + r * (nchunks * 32 * P);
#pragma unroll
  for (int t = 0; t < P; ++t)
    *reinterpret_cast<uint32_t*>(row + (c * P + t) * 32 + (lane & 7) * 4) = word[t];
  if (c == 0 && lane == 0 && r < rows && E_out) E_out[r] = E;
}

// K-strided source (element (r, h) at X[h*ld + r]): a block of 256 threads
// takes 32 vectors x 128 K-elements at a time, reads them coalesced along r
// into shared memory, then works like the K-contiguous kernel (warp w:
// vectors w, w+8, w+16, w+24; lane l: elements 4l .. 4l+3).  Element h of a
// vector is kept at column (h mod 4) * 33 + h / 4 and vectors are 133 words
// apart, so both the column-wise fill and the lane-wise reads are free of
// bank conflicts.
template <typename T, int P, bool F8>
__global__ void __launch_bounds__(256) split_I_kstrided(const T* __restrict__ X, int64_t ld, int64_t rows, int64_t k,
                                                        int64_t rows_pad, int64_t nchunks,
                                                        const unsigned long long* __restrict__ maxbits,
                                                        int8_t* __restrict__ hat, int32_t* __restrict__ E_out,
                                                        bool vec) {
  __shared__ uint64_t tile[32][133];
  const int64_t g = blockIdx.x;  // group of 4 chunks
  const int64_t hbase = g * 128;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c = g * 4 + (lane >> 3);
  for (int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32; r0 < rows_pad;
       r0 += static_cast<int64_t>(gridDim.y) * 32) {
    __syncthreads();  // the previous row block is done with the tile
    fill_tile_strided(tile, X, ld, rows, k, r0, hbase, vec);
    __syncthreads();
    for (int rl = warp; rl < 32; rl += 8) {
      const int64_t r = r0 + rl;
      if (r >= rows_pad || c >= nchunks) continue;
      const int E = exp_from_maxbits(maxbits, r, rows);
      uint64_t bits[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) bits[q] = tile[rl][q * 33 + lane];
      uint32_t word[P];
      pack4<P, F8>(bits, E, word);
      uint8_t* row = reinterpret_cast<uint8_t*>(hat) + r * (nchunks * 32 * P);
#pragma unroll
      for (int t = 0; t < P; ++t)
        *reinterpret_cast<uint32_t*>(row + (c * P + t) * 32 + (lane & 7) * 4) = word[t];
      if (c == 0 && lane == 0 && r < rows && E_out) E_out[r] = E;
    }
  }
}

// ------------------------------------------------------------------ split II
// The 16-bit digits of |a'| = trunc(|a| 2^shift) (|a'| < 2^80, so five
// digits), negated for a negative element: a' = sum_j d_j 2^(16 j).
__device__ __forceinline__ void digits16(uint64_t bits, int shift, int* d) {
  const ScaledInt s = scaled_trunc_bits(bits, shift);
  // s.mag 2^s.lsh = |a'| < 2^80 (the row exponent bounds every element), so s.lsh < 80
  const unsigned __int128 v = static_cast<unsigned __int128>(s.mag) << s.lsh;
  const uint64_t lo = static_cast<uint64_t>(v);
  const uint32_t hi = static_cast<uint32_t>(v >> 64);
  const int sg = (bits >> 63) ? -1 : 1;
  d[0] = sg * static_cast<int>(lo & 0xFFFFu);
  d[1] = sg * static_cast<int>((lo >> 16) & 0xFFFFu);
  d[2] = sg * static_cast<int>((lo >> 32) & 0xFFFFu);
  d[3] = sg * static_cast<int>(lo >> 48);
  d[4] = sg * static_cast<int>(hi & 0xFFFFu);
}

// Symmetric residue of a' modulo m_l from its digits.  t = sum_j d_j c_j
// with c_j the symmetric residue of 2^(16 j) (|c_j| <= 128) satisfies
// |t| <= 65535 (1 + 4 * 128) < 2^25.1.  q = floor(RN(RN(t) / m + off / m)) is
// floor((t + off) / m) or one off (the three roundings move the quotient,
// which is below 2^18, by less than 0.05), so r = t - q m lies in
// [-off - m, 2m - off) and one correction each way puts it in
// [-off, m - 1 - off].
__device__ __forceinline__ int sym_residue(const int* d, const ModTables& mt, int l) {
  int t = d[0];
#pragma unroll
  for (int j = 1; j < kResDigits; ++j) t += d[j] * mt.pow16[l][j];
  const int m = static_cast<int>(mt.mods[l]), off = mt.off[l];
  const int q = __float2int_rd(__fmaf_rn(__int2float_rn(t), mt.inv[l], mt.offinv[l]));
  int r = t - q * m;
  if (r < -off) r += m;
  if (r >= m - off) r -= m;
  return r;
}

// The same in binary32 for the bf16 planes: the ND lowest 14-bit digits of
// |a'|, negated for a negative element (|a'| < 2^b, so ND = ceil(b / 14),
// rounded up to 2, 4 or 6, covers it; six cover 2^84).  Every partial sum of
// t = sum_j d_j c_j is an integer with |t| <= 16383 (1 + 5 * 128) < 2^24, so
// the FMA chain is exact, and sym_residue_f below takes the symmetric
// residue of t on the FP32 pipe without a correction step.
template <int ND>
__device__ __forceinline__ void digits14f(uint64_t bits, int shift, float* d) {
  const ScaledInt s = scaled_trunc_bits(bits, shift);
  // a' = 0 keeps its digits +0 (no sign), so that no residue below comes out
  // as -0 (whose bf16 pattern is not that of the integer 0)
  const uint32_t sg = s.mag != 0 ? static_cast<uint32_t>(bits >> 63) << 31 : 0u;
  uint32_t dg[ND];
  if constexpr (ND <= 4) {  // |a'| < 2^(14 ND) <= 2^56: one 64-bit word holds it
    const uint64_t v = s.lsh < 64 ? s.mag << s.lsh : 0ull;
#pragma unroll
    for (int j = 0; j < ND; ++j) dg[j] = static_cast<uint32_t>(v >> (14 * j)) & 0x3FFFu;
  } else {
    // s.mag 2^s.lsh = |a'| < 2^80 (the row exponent bounds every element), so s.lsh < 80
    const unsigned __int128 v = static_cast<unsigned __int128>(s.mag) << s.lsh;
    const uint64_t lo = static_cast<uint64_t>(v);
    const uint64_t hi = static_cast<uint64_t>(v >> 64);
    dg[0] = static_cast<uint32_t>(lo & 0x3FFFu);
    dg[1] = static_cast<uint32_t>((lo >> 14) & 0x3FFFu);
    dg[2] = static_cast<uint32_t>((lo >> 28) & 0x3FFFu);
    dg[3] = static_cast<uint32_t>((lo >> 42) & 0x3FFFu);
    dg[4] = static_cast<uint32_t>(((lo >> 56) | (hi << 8)) & 0x3FFFu);
    dg[5] = static_cast<uint32_t>((hi >> 6) & 0x3FFFu);
  }
#pragma unroll
  for (int j = 0; j < ND; ++j)  // 2^23 + d has d in its low mantissa bits; the sign by bit
    d[j] = __uint_as_float(__float_as_uint(__uint_as_float(0x4B000000u | dg[j]) - 8388608.0f) | sg);
}

// The quotient needs no correction: with c = RN((off + 1/2) / m) and
// inv = RN(1/m), floor(t inv + c) (the exact value; the FMA rounds it
// downward, which never crosses the integer below it) equals
// floor((t + off) / m) for every integer |t| <= 16383 (1 + sum_j>=1 |c_j|)
// -- the range of t for the digit count ND <= 6 -- and every modulus of the
// list.  The half in the offset puts (t + off + 1/2) / m at least 1/(2m)
// from the integers, and the roundings of inv and c move t inv + c by at
// most |t| 2^-32 + 2^-25, below 1/(2m) for ND <= 4 (|t| < 2^22.6); the
// claim is checked exhaustively over the whole range, ND = 6 included, by
// the host tests.
// So r = t - q m is the symmetric residue in [-off, m - 1 - off] at once.
// No step produces -0 from the +0 digits of a' = 0 (t = +0, q = 0).
template <int ND>
__device__ __forceinline__ float sym_residue_f(const float* d, const ModTables& mt, int l) {
  float t = d[0];
#pragma unroll
  for (int j = 1; j < ND; ++j) t = __fmaf_rn(d[j], mt.pow14f[l][j], t);
  const float q = floorf(__fmaf_rd(t, mt.inv[l], mt.offhinv[l]));
  return __fmaf_rn(-q, mt.mf[l], t);
}

__device__ __forceinline__ uint32_t pack_bytes(int r0, int r1, int r2, int r3) {
  const uint32_t lo = __byte_perm(static_cast<uint32_t>(r0), static_cast<uint32_t>(r1), 0x0040u);
  const uint32_t hi = __byte_perm(static_cast<uint32_t>(r2), static_cast<uint32_t>(r3), 0x0040u);
  return __byte_perm(lo, hi, 0x5410u);
}

// Four residues as bf16 (exact: |r| <= 128 has at most 8 significant bits,
// so the upper half of the binary32 value is the bf16 value).
__device__ __forceinline__ uint2 pack_bf16(int r0, int r1, int r2, int r3) {
  const uint32_t f0 = __float_as_uint(__int2float_rn(r0)), f1 = __float_as_uint(__int2float_rn(r1));
  const uint32_t f2 = __float_as_uint(__int2float_rn(r2)), f3 = __float_as_uint(__int2float_rn(r3));
  return make_uint2(__byte_perm(f0, f1, 0x7632u), __byte_perm(f2, f3, 0x7632u));
}

template <bool BF>
__device__ __forceinline__ void store4(int8_t* p, int r0, int r1, int r2, int r3) {
  if (BF)
    *reinterpret_cast<uint2*>(p) = pack_bf16(r0, r1, r2, r3);
  else
    *reinterpret_cast<uint32_t*>(p) = pack_bytes(r0, r1, r2, r3);
}

// The residues of four consecutive K elements of one vector, one store per
// plane (INT8: four bytes, byte q = element q; BF: four bf16 values): real
// (cw = 1) one plane per modulus; complex three (re, im, re + im).
// `re`/`im` hold the binary64 bits of the elements; `base` is the address
// of the first element in plane 0, `plane` the plane stride in bytes.  The
// modulus loop is unrolled so that the table entries are kernel-parameter
// operands.
// Four binary32 residues (integers |r| <= 128, never -0) as bf16.
__device__ __forceinline__ void store4f(int8_t* p, float r0, float r1, float r2, float r3) {
  const uint32_t f0 = __float_as_uint(r0), f1 = __float_as_uint(r1);
  const uint32_t f2 = __float_as_uint(r2), f3 = __float_as_uint(r3);
  *reinterpret_cast<uint2*>(p) = make_uint2(__byte_perm(f0, f1, 0x7632u), __byte_perm(f2, f3, 0x7632u));
}

template <int CW, bool BF, int ND>
__device__ __forceinline__ void residues4(const ModTables& mt, int nm, int shift, const uint64_t* re,
                                          const uint64_t* im, int64_t plane, int8_t* base) {
  if constexpr (BF) {  // bf16 planes: the binary32 form
    float dr[4][ND], di[CW == 2 ? 4 : 1][ND];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      digits14f<ND>(re[q], shift, dr[q]);
      if (CW == 2) digits14f<ND>(im[q], shift, di[q]);
    }
#pragma unroll
    for (int l = 0; l < kMaxModuli; ++l) {
      if (l >= nm) break;
      float rr[4], ri[4], rs[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        rr[q] = sym_residue_f<ND>(dr[q], mt, l);
        if (CW == 2) {
          ri[q] = sym_residue_f<ND>(di[q], mt, l);
          const float m = mt.mf[l], off = mt.offf[l];
          float v = rr[q] + ri[q];
          if (v < -off) v += m;
          if (v >= m - off) v -= m;
          rs[q] = v;
        }
      }
      store4f(base + static_cast<int64_t>(l) * plane, rr[0], rr[1], rr[2], rr[3]);
      if (CW == 2) {
        store4f(base + static_cast<int64_t>(nm + l) * plane, ri[0], ri[1], ri[2], ri[3]);
        store4f(base + static_cast<int64_t>(2 * nm + l) * plane, rs[0], rs[1], rs[2], rs[3]);
      }
    }
  } else {
    int dr[4][kResDigits], di[4][kResDigits];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      digits16(re[q], shift, dr[q]);
      if (CW == 2) digits16(im[q], shift, di[q]);
    }
#pragma unroll
    for (int l = 0; l < kMaxModuli; ++l) {
      if (l >= nm) break;
      int rr[4], ri[4], rs[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        rr[q] = sym_residue(dr[q], mt, l);
        if (CW == 2) {
          ri[q] = sym_residue(di[q], mt, l);
          const int m = static_cast<int>(mt.mods[l]), off = mt.off[l];
          int v = rr[q] + ri[q];
          if (v < -off) v += m;
          if (v >= m - off) v -= m;
          rs[q] = v;
        }
      }
      store4<BF>(base + static_cast<int64_t>(l) * plane, rr[0], rr[1], rr[2], rr[3]);
      if (CW == 2) {
        store4<BF>(base + static_cast<int64_t>(nm + l) * plane, ri[0], ri[1], ri[2], ri[3]);
        store4<BF>(base + static_cast<int64_t>(2 * nm + l) * plane, rs[0], rs[1], rs[2], rs[3]);
      }
    }
  }
}

// Scheme II split.  Planes: set q, modulus l at element
// ((q*nm + l)*rows_pad + r)*kpad + h of `res` (set = 0 for real; 0, 1, 2 =
// re, im, re + im for complex); elements are INT8, or bf16 (BF) for the
// tcgen05 kernel.  Row exponent: of the maximum (worst-case
// scaling) or of the 2-norm (Ein).  K-contiguous sources: one warp per
// (vector, 128 K-elements), lane l takes elements 4l .. 4l+3 and writes one
// word per plane; strided sources go through a shared-memory tile of 32
// vectors (16 for complex) x 128 elements as in the Scheme I split.
template <typename T, int CW, bool BF, int ND>
__global__ void split_II_kcontig(const T* __restrict__ X, int64_t ld, int64_t rows, int64_t k, int64_t rows_pad,
                                 int64_t kpad, int nm, int b, const __grid_constant__ ModTables mt,
                                 const unsigned long long* __restrict__ maxbits, const int32_t* __restrict__ Ein,
                                 int8_t* __restrict__ res, int32_t* __restrict__ E_out, bool vec) {
  const int lane = threadIdx.x & 31;
  const int64_t ngroups = kpad / 128;
  const int64_t w = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= rows_pad * ngroups) return;
  const int64_t r = w / ngroups, h0 = (w % ngroups) * 128 + lane * 4;
  const int E = Ein ? (r < rows ? Ein[r] : 0) : exp_from_maxbits(maxbits, r, rows);
  uint64_t re[4], im[4];
  if constexpr (CW == 1) {
    load4_kcontig(X + (r < rows ? r : 0) * ld, h0, k, r < rows, vec, re);
#pragma unroll
    for (int q = 0; q < 4; ++q) im[q] = 0ull;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool valid = r < rows && h0 + q < k;
      const T* p = X + (r * ld + h0 + q) * CW;
      re[q] = valid ? load_bits(p) : 0ull;
      im[q] = valid ? load_bits(p + 1) : 0ull;
    }
  }
  residues4<CW, BF, ND>(mt, nm, b - E, re, im, rows_pad * kpad * (BF ? 2 : 1), res + (r * kpad + h0) * (BF ? 2 : 1));
  if (h0 == 0 && r < rows && E_out) E_out[r] = E;
}

template <typename T, int CW, bool BF, int ND>
__global__ void __launch_bounds__(256) split_II_kstrided(const T* __restrict__ X, int64_t ld, int64_t rows, int64_t k,
                                                         int64_t rows_pad, int64_t kpad, int nm, int b,
                                                         const __grid_constant__ ModTables mt,
                                                         const unsigned long long* __restrict__ maxbits,
                                                         const int32_t* __restrict__ Ein, int8_t* __restrict__ res,
                                                         int32_t* __restrict__ E_out, bool vec) {
  constexpr int TR = CW == 2 ? 16 : 32;  // vectors per tile (two tiles for complex)
  __shared__ uint64_t tre[TR][133];
  __shared__ uint64_t tim[CW == 2 ? TR : 1][CW == 2 ? 133 : 1];
  const int64_t hbase = static_cast<int64_t>(blockIdx.x) * 128;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t r0 = static_cast<int64_t>(blockIdx.y) * TR; r0 < rows_pad;
       r0 += static_cast<int64_t>(gridDim.y) * TR) {
    __syncthreads();  // the previous row block is done with the tiles
    if constexpr (CW == 1) {
      fill_tile_strided(tre, X, ld, rows, k, r0, hbase, vec);
    } else {
      for (int i = threadIdx.x; i < TR * 128; i += 256) {
        const int rl = i % TR, hl = i / TR;
        const int64_t r = r0 + rl, h = hbase + hl;
        const bool valid = r < rows && h < k;
        const T* p = X + (h * ld + r) * CW;
        const int col = (hl & 3) * 33 + (hl >> 2);
        tre[rl][col] = valid ? load_bits(p) : 0ull;
        tim[rl][col] = valid ? load_bits(p + 1) : 0ull;
      }
    }
    __syncthreads();
    for (int rl = warp; rl < TR; rl += 8) {
      const int64_t r = r0 + rl;
      if (r >= rows_pad) continue;
      const int E = Ein ? (r < rows ? Ein[r] : 0) : exp_from_maxbits(maxbits, r, rows);
      uint64_t re[4], im[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        re[q] = tre[rl][q * 33 + lane];
        im[q] = CW == 2 ? tim[rl][q * 33 + lane] : 0ull;
      }
      const int64_t h0 = hbase + lane * 4;
      residues4<CW, BF, ND>(mt, nm, b - E, re, im, rows_pad * kpad * (BF ? 2 : 1), res + (r * kpad + h0) * (BF ? 2 : 1));
      if (h0 == 0 && r < rows && E_out) E_out[r] = E;
    }
  }
}

// ------------------------------------------------------------------ launchers
// K segment (elements of a vector per block) of the scan and norm kernels:
// `seg0` (2048 along K-contiguous rows, 256 down strided columns), halved
// while the grid would hold fewer than four blocks per SM -- small operands
// then still have enough loads in flight -- down to `seg_min`, and doubled
// while the segment count exceeds the grid's y limit.
static int64_t scan_seg(int64_t vec_blocks, int64_t len, int64_t seg0, int64_t seg_min) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t seg = seg0;
  while (seg > seg_min && vec_blocks * ((len + seg - 1) / seg) < 4 * static_cast<int64_t>(sms)) seg >>= 1;
  while ((len + seg - 1) / seg > 65535) seg <<= 1;
  return seg;
}

template <typename T>
void launch_scan(const T* X, int64_t ld, bool kcontig, int64_t rows, int64_t k, int cw,
                 unsigned long long* maxbits, int* status, cudaStream_t st) {
  cudaMemsetAsync(maxbits, 0, sizeof(unsigned long long) * (rows > 0 ? rows : 1), st);
  if (rows == 0 || k == 0) return;
  // 16-byte loads when every vector starts on a 16-byte boundary
  const bool vec = (reinterpret_cast<uintptr_t>(X) & 15u) == 0 &&
                   (static_cast<uint64_t>(ld) * cw * sizeof(T)) % 16 == 0;
  if (kcontig) {
    const int64_t len = k * cw, rb = (rows + 7) / 8, seg = scan_seg(rb, len, 2048, 256);
    dim3 grid(static_cast<unsigned>(rb), static_cast<unsigned>((len + seg - 1) / seg));
    if (vec)
      scan_vec_kernel<T, true><<<grid, 256, 0, st>>>(X, ld, rows, k, cw, seg, maxbits, status);
    else
      scan_kernel<T, true><<<grid, 256, 0, st>>>(X, ld, rows, k, cw, seg, maxbits, status);
  } else if (vec) {
    const int64_t per_block = 32 * static_cast<int64_t>(16 / sizeof(T)) / cw;
    const int64_t rb = (rows + per_block - 1) / per_block, seg = scan_seg(rb, k, 256, 32);
    dim3 grid(static_cast<unsigned>(rb), static_cast<unsigned>((k + seg - 1) / seg));
    scan_vec_kernel<T, false><<<grid, dim3(32, 8), 0, st>>>(X, ld, rows, k, cw, seg, maxbits, status);
  } else {
    const int64_t rb = (rows + 31) / 32, seg = scan_seg(rb, k, 256, 32);
    dim3 grid(static_cast<unsigned>(rb), static_cast<unsigned>((k + seg - 1) / seg));
    scan_kernel<T, false><<<grid, dim3(32, 8), 0, st>>>(X, ld, rows, k, cw, seg, maxbits, status);
  }
}
template void launch_scan<double>(const double*, int64_t, bool, int64_t, int64_t, int,
                                  unsigned long long*, int*, cudaStream_t);
template void launch_scan<float>(const float*, int64_t, bool, int64_t, int64_t, int,
                                 unsigned long long*, int*, cudaStream_t);

template <typename T, int P, bool F8>
static void launch_split_I_p(const T* X, int64_t ld, bool kcontig, int64_t rows, int64_t k,
                             const unsigned long long* maxbits, int8_t* hat, int32_t* E,
                             cudaStream_t st) {
  int64_t rows_pad = split_rows(rows), nchunks = split_cols_I(k, 1) / 32;
  if (rows_pad == 0 || nchunks == 0) return;
  if (kcontig) {
    int64_t warps = rows_pad * ((nchunks + 3) / 4);
    int64_t blocks = (warps + 7) / 8;
    split_I_kcontig<T, P, F8><<<static_cast<unsigned>(blocks), 256, 0, st>>>(X, ld, rows, k, rows_pad,
                                                                             nchunks, maxbits, hat, E,
                                                                             vec16_ok(X, ld));
  } else {
    const int64_t rb = rows_pad / 32;
    dim3 grid(static_cast<unsigned>((nchunks + 3) / 4), static_cast<unsigned>(rb < 65535 ? rb : 65535));
    split_I_kstrided<T, P, F8><<<grid, 256, 0, st>>>(X, ld, rows, k, rows_pad, nchunks, maxbits, hat, E,
                                                     vec16_ok(X, ld));
  }
}

template <typename T>
void launch_split_I(const T* X, int64_t ld, bool kcontig, int64_t rows, int64_t k, int p,
                    const unsigned long long* maxbits, int8_t* hat, int32_t* E, cudaStream_t st, bool f8) {
  switch (p) {
#define EMU_CASE(PP)                                                                         \
  case PP:                                                                                   \
    if (f8)                                                                                  \
      launch_split_I_p<T, PP, true>(X, ld, kcontig, rows, k, maxbits, hat, E, st);          \
    else                                                                                     \
      launch_split_I_p<T, PP, false>(X, ld, kcontig, rows, k, maxbits, hat, E, st);         \
    break;
    EMU_CASE(1) EMU_CASE(2) EMU_CASE(3) EMU_CASE(4) EMU_CASE(5) EMU_CASE(6)
    EMU_CASE(7) EMU_CASE(8) EMU_CASE(9) EMU_CASE(10) EMU_CASE(11) EMU_CASE(12)
#undef EMU_CASE
    default:
      break;
  }
}
template void launch_split_I<double>(const double*, int64_t, bool, int64_t, int64_t, int,
                                     const unsigned long long*, int8_t*, int32_t*, cudaStream_t, bool);
template void launch_split_I<float>(const float*, int64_t, bool, int64_t, int64_t, int,
                                    const unsigned long long*, int8_t*, int32_t*, cudaStream_t, bool);

template <typename T>
void launch_split_II(const T* X, int64_t ld, bool kcontig, int64_t rows, int64_t k, int nm, int b,
                     int cw, const ModTables& tabs, const unsigned long long* maxbits, int8_t* res,
                     int32_t* E, cudaStream_t st, const int32_t* Ein, bool bf16) {
  const int64_t rows_pad = split_rows(rows), kpad = split_cols_II(k);
  if (rows_pad == 0 || kpad == 0) return;
  // 14-bit digits that hold |a'| < 2^b (bf16 planes; the INT8 form has its own)
  const int nd = b <= 28 ? 2 : b <= 56 ? 4 : 6;
  const bool vec = cw == 1 && vec16_ok(X, ld);
#define EMU_SPLIT_II_ARGS X, ld, rows, k, rows_pad, kpad, nm, b, tabs, maxbits, Ein, res, E, vec
#define EMU_SPLIT_II(KERNEL, GRID, CW)                                             \
  (!bf16      ? KERNEL<T, CW, false, 6><<<GRID, 256, 0, st>>>(EMU_SPLIT_II_ARGS) \
   : nd == 2 ? KERNEL<T, CW, true, 2><<<GRID, 256, 0, st>>>(EMU_SPLIT_II_ARGS)  \
   : nd == 4 ? KERNEL<T, CW, true, 4><<<GRID, 256, 0, st>>>(EMU_SPLIT_II_ARGS)  \
             : KERNEL<T, CW, true, 6><<<GRID, 256, 0, st>>>(EMU_SPLIT_II_ARGS))
  if (kcontig) {
    const int64_t warps = rows_pad * (kpad / 128);
    const unsigned blocks = static_cast<unsigned>((warps + 7) / 8);
    if (cw == 2)
      EMU_SPLIT_II(split_II_kcontig, blocks, 2);
    else
      EMU_SPLIT_II(split_II_kcontig, blocks, 1);
  } else {
    const int64_t rb = rows_pad / (cw == 2 ? 16 : 32);
    dim3 grid(static_cast<unsigned>(kpad / 128), static_cast<unsigned>(rb < 65535 ? rb : 65535));
    if (cw == 2)
      EMU_SPLIT_II(split_II_kstrided, grid, 2);
    else
      EMU_SPLIT_II(split_II_kstrided, grid, 1);
  }
#undef EMU_SPLIT_II
#undef EMU_SPLIT_II_ARGS
}

template <typename T>
void launch_norm(const T* X, int64_t ld, bool kcontig, int64_t rows, int64_t k, int cw,
                 const unsigned long long* maxbits, unsigned long long* acc, int32_t* E, cudaStream_t st) {
  if (rows == 0) return;
  cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 2 * rows, st);
  if (k > 0) {
    if (kcontig) {
      const int64_t len = k * cw, rb = (rows + 7) / 8, seg = scan_seg(rb, len, 2048, 256);
      dim3 grid(static_cast<unsigned>(rb), static_cast<unsigned>((len + seg - 1) / seg));
      norm_kernel<T, true><<<grid, 256, 0, st>>>(X, ld, rows, k, cw, seg, maxbits, acc);
    } else {
      const int64_t rb = (rows + 31) / 32, seg = scan_seg(rb, k, 256, 32);
      dim3 grid(static_cast<unsigned>(rb), static_cast<unsigned>((k + seg - 1) / seg));
      norm_kernel<T, false><<<grid, dim3(32, 8), 0, st>>>(X, ld, rows, k, cw, seg, maxbits, acc);
    }
  }
  norm_finish_kernel<<<static_cast<unsigned>((rows + 255) / 256), 256, 0, st>>>(rows, maxbits, acc, E);
}
template void launch_norm<double>(const double*, int64_t, bool, int64_t, int64_t, int, const unsigned long long*,
                                  unsigned long long*, int32_t*, cudaStream_t);
template void launch_norm<float>(const float*, int64_t, bool, int64_t, int64_t, int, const unsigned long long*,
                                 unsigned long long*, int32_t*, cudaStream_t);

template void launch_split_II<double>(const double*, int64_t, bool, int64_t, int64_t, int, int, int,
                                      const ModTables&, const unsigned long long*, int8_t*, int32_t*,
                                      cudaStream_t, const int32_t*, bool);
template void launch_split_II<float>(const float*, int64_t, bool, int64_t, int64_t, int, int, int,
                                     const ModTables&, const unsigned long long*, int8_t*, int32_t*,
                                     cudaStream_t, const int32_t*, bool);

}  // namespace emu
