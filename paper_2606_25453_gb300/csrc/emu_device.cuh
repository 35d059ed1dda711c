// emu_device.cuh -- device-side building blocks for the sm_103a kernels:
// inline-PTX wrappers (mbarrier, TMA, ldmatrix, INT8 mma.sync), bounded
// waits, the device status word, and exact integer <-> binary64 helpers
// written from the IEEE-754 bit layout.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace emu {

// ---------------------------------------------------------------- status word
enum : int { ST_NONFINITE = 1, ST_TIMEOUT = 2 };

__device__ __forceinline__ void set_status(int* status, int bit) {
  if (status) atomicOr(status, bit);
}

// Bounded waits give up after ~1 s of GPU time (clock64 at <= 2.1 GHz).
constexpr long long kWaitCycles = 2000000000LL;

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of the phase with the given parity (never suspends).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; false after `limit`
// clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_prefetch_desc(const void* desc) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(desc)) : "memory");
}

// 2D tiled load global -> shared, completion counted on `bar` in bytes.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const void* desc, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(desc)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// ---------------------------------------------------------------- ldmatrix / mma
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// D = A*B + D, m16n8k32, A row / B col, int32 accumulate (wraps mod 2^32;
// the callers keep every partial sum inside int32).
// SA / SB: true = signed bytes (s8), false = unsigned bytes (u8).
template <bool SA, bool SB>
__device__ __forceinline__ void mma_i8(int32_t* d, const uint32_t* a, const uint32_t* b);

#define EMU_MMA_I8(SA, SB, TA, TB)                                                                \
  template <>                                                                                     \
  __device__ __forceinline__ void mma_i8<SA, SB>(int32_t * d, const uint32_t* a, const uint32_t* b) { \
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32." TA "." TB ".s32"                      \
                 " {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"                          \
                 : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])                                 \
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));           \
  }
EMU_MMA_I8(true, true, "s8", "s8")
EMU_MMA_I8(true, false, "s8", "u8")
EMU_MMA_I8(false, true, "u8", "s8")
EMU_MMA_I8(false, false, "u8", "u8")
#undef EMU_MMA_I8

// D = A*B + D, m16n8k32, E4M3 x E4M3 -> FP32.  The library only feeds it
// integers |d| <= 16 and keeps every partial sum within 2^24, where FP32
// accumulation is exact.
__device__ __forceinline__ void mma_e4m3(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32"
               " {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// E4M3 byte of an integer v with |v| <= 16 (exact): sign, exponent
// floor(log2 |v|) + 7, three mantissa bits.
__device__ __forceinline__ uint32_t e4m3_of_int(int v) {
  uint32_t a = static_cast<uint32_t>(v < 0 ? -v : v);
  if (a == 0) return 0u;
  int e = 31 - __clz(static_cast<int>(a));
  uint32_t mant = ((a << 3) >> e) & 7u;
  return (v < 0 ? 0x80u : 0u) | (static_cast<uint32_t>(e + 7) << 3) | mant;
}

// Byte offset inside a [rows][32 B] block written by TMA with 32-byte
// swizzling: the 16-byte half `chunk` of row `row` is stored at
// chunk ^ ((row >> 2) & 1).
__device__ __forceinline__ uint32_t swz32(int row, int chunk) {
  return static_cast<uint32_t>(row * 32 + ((chunk ^ ((row >> 2) & 1)) << 4));
}

// ---------------------------------------------------------------- binary64 bits
__device__ __forceinline__ uint64_t dbits(double x) { return static_cast<uint64_t>(__double_as_longlong(x)); }
__device__ __forceinline__ double bitsd(uint64_t b) { return __longlong_as_double(static_cast<long long>(b)); }

// frexp exponent of a nonnegative finite value given its bits: smallest E
// with x < 2^E; 0 for x == 0.
__device__ __forceinline__ int frexp_exp_bits(uint64_t absbits) {
  if (absbits == 0) return 0;
  int be = static_cast<int>(absbits >> 52);
  if (be != 0) return be - 1022;
  // subnormal: x = mant * 2^-1074, mant < 2^52
  int len = 64 - __clzll(static_cast<long long>(absbits));
  return len - 1074;
}

// x = trunc(|a| * 2^shift) for finite a given by its bits, as (mag, lsh):
// the value is mag << lsh with mag < 2^53 (lsh >= 0 only when no bits drop).
struct ScaledInt {
  uint64_t mag;  // significand part after any right shift
  int lsh;       // remaining left shift (>= 0)
};
__device__ __forceinline__ ScaledInt scaled_trunc_bits(uint64_t bits, int shift) {
  uint64_t ab = bits & 0x7FFFFFFFFFFFFFFFull;
  ScaledInt r{0, 0};
  if (ab == 0) return r;
  int be = static_cast<int>(ab >> 52);
  uint64_t M = ab & 0x000FFFFFFFFFFFFFull;
  int e2;  // value = M * 2^e2
  if (be) {
    M |= 0x0010000000000000ull;
    e2 = be - 1075;
  } else {
    e2 = -1074;
  }
  int sh = e2 + shift;
  if (sh >= 0) {
    r.mag = M;
    r.lsh = sh;
  } else {
    r.mag = (-sh) < 64 ? (M >> (-sh)) : 0ull;
    r.lsh = 0;
  }
  return r;
}

// Round an unsigned 128-bit integer to binary64, nearest-even, from its bits.
__device__ __forceinline__ double u128_to_double_rn(unsigned __int128 u) {
  uint64_t hi = static_cast<uint64_t>(u >> 64), lo = static_cast<uint64_t>(u);
  if (hi == 0 && lo < (1ull << 53)) {  // exact: built from the bits (no FP64 instruction)
    if (lo == 0) return 0.0;
    const int Ls = 64 - __clzll(static_cast<long long>(lo));  // 1 .. 53 significant bits
    const uint64_t m = lo << (53 - Ls);                       // in [2^52, 2^53)
    return bitsd((static_cast<uint64_t>(Ls - 1 + 1023) << 52) | (m & 0x000FFFFFFFFFFFFFull));
  }
  int L = hi ? 128 - __clzll(static_cast<long long>(hi)) : 64 - __clzll(static_cast<long long>(lo));
  int drop = L - 53;  // >= 1
  uint64_t top = static_cast<uint64_t>(u >> drop);
  unsigned __int128 rest = u - (static_cast<unsigned __int128>(top) << drop);
  unsigned __int128 half = static_cast<unsigned __int128>(1) << (drop - 1);
  if (rest > half || (rest == half && (top & 1))) top += 1;
  int exp = drop;  // value = top * 2^exp, top in [2^52, 2^53]
  if (top == (1ull << 53)) {
    top >>= 1;
    exp += 1;
  }
  uint64_t bits = (static_cast<uint64_t>(exp + 52 + 1023) << 52) | (top & 0x000FFFFFFFFFFFFFull);
  return bitsd(bits);
}

// Signed 128-bit integer to binary64, nearest-even.
__device__ __forceinline__ double i128_to_double_rn(__int128 v) {
  bool neg = v < 0;
  unsigned __int128 u = neg ? static_cast<unsigned __int128>(0) - static_cast<unsigned __int128>(v)
                            : static_cast<unsigned __int128>(v);
  double r = u128_to_double_rn(u);
  return neg ? -r : r;
}

// x * 2^e with a single rounding (the CUDA math library's ldexp).
__device__ __forceinline__ double scale2(double x, int e) { return ldexp(x, e); }

// BLAS update with a fixed operation order: beta == 0 -> alpha*r, else
// fma(alpha, r, beta*c).  __dmul_rn keeps the product out of any FMA.
__device__ __forceinline__ double blas_update(double alpha, double r, double beta, double c) {
  if (beta == 0.0) return __dmul_rn(alpha, r);
  return __fma_rn(alpha, r, __dmul_rn(beta, c));
}

}  // namespace emu
