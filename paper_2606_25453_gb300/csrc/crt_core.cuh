// crt_core.cuh -- multi-word CRT accumulation and finish (Eq. 8 and the
// inverse scaling after it), shared by the Scheme II kernels.
#pragma once
#include "emu_internal.h"

namespace emu {

constexpr int kSL = kCrtLimbs + 1;  // CRT accumulator limbs (S < nm * 256 * P)

// S += w * r for a 5-limb w and r < 256.
__device__ __forceinline__ void crt_acc(uint32_t* S, const uint32_t* w, uint32_t r) {
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < kCrtLimbs; ++i) {
    c += static_cast<uint64_t>(w[i]) * r + S[i];
    S[i] = static_cast<uint32_t>(c);
    c >>= 32;
  }
  S[kCrtLimbs] += static_cast<uint32_t>(c);
}

// Round a nonnegative 5-limb integer to binary64, nearest-even.  Below
// 2^128 the four low limbs are rounded directly; otherwise the window of
// limbs 1..4 (>= 97 significant bits) plus a sticky bit for limb 0 has the
// same rounding, scaled back by 2^32 exactly.  Straight-line code: no limb
// is indexed at run time.
__device__ __forceinline__ double limbs_to_double_rn(const uint32_t* x) {
  if (x[4] == 0) {
    const unsigned __int128 u = (static_cast<unsigned __int128>(x[3]) << 96) |
                                (static_cast<unsigned __int128>(x[2]) << 64) |
                                (static_cast<unsigned __int128>(x[1]) << 32) | x[0];
    return u128_to_double_rn(u);
  }
  unsigned __int128 u = (static_cast<unsigned __int128>(x[4]) << 96) |
                        (static_cast<unsigned __int128>(x[3]) << 64) |
                        (static_cast<unsigned __int128>(x[2]) << 32) | x[1];
  if (x[0]) u |= 1;
  return __dmul_rn(u128_to_double_rn(u), 4294967296.0);  // exact power-of-two scaling
}

// Eq. (8) finish: S mod P, symmetric lift, binary64.
__device__ __forceinline__ double crt_finish(const uint32_t* S, const CrtTables& ct) {
  // quotient estimate q = floor(S / P) <= nm * 255, corrected exactly below
  double sd = 0.0;
#pragma unroll
  for (int i = kSL - 1; i >= 0; --i) sd = __fma_rn(sd, 4294967296.0, static_cast<double>(S[i]));
  int q = static_cast<int>(floor(__dmul_rn(sd, ct.invP)));
  if (q < 0) q = 0;
  // R = S - q * P (6 limbs, may go negative by < 2P)
  uint32_t R[kSL];
  {
    uint64_t mul = 0;
    int64_t br = 0;
#pragma unroll
    for (int i = 0; i < kSL; ++i) {
      uint64_t pi = i < kCrtLimbs ? ct.P[i] : 0u;
      mul += pi * static_cast<uint64_t>(q);
      int64_t d = static_cast<int64_t>(S[i]) - static_cast<int64_t>(static_cast<uint32_t>(mul)) - br;
      mul >>= 32;
      br = d < 0;
      R[i] = static_cast<uint32_t>(d + (br ? (1ll << 32) : 0));
    }
  }
  // fix up: while R < 0 add P; while R >= P subtract P (at most a few steps)
  for (int step = 0; step < 4; ++step) {
    if (static_cast<int32_t>(R[kSL - 1]) < 0) {  // negative (two's complement, 6 limbs)
      uint64_t c = 0;
#pragma unroll
      for (int i = 0; i < kSL; ++i) {
        c += static_cast<uint64_t>(R[i]) + (i < kCrtLimbs ? ct.P[i] : 0u);
        R[i] = static_cast<uint32_t>(c);
        c >>= 32;
      }
      continue;
    }
    bool ge = R[kSL - 1] != 0;
    if (!ge) {
      ge = true;
      for (int i = kCrtLimbs - 1; i >= 0; --i) {
        if (R[i] != ct.P[i]) {
          ge = R[i] > ct.P[i];
          break;
        }
      }
    }
    if (!ge) break;
    int64_t br = 0;
#pragma unroll
    for (int i = 0; i < kSL; ++i) {
      int64_t d = static_cast<int64_t>(R[i]) - (i < kCrtLimbs ? ct.P[i] : 0u) - br;
      br = d < 0;
      R[i] = static_cast<uint32_t>(d + (br ? (1ll << 32) : 0));
    }
  }
  // symmetric lift: R > floor(P/2) -> R - P
  bool gt = false;
  for (int i = kCrtLimbs - 1; i >= 0; --i) {
    if (R[i] != ct.Phalf[i]) {
      gt = R[i] > ct.Phalf[i];
      break;
    }
  }
  if (gt) {
    uint32_t mag[kCrtLimbs];
    int64_t br = 0;
#pragma unroll
    for (int i = 0; i < kCrtLimbs; ++i) {
      int64_t d = static_cast<int64_t>(ct.P[i]) - R[i] - br;
      br = d < 0;
      mag[i] = static_cast<uint32_t>(d + (br ? (1ll << 32) : 0));
    }
    return -limbs_to_double_rn(mag);
  }
  return limbs_to_double_rn(R);
}

// ---------------------------------------------------------------- lazy form
// S = sum_l w_l r_l kept as one 64-bit sum per 32-bit limb of w (each below
// nm * 255 * 2^32 < 2^45, so no carries until the end), next to the binary32
// estimate t = sum_l r_l (w_l / P) of S / P.
struct CrtLazy {
  uint64_t s[kCrtLimbs];
  float t;
};

__device__ __forceinline__ void crt_lazy_init(CrtLazy& a) {
#pragma unroll
  for (int i = 0; i < kCrtLimbs; ++i) a.s[i] = 0;
  a.t = 0.0f;
}

// a += w_l r_l, r in [0, m_l).
__device__ __forceinline__ void crt_lazy_acc(CrtLazy& a, const CrtTables& ct, int l, uint32_t r) {
#pragma unroll
  for (int i = 0; i < kCrtLimbs; ++i) a.s[i] += static_cast<uint64_t>(ct.w[l][i]) * r;
  // r as binary32 without a conversion instruction: 2^23 + r has r in its low mantissa bits
  a.t = __fmaf_rn(__uint_as_float(0x4B000000u | r) - 8388608.0f, ct.wP[l], a.t);
}

// Eq. (8) finish from the lazy form: x = S - kP with k = rint(t), which is
// round(S / P) or one off (t errs by less than 0.02 for up to 20 moduli), then
// one exact correction each way into the symmetric range (-P/2, P/2] (the
// lift of S mod P: above floor(P/2) it becomes negative), rounded once to
// binary64.  All limb arithmetic is exact; only the choice of k is estimated.
__device__ __forceinline__ double crt_finish_lazy(const CrtLazy& a, const CrtTables& ct) {
  // S in 32-bit limbs (kSL of them)
  uint32_t S[kSL];
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < kCrtLimbs; ++i) {
    c += a.s[i];
    S[i] = static_cast<uint32_t>(c);
    c >>= 32;
  }
  S[kCrtLimbs] = static_cast<uint32_t>(c);
  const uint32_t k = static_cast<uint32_t>(__float2int_rn(a.t));
  // R = S - k P (two's complement in kSL limbs)
  uint32_t R[kSL];
  {
    uint64_t mul = 0;
    int64_t br = 0;
#pragma unroll
    for (int i = 0; i < kSL; ++i) {
      mul += static_cast<uint64_t>(i < kCrtLimbs ? ct.P[i] : 0u) * k;
      const int64_t d = static_cast<int64_t>(S[i]) - static_cast<int64_t>(static_cast<uint32_t>(mul)) - br;
      mul >>= 32;
      br = d < 0;
      R[i] = static_cast<uint32_t>(d + (br ? (1ll << 32) : 0));
    }
  }
  bool neg = static_cast<int32_t>(R[kSL - 1]) < 0;
  uint32_t mag[kSL];
  {  // |R|
    uint64_t cc = neg ? 1u : 0u;
#pragma unroll
    for (int i = 0; i < kSL; ++i) {
      cc += static_cast<uint64_t>(neg ? ~R[i] : R[i]);
      mag[i] = static_cast<uint32_t>(cc);
      cc >>= 32;
    }
  }
  // compare |R| with floor(P/2) = P/2 (P is even: 256 is always a modulus)
  int cmp = mag[kSL - 1] != 0 ? 1 : 0;
#pragma unroll
  for (int i = kCrtLimbs - 1; i >= 0; --i)
    if (cmp == 0 && mag[i] != ct.Phalf[i]) cmp = mag[i] > ct.Phalf[i] ? 1 : -1;
  // R > P/2: R - P (negative, magnitude P - R); R <= -P/2: R + P (magnitude P - |R|)
  if ((!neg && cmp > 0) || (neg && cmp >= 0)) {
    int64_t br = 0;
#pragma unroll
    for (int i = 0; i < kSL; ++i) {
      const int64_t d = static_cast<int64_t>(i < kCrtLimbs ? ct.P[i] : 0u) - mag[i] - br;
      br = d < 0;
      mag[i] = static_cast<uint32_t>(d + (br ? (1ll << 32) : 0));
    }
    neg = !neg;
  }
  const double v = limbs_to_double_rn(mag);  // |x| <= P/2 < 2^159: five limbs
  return neg ? bitsd(dbits(v) ^ 0x8000000000000000ull) : v;  // sign flip without an FP64 instruction
}

// x 2^e for a nonzero finite x whose result stays normal: exponent-field
// arithmetic (exact, as is ldexp); other cases go to ldexp.
__device__ __forceinline__ double scale2_fast(double x, int e) {
  const uint64_t b = dbits(x);
  const int ex = static_cast<int>((b >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF || ex + e <= 0 || ex + e >= 0x7FF) return ldexp(x, e);
  return bitsd(b + (static_cast<uint64_t>(static_cast<int64_t>(e)) << 52));
}

}  // namespace emu
