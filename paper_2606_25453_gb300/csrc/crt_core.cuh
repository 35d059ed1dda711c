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
// nm * 3 * 256 * 2^32 < 2^46 for residues r_l < 3 m_l, so no carries until
// the end), next to the binary32 estimate t = sum_l r_l (w_l / P) of S / P.
// Residues may exceed m_l (the complex modes add m_l or 2 m_l instead of
// reducing): w_l m_l is a multiple of P, so S mod P is unchanged.
struct CrtLazy {
  uint64_t s[kCrtLimbs];
  float t;
};

__device__ __forceinline__ void crt_lazy_init(CrtLazy& a) {
#pragma unroll
  for (int i = 0; i < kCrtLimbs; ++i) a.s[i] = 0;
  a.t = 0.0f;
}

// a += w_l r_l, r in [0, 3 m_l).  L: the number of 32-bit limbs of P (and so
// of every w_l < P); the limbs above stay zero, their products are skipped.
template <int L = kCrtLimbs>
__device__ __forceinline__ void crt_lazy_acc(CrtLazy& a, const CrtTables& ct, int l, uint32_t r) {
  static_assert(L >= 1 && L <= kCrtLimbs, "limb count");
#pragma unroll
  for (int i = 0; i < L; ++i) a.s[i] += static_cast<uint64_t>(ct.w[l][i]) * r;
  // r as binary32 without a conversion instruction: 2^23 + r has r in its low mantissa bits
  a.t = __fmaf_rn(__uint_as_float(0x4B000000u | r) - 8388608.0f, ct.wP[l], a.t);
}

// Six-limb (192-bit) helpers on 32-bit carry chains (PTX add/sub/mad with
// carry; one instruction per limb).  Outputs are early-clobber: they are
// written while later inputs are still to be read.
// d = a - b (mod 2^192); returns 1 if a < b (unsigned).
__device__ __forceinline__ uint32_t sub6(const uint32_t* a, const uint32_t* b, uint32_t* d) {
  uint32_t br;
  asm("sub.cc.u32 %0, %7, %13;\n\t"
      "subc.cc.u32 %1, %8, %14;\n\t"
      "subc.cc.u32 %2, %9, %15;\n\t"
      "subc.cc.u32 %3, %10, %16;\n\t"
      "subc.cc.u32 %4, %11, %17;\n\t"
      "subc.cc.u32 %5, %12, %18;\n\t"
      "subc.u32 %6, 0, 0;"
      : "=&r"(d[0]), "=&r"(d[1]), "=&r"(d[2]), "=&r"(d[3]), "=&r"(d[4]), "=&r"(d[5]), "=&r"(br)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(b[0]), "r"(b[1]), "r"(b[2]),
        "r"(b[3]), "r"(b[4]), "r"(b[5]));
  return br & 1u;
}

// d = k * P for a five-limb P and k < 2^32 (six limbs).  h0..h3 are scratch
// outputs of the multiply chain (hence the front-end note suppressed here).
#pragma nv_diag_suppress 550
__device__ __forceinline__ void mul6(const uint32_t* P, uint32_t k, uint32_t* d) {
  uint32_t h0, h1, h2, h3;
  asm("mul.lo.u32 %0, %10, %15;\n\t"
      "mul.hi.u32 %6, %10, %15;\n\t"
      "mul.hi.u32 %7, %11, %15;\n\t"
      "mul.hi.u32 %8, %12, %15;\n\t"
      "mul.hi.u32 %9, %13, %15;\n\t"
      "mad.lo.cc.u32 %1, %11, %15, %6;\n\t"
      "madc.lo.cc.u32 %2, %12, %15, %7;\n\t"
      "madc.lo.cc.u32 %3, %13, %15, %8;\n\t"
      "madc.lo.cc.u32 %4, %14, %15, %9;\n\t"
      "madc.hi.u32 %5, %14, %15, 0;"
      : "=&r"(d[0]), "=&r"(d[1]), "=&r"(d[2]), "=&r"(d[3]), "=&r"(d[4]), "=&r"(d[5]), "=&r"(h0), "=&r"(h1),
        "=&r"(h2), "=&r"(h3)
      : "r"(P[0]), "r"(P[1]), "r"(P[2]), "r"(P[3]), "r"(P[4]), "r"(k));
}
#pragma nv_diag_default 550

// Eq. (8) finish from the lazy form: x = S - kP with k = rint(t) (below
// 3 * 20 * 256), which is round(S / P) or one off (t errs by less than 0.02
// for up to 20 moduli), then
// one exact correction each way into the symmetric range (-P/2, P/2] (the
// lift of S mod P: above floor(P/2) it becomes negative), rounded once to
// binary64.  All limb arithmetic is exact; only the choice of k is estimated.
__device__ __forceinline__ double crt_finish_lazy(const CrtLazy& a, const CrtTables& ct) {
  // S in six 32-bit limbs: the 64-bit lazy sums (each < 2^46) overlap by 32 bits
  uint32_t S[kSL];
  {
    uint32_t l[kCrtLimbs], h[kCrtLimbs];
#pragma unroll
    for (int i = 0; i < kCrtLimbs; ++i) {
      l[i] = static_cast<uint32_t>(a.s[i]);
      h[i] = static_cast<uint32_t>(a.s[i] >> 32);
    }
    S[0] = l[0];
    asm("add.cc.u32 %0, %5, %10;\n\t"
        "addc.cc.u32 %1, %6, %11;\n\t"
        "addc.cc.u32 %2, %7, %12;\n\t"
        "addc.cc.u32 %3, %8, %13;\n\t"
        "addc.u32 %4, %9, 0;"
        : "=&r"(S[1]), "=&r"(S[2]), "=&r"(S[3]), "=&r"(S[4]), "=&r"(S[5])
        : "r"(l[1]), "r"(l[2]), "r"(l[3]), "r"(l[4]), "r"(h[4]), "r"(h[0]), "r"(h[1]), "r"(h[2]), "r"(h[3]));
  }
  const uint32_t k = static_cast<uint32_t>(__float2int_rn(a.t));
  uint32_t kP[kSL], R[kSL];
  mul6(ct.P, k, kP);
  sub6(S, kP, R);  // S - kP, two's complement
  bool neg = static_cast<int32_t>(R[kSL - 1]) < 0;
  uint32_t mag[kSL];
  {
    const uint32_t zero[kSL] = {0, 0, 0, 0, 0, 0};
    uint32_t nr[kSL];
    sub6(zero, R, nr);
#pragma unroll
    for (int i = 0; i < kSL; ++i) mag[i] = neg ? nr[i] : R[i];
  }
  // |R| against floor(P/2) = P/2 (P is even: 256 is always a modulus)
  const uint32_t half[kSL] = {ct.Phalf[0], ct.Phalf[1], ct.Phalf[2], ct.Phalf[3], ct.Phalf[4], 0};
  uint32_t diff[kSL];
  const bool below = sub6(mag, half, diff) != 0;  // |R| < P/2
  const bool equal = !below && (diff[0] | diff[1] | diff[2] | diff[3] | diff[4] | diff[5]) == 0;
  // R > P/2: R - P (negative, magnitude P - R); R <= -P/2: R + P (magnitude P - |R|)
  if ((!neg && !below && !equal) || (neg && !below)) {
    const uint32_t P6[kSL] = {ct.P[0], ct.P[1], ct.P[2], ct.P[3], ct.P[4], 0};
    sub6(P6, mag, mag);
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
