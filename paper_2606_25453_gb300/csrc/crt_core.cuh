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

// Round a nonnegative 5-limb integer to binary64, nearest-even.
__device__ __forceinline__ double limbs_to_double_rn(const uint32_t* x) {
  int L = kCrtLimbs - 1;
  while (L > 0 && x[L] == 0) --L;
  if (L <= 3) {
    unsigned __int128 u = 0;
    for (int i = L; i >= 0; --i) u = (u << 32) | x[i];
    return u128_to_double_rn(u);
  }
  // L == 4: window of limbs 1..4 (>= 97 significant bits) plus a sticky bit
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

}  // namespace emu
