// Device helpers shared by the qdot kernels: exponent extraction, significand
// rounding, exact fixed-point accumulation, the exact floor(log2(eps/N)) and
// one-time rounding of a fixed-point sum to double.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "qdot.h"

namespace qd {

constexpr int kKeyMin = QDOT_KEY_MIN;
constexpr int kKeyCount = QDOT_KEY_COUNT;
constexpr int kPerf = QDOT_PERF, kHalf = QDOT_HALF, kSingle = QDOT_SINGLE, kDouble = QDOT_DOUBLE,
              kZero = QDOT_ZERO;

typedef __int128 i128;
typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Component decoding (Sec. 1.1 flexp = unbiased exponent; Sec. 3.2 bitmask).
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool is_nonfinite(uint64_t bits) {
  return ((bits >> 52) & 0x7FFu) == 0x7FFu;
}
__device__ __forceinline__ bool is_zero(uint64_t bits) { return (bits << 1) == 0; }

// floor(log2|v|) of a finite nonzero double given by its bits (subnormals
// normalised).
__device__ __forceinline__ int exponent_of(uint64_t bits) {
  int biased = (int)((bits >> 52) & 0x7FFu);
  if (biased) return biased - 1023;
  uint64_t m = bits & 0x000FFFFFFFFFFFFFull;
  return -1011 - __clzll((long long)m);
}

// 53-bit significand with the leading one at bit 52 (finite nonzero v).
__device__ __forceinline__ uint64_t significand_of(uint64_t bits) {
  uint64_t m = bits & 0x000FFFFFFFFFFFFFull;
  if ((bits >> 52) & 0x7FFu) return m | (1ull << 52);
  return m << (__clzll((long long)m) - 11);
}

// Drop the low k bits of X with round-to-nearest-even, keeping X's alignment
// (0 <= k <= 52).  A carry may make the result 2^53.
__device__ __forceinline__ uint64_t round_drop(uint64_t X, int k) {
  if (k == 0) return X;
  uint64_t lsb = (X >> k) & 1ull;
  uint64_t t = X + ((1ull << (k - 1)) - 1ull) + lsb;
  return t & ~((1ull << k) - 1ull);
}

// Bits dropped from a 53-bit significand for each class (PERF / ZERO: all).
__device__ __forceinline__ int drop_bits(int cls) {
  return cls == kHalf ? 42 : (cls == kSingle ? 29 : (cls == kDouble ? 0 : 64));
}

// Quantized significand for class cls (0 for PERF / ZERO).
__device__ __forceinline__ uint64_t quantize_sig(uint64_t X, int cls) {
  int k = drop_bits(cls);
  return k >= 64 ? 0ull : round_drop(X, k);
}

// Double with value (-1)^neg * Xq * 2^(e - 52), Xq <= 2^53 with the alignment
// of a 53-bit significand (low bits beyond the representable range are zero
// by construction).  Overflow gives +-Inf.
__device__ __forceinline__ double compose_double(uint32_t neg, uint64_t Xq, int e) {
  if (Xq == 0) return 0.0;  // perforated / zero components read +0
  uint64_t sign = (uint64_t)neg << 63;
  if (Xq >> 53) {  // carry: 2^53 * 2^(e-52) = 2^(e+1)
    Xq >>= 1;
    e += 1;
  }
  if (e > 1023) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  if (e >= -1022) {
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 1023) << 52) | (Xq & 0x000FFFFFFFFFFFFFull)));
  }
  int sh = -1022 - e;  // subnormal: value = (Xq >> sh) * 2^-1074
  uint64_t m = sh >= 64 ? 0ull : (Xq >> sh);
  return __longlong_as_double((long long)(sign | m));
}

__device__ __forceinline__ int ceil_log2_u32(uint32_t m) { return m <= 1u ? 0 : 32 - __clz((int)(m - 1u)); }

// Precision function, eq. (precision-def); a score >= m_single stays double.
__device__ __forceinline__ int precision_of(long long sigma, int m_half, int m_single) {
  return sigma < 0 ? kPerf : (sigma < m_half ? kHalf : (sigma < m_single ? kSingle : kDouble));
}

// ---------------------------------------------------------------------------
// floor(log2(eps / N)) exactly: the largest integer k with N * 2^k <= eps.
// ---------------------------------------------------------------------------
__device__ inline bool count_times_pow2_le(unsigned long long N, int k, double eps) {
  uint64_t bits = (uint64_t)__double_as_longlong(eps);
  uint64_t Me = significand_of(bits);   // eps = Me * 2^(Ee)
  int Ee = exponent_of(bits) - 52;
  int d = k - Ee;
  if (d >= 0) {
    if (d >= 64) return false;
    u128 lhs = (u128)N << d;
    return lhs <= (u128)Me;
  }
  if (-d >= 64) return true;
  u128 rhs = (u128)Me << (-d);
  return (u128)N <= rhs;
}

__device__ inline int floor_log2_ratio(double eps, unsigned long long N) {
  int k = exponent_of((uint64_t)__double_as_longlong(eps)) - (64 - __clzll((long long)N));
  while (count_times_pow2_le(N, k + 1, eps)) ++k;
  while (!count_times_pow2_le(N, k, eps)) --k;
  return k;
}

// ---------------------------------------------------------------------------
// Round a signed fixed-point value v * 2^lsb to the nearest double (ties to
// even), directly from the integer.
// ---------------------------------------------------------------------------
__device__ inline int clz128(u128 m) {
  uint64_t hi = (uint64_t)(m >> 64), lo = (uint64_t)m;
  return hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
}

__device__ inline double fixed_to_double(i128 v, int lsb) {
  if (v == 0) return 0.0;
  uint32_t neg = v < 0;
  u128 m = neg ? (u128)(-v) : (u128)v;
  int h = 127 - clz128(m);     // index of the top set bit
  int r = h - 52;              // index of the result's last place
  int rmin = -1074 - lsb;      // index of 2^-1074
  if (r < rmin) r = rmin;
  uint64_t mi;
  uint32_t round_bit = 0, sticky = 0;
  if (r <= 0) {
    mi = (uint64_t)(m << (-r));  // exact, fits 53 bits
  } else if (r > 128) {
    mi = 0;  // value < 2^(r - 1 + lsb) <= 2^-1075: rounds to zero
  } else if (r == 128) {
    mi = 0;
    round_bit = (uint32_t)((m >> 127) & 1u);
    sticky = (m & ((((u128)1) << 127) - 1)) != 0;
  } else {
    mi = (uint64_t)(m >> r);
    round_bit = (uint32_t)((m >> (r - 1)) & 1u);
    u128 below = (r - 1 == 0) ? (u128)0 : (m & ((((u128)1) << (r - 1)) - 1));
    sticky = below != 0;
  }
  if (round_bit && (sticky || (mi & 1u))) mi += 1;
  // value = mi * 2^(r + lsb), mi <= 2^53
  int e = r + lsb + 52;  // exponent if mi had its top bit at 52
  uint64_t sign = (uint64_t)neg << 63;
  if (mi == 0) return __longlong_as_double((long long)sign);
  if (mi >> 53) {
    mi >>= 1;
    e += 1;
  }
  if (mi >> 52) {
    if (e > 1023) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
    return __longlong_as_double((long long)(sign | ((uint64_t)(e + 1023) << 52) | (mi & 0x000FFFFFFFFFFFFFull)));
  }
  // mi < 2^52 only when r == rmin: subnormal, value = mi * 2^-1074
  return __longlong_as_double((long long)(sign | mi));
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_max_i32(int v) {
  return __reduce_max_sync(0xffffffffu, v);
}
__device__ __forceinline__ int warp_min_i32(int v) {
  return __reduce_min_sync(0xffffffffu, v);
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int o) {
  unsigned long long lo = (unsigned long long)(u128)v, hi = (unsigned long long)((u128)v >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, o);
  hi = __shfl_xor_sync(0xffffffffu, hi, o);
  return (i128)(((u128)hi << 64) | lo);
}
__device__ __forceinline__ i128 warp_sum_i128(i128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor_i128(v, o);
  return v;
}

// Fraction bits L of the fixed-point accumulator (LSB 2^(e_max - L)): every
// |q(x_i) q(y_i)| <= 2^(e_max + 2), so n of them stay below 2^(L + 2 + ceil(log2 n))
// <= 2^126 in units of the LSB with L = min(104, 124 - ceil(log2 n)).
__host__ __device__ inline int fixed_point_bits(long long n) {
  int c = 0;
  while (c < 63 && (1ll << c) < n) ++c;
  int L = 124 - c;
  return L < 104 ? L : 104;
}

}  // namespace qd
