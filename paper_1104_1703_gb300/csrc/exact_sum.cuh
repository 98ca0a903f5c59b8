// Sum of a few doubles without the FP64 pipe: the FP64 level-0 sweep's
// neighbour sum (Section 2's 7-point stencil: the six neighbour values of a
// cell) formed with integer instructions, so that the sweep issues one FP64
// instruction per update (the final multiply-add) instead of six.
//
// Method: fixed-point accumulation in one 64-bit window anchored at the
// largest exponent of the terms (a narrow form of Kulisch's long
// accumulator).  With e_max the largest biased exponent and G guard bits,
// term x_j = m_j 2^(e_j - 1075) (m_j its 53-bit significand) enters as the
// integer a_j = floor(m_j 2^(G - (e_max - e_j))) with x_j's sign; the sum
// S = sum_j a_j is exact in 64 bits as long as N 2^(53 + G) <= 2^63, and
// the result is S 2^(e_max - 1075 - G) rounded once to the nearest double
// (ties to even).  Error against the exact real sum: below half an ulp of
// the result plus N - 1 units of 2^(e_max - 1075 - G) (the truncated low bits
// of the terms more than G binades below the largest), i.e. at most
// (N - 1) 2^(-52 - G) times the largest term.  With N = 6 and G = 7 that is
// below 2^-57 |x|_max + half an ulp, tighter than the 5 roundings of a plain
// FP64 sum.
//
// Edge cases: subnormal terms count as zero; a sum whose largest term is
// below 2^(64 - 1023) (every term below about 1e-289) is returned as zero,
// and a result below the smallest normal double flushes to a zero of its
// sign; an overflow rounds to the infinity of its sign.  If any term is
// infinite or NaN the result is what IEEE addition gives: NaN if a term is
// NaN or infinities of both signs meet, else the infinity (so a diverging
// solve still sees a non-finite value).
#pragma once

#include <cstdint>
#include <cstring>

namespace gbmg {

__host__ __device__ __forceinline__ unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}

__host__ __device__ __forceinline__ double double_of(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}

__host__ __device__ __forceinline__ int clz64(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)u);
#else
  return u ? __builtin_clzll(u) : 64;
#endif
}

// guard bits for N terms: the largest G with N 2^(53 + G) <= 2^63
template <int N>
struct SumGuard {
  static constexpr int value = N <= 1 ? 10 : (N <= 2 ? 9 : (N <= 4 ? 8 : (N <= 8 ? 7 : (N <= 16 ? 6 : 5))));
};

template <int N>
__host__ __device__ __forceinline__ double exact_sum(const double (&x)[N]) {
  static_assert(N >= 1 && N <= 32, "exact_sum: 1..32 terms");
  constexpr int G = SumGuard<N>::value;
  unsigned long long b[N];
  int e[N];
  int emax = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    b[j] = bits_of(x[j]);
    e[j] = (int)((b[j] >> 52) & 0x7ffu);
    emax = e[j] > emax ? e[j] : emax;
  }
  if (emax == 0x7ff) {
    // an infinity or a NaN among the terms: the IEEE sum's value, decided on
    // the bits (no FP64 instruction on this path either)
    bool nan = false, pinf = false, ninf = false;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (e[j] != 0x7ff) continue;
      if (b[j] & 0xfffffffffffffull) nan = true;
      else if (b[j] >> 63) ninf = true;
      else pinf = true;
    }
    if (nan || (pinf && ninf)) return double_of(0x7ff8000000000000ull);
    return double_of(pinf ? 0x7ff0000000000000ull : 0xfff0000000000000ull);
  }
  if (emax < 64) return 0.0;
  long long S = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    // the significand with its leading bit, G bits up, then aligned to the
    // largest exponent; a zero (e = 0, so a shift of e_max >= 64, clamped to
    // 63) leaves nothing, as 2^(53 + G) < 2^63
    const unsigned long long m = ((b[j] & 0xfffffffffffffull) | 0x10000000000000ull) << G;
    const int sh = emax - e[j];
    const long long a = (long long)(m >> (sh < 63 ? sh : 63));
    S += (b[j] >> 63) ? -a : a;
  }
  if (S == 0) return 0.0;
  const unsigned long long sign = S < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long u = S < 0 ? 0ull - (unsigned long long)S : (unsigned long long)S;
  const int lz = clz64(u);        // >= 1: |S| < 2^63
  const unsigned long long n = u << lz;  // leading bit at 63
  unsigned long long M = n >> 11;         // 53 bits, leading bit at 52
  const unsigned r = (unsigned)(n & 0x7ffu);
  M += (r > 0x400u || (r == 0x400u && (M & 1ull))) ? 1ull : 0ull;  // round to nearest, ties to even
  // value = (n / 2^63) 2^(63 - lz + e_max - 1075 - G): biased exponent
  const int E = emax + 11 - G - lz;
  if (E <= 0) return double_of(sign);
  // M = 2^53 after rounding carries into the exponent field by the addition
  const unsigned long long v = ((unsigned long long)(E - 1) << 52) + M;
  if (v >= 0x7ff0000000000000ull) return double_of(sign | 0x7ff0000000000000ull);
  return double_of(sign | v);
}

}  // namespace gbmg
