// Exact split-integer evaluation of the Kronecker-sum Laplacian on cubic
// cells (FP64 results from int32 and FP32 arithmetic), shared by the leaf
// operator and the FP64 level smoother.
//
// For cubic cells the 1-D element matrices are integer matrices over common
// denominators: M = M~ / DM, K = K~ / DK with DM = 30, DK = 3 for Q2 and
// DM = 6, DK = 1 for Q1.  The operator of a group (or brick) is then
//   y = a s / (DM^(d-1) DK) * (integer Kronecker sum) x,
// and the integer Kronecker sum applied to integers is exact.  Relative to a
// power of two q = 2^eq set by the group's largest |x| (|x| < 2^15 q), each
// value is split exactly into x / q = P1 + 2^-15 (P2 + r) with integers
// |P1|, |P2| < 2^15 and r in [0, 1) rounded to 24 bits.  P1 and P2 go
// through the int32 sum factorisation (the bound of the integer Kronecker sum
// keeps every partial sum below 2^31), r through an FP32 one.  The three
// results are recombined in integers, 2^(15+kR) y(P1) + 2^kR y(P2) +
// rint(2^kR y(r)) with kR as large as the same bound keeps this below 2^51
// (5 for 3D Q2, up to 15 for 2D Q1), converted to FP64 exactly, and scaled:
// three FP64 operations per node (conversion, scaling, the energy) instead
// of about thirty.  In units of 2^-15 q the result differs from the exact
// one by 2^-(kR+1) from the rounding of 2^kR y(r) to an integer and by
// B 2^-24 from the 24-bit roundings of r and of the FP32 sum y(r), B the
// bound of the integer Kronecker sum; partial sums reach B 2^30 units, so
// both are near 2^-52 of them, as the roundings of a direct FP64 sum
// factorisation are.
#pragma once
#include <cuda_runtime.h>

namespace gmg {

template <int K>
struct IntElem {
  static constexpr int DM = K == 1 ? 6 : 30, DK = K == 1 ? 1 : 3;
};

template <int K, bool STIFF>
__host__ __device__ constexpr int ielem1(int i, int j) {
  if constexpr (K == 1) {
    return STIFF ? (i == j ? 1 : -1) : (i == j ? 2 : 1);
  } else {
    if constexpr (STIFF) return (i == 1 && j == 1) ? 16 : (i == 1 || j == 1) ? -8 : (i == j) ? 7 : 1;
    else return (i == 1 && j == 1) ? 16 : (i == 1 || j == 1) ? 2 : (i == j) ? 4 : -1;
  }
}

// 2^(15+k) o1 + 2^k o2 + rint(2^k o3) below 2^51 and 2^k o3 below 2^22, for
// an integer Kronecker sum bounded by b per unit input
constexpr bool int_recombination_fits_bound(long long b, int k) {
  return b * ((1LL << (30 + k)) + (1LL << (15 + k)) + (1LL << k)) < (1LL << 51) && b * (1LL << k) < (1LL << 22);
}
// fixed-point bits of the r component in the integer recombination: the most
// that fit (5 for 3D Q2, 10 for 2D Q2, 12 for 3D Q1, 15 for 2D Q1), so the
// rounding of 2^kR y(r) stays near 2^-52 of the integer sum's scale
constexpr int int_recombination_bits_bound(long long b) {
  int k = 0;
  while (k < 20 && int_recombination_fits_bound(b, k + 1)) ++k;
  return k;
}

// |x| = m 2^e split against q = 2^eq (|x| < 2^15 q): x / q = p1 + 2^-15 (p2 + r)
__device__ __forceinline__ void split_exact(double x, int eq, int& p1, int& p2, float& r) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (E) m |= 1ull << 52;
  const int e = (E ? E : 1) - 1075;
  const int s = eq - e;                 // |x| / q = m 2^-s, s >= 38
  const unsigned long long hi = s < 64 ? (m >> s) : 0ull;
  const unsigned long long rem1 = s < 64 ? (m & ((1ull << s) - 1ull)) : m;
  const int s2 = s - 15;                // >= 23
  const unsigned long long mid = s2 < 64 ? (rem1 >> s2) : 0ull;
  const unsigned long long rem2 = s2 < 64 ? (rem1 & ((1ull << s2) - 1ull)) : rem1;
  float rf = 0.f;
  if (rem2) {  // rem2 2^-s2 in [0, 1): its leading 24 bits as a float
    const int nb = 64 - __clzll((long long)rem2);
    const unsigned mant = nb > 24 ? (unsigned)(rem2 >> (nb - 24)) : (unsigned)(rem2 << (24 - nb));
    const int fexp = nb - 1 - s2;
    if (fexp >= -126) rf = __int_as_float(((fexp + 127) << 23) | (int)(mant & 0x7FFFFFu));
  }
  const bool neg = (b >> 63) != 0;
  p1 = neg ? -(int)hi : (int)hi;
  p2 = neg ? -(int)mid : (int)mid;
  r = neg ? -rf : rf;
}

// exact conversions without the FP64 conversion unit
__device__ __forceinline__ double i64_to_double(long long v) {  // |v| < 2^51
  return __longlong_as_double(0x4338000000000000LL + v) - 6755399441055744.0;
}
// exact int64 -> double for |v| < 2^53 with integer operations only, for
// kernels whose FP64 pipe is the scarce unit: the normalised magnitude plus
// the exponent field, the implicit bit carrying into the exponent
__device__ __forceinline__ double i64_to_double_alu(long long v) {
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const int e = 63 - __clzll((long long)a);  // a in [2^e, 2^(e+1)); -1 for a = 0
  const unsigned long long bits = a == 0 ? 0ull : ((unsigned long long)(e + 1022) << 52) + (a << (52 - e));
  return __longlong_as_double((long long)(sgn | bits));
}
// 2^n for -1022 <= n <= 1023 from its bit pattern
__device__ __forceinline__ double pow2_normal(int n) {
  return __longlong_as_double((long long)(n + 1023) << 52);
}
// rint(f 2^KR) for |f 2^KR| < 2^22: the sum lands in [2^23, 2^24), where the
// FP32 spacing is 1, so its low mantissa bits are the rounded integer
template <int KR>
__device__ __forceinline__ int f32_fixed_rint(float f) {
  return __float_as_int(fmaf(f, (float)(1 << KR), 12582912.0f)) - 0x4B400000;
}


}  // namespace gmg
