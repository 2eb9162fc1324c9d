// Device building blocks shared by the GB300 kernels: the counter-based
// random stream, the AR trial, warp/block reductions and the exact
// fixed-point accumulation used for the FP64-grade total propensity.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gbar.h"

namespace gbar {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
//   (x0,x1,x2,x3) -> (hi(B*x2)^x1^k0, lo(B*x2), hi(A*x0)^x3^k1, lo(A*x0))
// with A = 0xD2511F53, B = 0xCD9E8D57 and the key advanced by the Weyl
// increments (0x9E3779B9, 0xBB67AE85) after every round.  Generated in
// registers: the paper's K x M uniform array in global memory (Section
// "Materials", Discussion) is never materialised.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo_a = 0xD2511F53u * c.x;
    const uint32_t hi_a = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo_b = 0xCD9E8D57u * c.z;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The ten round keys of a Philox4x32-10 key (k0, k1): (k0 + r 0x9E3779B9,
// k1 + r 0xBB67AE85), r = 0..9, computed once on the host and passed in a
// kernel's parameters, so that every round XORs a constant operand instead of
// advancing the key in registers.  philox10k computes what philox10 does.
struct PhiloxKeys {
  uint32_t k[20];  // k[2r] = k0 of round r, k[2r + 1] = k1 of round r
};
inline PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys K;
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.k[2 * r] = k0;
    K.k[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return K;
}
__device__ __forceinline__ uint4 philox10k(uint4 c, const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo_a = 0xD2511F53u * c.x;
    const uint32_t hi_a = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo_b = 0xCD9E8D57u * c.z;
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi_b ^ c.y ^ K.k[2 * r], lo_b, hi_a ^ c.w ^ K.k[2 * r + 1], lo_a);
  }
  return c;
}

// Candidate index of a trial: floor(w * M / 2^32) (uniform over 0..M-1 up to
// a 2^-32 preimage lattice).  Requires M < 2^31.
__device__ __forceinline__ uint32_t candidate(uint32_t w, uint32_t M) {
  return __umulhi(w, M);
}

// The AR acceptance test u * T < alpha_j with u in [0,1) (Section "A GPU
// acceptance-rejection algorithm"; strict '<' so that alpha_j = 0 is never
// chosen).  One IEEE round-to-nearest multiply, no contraction.
__device__ __forceinline__ bool accept_f32(uint32_t w, float T, float a) {
  const float u = __fmul_rn(__uint2float_rn(w >> 8), 0x1p-24f);
  return __fmul_rn(u, T) < a;
}
__device__ __forceinline__ bool accept_f64_exact(uint32_t w, double T, double a) {
  const double u = __dmul_rn(__uint2double_rn(w), 0x1p-32);
  return __dmul_rn(u, T) < a;
}

// The FP64 test decided in FP32 where that is provably exact.  GB300 runs
// FP64 arithmetic at a small fraction of its FP32 rate, so a kernel bound by
// the test's FP64 multiplies first compares in FP32 with margins:
//   p_f = RN32(RN32(w) Tq), Tq = RN32(T) 2^-32: within 2^-22 of u T (three
//         roundings; every value is normal when 2^-94 <= T < 2^127);
//   a_f = alpha, or alpha truncated to FP32 from its bits: within 2^-23 below;
//   p_f < RN32(a_f (1 - 2^-18)) gives u T < alpha (1 - 2^-19), so
//         RN64(u T) < alpha: accept;
//   p_f > RN32(a_f (1 + 2^-18)) gives u T > alpha, so RN64(u T) >= alpha:
//         reject;
// alpha = +-0 is rejected (RN64(u T) >= 0).  Trials in between (a relative
// band of about 2^-17 around the threshold) and propensities outside FP32's
// normal range (or negative, infinite, NaN) take the FP64 test, so the
// decision is always that of accept_f64_exact.
struct F64Bound {
  double T;
  float Tq;  // RN32(T) 2^-32 (>= 2^-126) when 2^-94 <= T < 2^127, where the
             // FP32 margins hold; 0 otherwise (the FP64 test only)
};
__device__ __forceinline__ F64Bound f64_bound(double T) {
  F64Bound b;
  b.T = T;
  // the exponent field with the sign bit above it: negatives are not fast
  const bool fast = ((uint32_t)__double2hiint(T) >> 20) - (1023u - 94u) <= 220u;
  b.Tq = fast ? __fmul_rn(__double2float_rn(T), 0x1p-32f) : 0.f;
  return b;
}
constexpr float kF64FilterLo = 1.0f - 0x1p-18f;
constexpr float kF64FilterHi = 1.0f + 0x1p-18f;
// The pre-filter's FP32 operand: alpha itself (FP32 data) or alpha truncated
// to FP32 from its bits, when alpha is positive with an exponent in
// [-125, 127]; 0 for +-0 (never accepted); -1 otherwise (the FP64 test
// decides).  One register per trial instead of a double.
__device__ __forceinline__ float f64_filter_operand(double a) {
  const uint32_t hi = (uint32_t)__double2hiint(a), lo = (uint32_t)__double2loint(a);
  const uint32_t e = hi >> 20;  // with the sign bit: negatives fail the range check
  if (e - (1023u - 125u) <= 252u)
    return __uint_as_float(((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  return ((hi & 0x7fffffffu) | lo) == 0u ? 0.f : -1.f;
}
__device__ __forceinline__ float f64_filter_operand(float a) {
  const uint32_t bits = __float_as_uint(a);
  if ((bits >> 23) - 2u <= 252u) return a;  // positive, exponent field in [2, 254]
  return (bits & 0x7fffffffu) == 0u ? 0.f : -1.f;
}
// 1: accept, 0: reject, 2: the FP64 test decides.
__device__ __forceinline__ int f64_filter(uint32_t w, const F64Bound& t, float af) {
  if (!(t.Tq > 0.f) || af < 0.f) return 2;
  if (af == 0.f) return 0;
  const float pf = __fmul_rn(__uint2float_rn(w), t.Tq);
  if (pf < __fmul_rn(af, kF64FilterLo)) return 1;
  if (pf > __fmul_rn(af, kF64FilterHi)) return 0;
  return 2;
}
// The FP64 product out of line: about one trial in 10^5 needs it, and the
// selection loops that reach it keep their registers.
static __device__ __noinline__ bool accept_f64_slow(uint32_t w, double T, double a) {
  return accept_f64_exact(w, T, a);
}
template <typename TA>
__device__ __forceinline__ bool accept_f64(uint32_t w, const F64Bound& t, TA a) {
  const int d = f64_filter(w, t, f64_filter_operand(a));
  return d == 2 ? accept_f64_slow(w, t.T, (double)a) : d == 1;
}

// ---------------------------------------------------------------------------
// Warp / block reductions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_max_u32(uint32_t v) {
  return __reduce_max_sync(kFull, v);
}
__device__ __forceinline__ int32_t warp_max_i32(int32_t v) {
  return __reduce_max_sync(kFull, v);
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ long long warp_max_i64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long w = __shfl_xor_sync(kFull, v, o);
    v = w > v ? w : v;
  }
  return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(kFull, v, o);
    v = w > v ? w : v;
  }
  return v;
}
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// Exact integer sums: 128-bit unsigned accumulators and their rounding to FP64.
// ---------------------------------------------------------------------------
struct U128 {
  unsigned long long hi = 0, lo = 0;
};
__device__ __forceinline__ U128 add128(U128 x, U128 y) {
  U128 r;
  r.lo = x.lo + y.lo;
  r.hi = x.hi + y.hi + (r.lo < x.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ U128 shl128(unsigned long long x, int s) {  // 0 <= s < 64
  U128 r;
  r.lo = x << s;
  r.hi = s == 0 ? 0ull : (x >> (64 - s));
  return r;
}
__device__ __forceinline__ U128 shr128(U128 x, int s) {  // s >= 0
  U128 r;
  if (s >= 128) return r;
  if (s >= 64) {
    r.lo = x.hi >> (s - 64);
    return r;
  }
  if (s == 0) return x;
  r.lo = (x.lo >> s) | (x.hi << (64 - s));
  r.hi = x.hi >> s;
  return r;
}
__device__ __forceinline__ U128 warp_sum128(U128 x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    U128 y;
    y.hi = __shfl_xor_sync(kFull, x.hi, o);
    y.lo = __shfl_xor_sync(kFull, x.lo, o);
    x = add128(x, y);
  }
  return x;
}

// x * 2^e rounded to the nearest double (ties to even), integer arithmetic
// only.  Callers keep every nonzero result at or above the smallest normal
// double; a result beyond the largest finite double is +inf.
__device__ inline double u128_to_double(U128 x, int e) {
  if (x.hi == 0 && x.lo == 0) return 0.0;
  const int nbits = x.hi ? 128 - __clzll((long long)x.hi) : 64 - __clzll((long long)x.lo);
  int ex = e + nbits - 1;  // exponent of the leading bit
  unsigned long long mant;
  if (nbits <= 53) {
    mant = x.lo << (53 - nbits);
  } else {
    const int sh = nbits - 53;  // bits below the kept 53 (1..75)
    mant = shr128(x, sh).lo;
    const int hb = sh - 1;      // the half bit
    const bool half = hb >= 64 ? ((x.hi >> (hb - 64)) & 1ull) : ((x.lo >> hb) & 1ull);
    const bool sticky = hb >= 64 ? (x.lo != 0 || (x.hi & ((1ull << (hb - 64)) - 1ull)) != 0)
                                 : (x.lo & ((1ull << hb) - 1ull)) != 0;
    if (half && (sticky || (mant & 1ull))) {
      ++mant;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        ++ex;
      }
    }
  }
  if (ex > 1023) return __longlong_as_double(0x7ff0000000000000ll);
  const unsigned long long bits =
      ((unsigned long long)(ex + 1023) << 52) | (mant & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

// ---------------------------------------------------------------------------
// FP32 validity and maximum on bit patterns.  For non-negative IEEE values
// the unsigned bit order is the value order, so the maximum is exact and
// needs no floating-point unit.  A value is valid when it is +finite or -0:
//   smax = max of the bits read as int32   (negative patterns drop out)
//   umax = max of the bits read as uint32  (> 0x80000000 => negative value)
// ---------------------------------------------------------------------------
struct MaxF32 {
  int32_t smax = INT32_MIN;
  uint32_t umax = 0;
  __device__ __forceinline__ void add(uint32_t bits) {
    smax = max(smax, (int32_t)bits);
    umax = max(umax, bits);
  }
  __device__ __forceinline__ bool bad() const {
    return smax >= 0x7f800000 || umax > 0x80000000u;
  }
  __device__ __forceinline__ uint32_t value_bits() const {
    return smax < 0 ? 0u : (uint32_t)smax;
  }
};
struct MaxF64 {
  long long smax = INT64_MIN;
  unsigned long long umax = 0;
  __device__ __forceinline__ void add(unsigned long long bits) {
    smax = max(smax, (long long)bits);
    umax = max(umax, bits);
  }
  __device__ __forceinline__ bool bad() const {
    return smax >= 0x7ff0000000000000ll || umax > 0x8000000000000000ull;
  }
  __device__ __forceinline__ unsigned long long value_bits() const {
    return smax < 0 ? 0ull : (unsigned long long)smax;
  }
};

// ---------------------------------------------------------------------------
// Exact fixed-point accumulation of non-negative FP32 values given the
// biased exponent e_ref of their maximum (GB300 runs FP64 adds at a small
// fraction of its integer rate, so the per-element work stays in integers):
//   value = m * 2^(e - 150), m the 24-bit significand, e >= 1 the exponent;
//   d = e_ref - e >= 0;  d <= 24: a1 += m << (24 - d)   (unit 2^(e_ref-174))
//                        d <= 49: a2 += m << (49 - d)   (unit 2^(e_ref-199))
//                        else     a3 += value (FP32; each term < 2^-48 max)
// Terms are < 2^48, so a1 and a2 stay exact for up to 2^15 elements; they
// are order-independent integers.  The result, rounded once to FP64 per
// window, is within 3 * 2^-53 * sum + 2^-60 * max of the exact sum.
// ---------------------------------------------------------------------------
struct FxSum {
  unsigned long long a1 = 0, a2 = 0;
  float a3 = 0.f;
  __device__ __forceinline__ void add(uint32_t bits, int e_ref) {
    bits &= 0x7fffffffu;
    int e = (int)(bits >> 23);
    uint32_t m = bits & 0x7fffffu;
    if (e) m |= 0x800000u; else e = 1;
    const int d = e_ref - e;
    if (d <= 24) {
      a1 += (unsigned long long)m << (24 - d);
    } else if (d <= 49) {
      a2 += (unsigned long long)m << (49 - d);
    } else {
      a3 = __fadd_rn(a3, __uint_as_float(bits));
    }
  }
  __device__ __forceinline__ void merge(const FxSum& o) {
    a1 += o.a1;
    a2 += o.a2;
    a3 = __fadd_rn(a3, o.a3);
  }
  __device__ __forceinline__ void warp_reduce() {
    a1 = warp_sum_u64(a1);
    a2 = warp_sum_u64(a2);
    a3 = warp_sum_f32(a3);
  }
  // e_ref here is max(biased exponent of the maximum, 1).
  __device__ __forceinline__ double to_double(int e_ref) const {
    const double s1 = __hiloint2double((e_ref - 174 + 1023) << 20, 0);
    const double s2 = __hiloint2double((e_ref - 199 + 1023) << 20, 0);
    const double hi = __dmul_rn(__ull2double_rn(a1), s1);
    const double mid = __dmul_rn(__ull2double_rn(a2), s2);
    return __dadd_rn(__dadd_rn(hi, mid), (double)a3);
  }
};

__device__ __forceinline__ int fx_eref(uint32_t max_bits) {
  const int e = (int)((max_bits & 0x7fffffffu) >> 23);
  return e < 1 ? 1 : e;
}

}  // namespace gbar
