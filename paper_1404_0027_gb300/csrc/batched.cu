// ar_select_batched: thousands of realizations with uneven M_b and K_b.  The
// paper runs K realizations as K thread blocks of M threads (Section "A GPU
// acceptance-rejection algorithm"; a 1D grid limited to 65536 blocks, Section
// "Implementation"; several blocks per realization when M exceeds a block,
// Discussion).
//
// With a plan whose realizations all sit in CTA home lists (global share 0,
// the default) and 16-byte aligned FP32 data, ar_select_batched is ONE launch
// of k_batched_select<..., FUSED>: each CTA first reduces the chunks of its
// own home realizations, then selects them (see the kernel).  Otherwise it is
// two launches on the caller's stream, the reduction and the selections
// (ar_bound_batched: the reduction and the combine):
//
//   k_bound_reg / k_batched_bound   per-chunk partial results: maximum
//       (exact, on bit patterns), validity and exact sum of chunks of at most
//       1024 propensities (with a plan: each realization cut into equal
//       chunks).  Each warp loads its chunk with 16-byte vector loads into
//       registers (one chunk in flight per warp, 32 warps per SM), and only touches
//       the 16-byte groups a chunk has.  A chunk's sum is an exact integer in
//       units of a power of two set by the chunk's maximum: when every
//       non-zero value lies within 2^24 of that maximum (the common case) it
//       comes from packed FP32 additions that are exact by construction
//       (three-level splitting against power-of-two constants), otherwise
//       from integer windows.  GB300's FP64 rate is a small fraction of its
//       FP32 and integer rates, so no FP64 operation touches the elements.
//   k_batched_combine   one warp per realization: T_b = the maximum of its
//       chunk maxima, the chunk sums aligned and added exactly in 128 bits and
//       rounded once to FP64, the status.  In ar_select_batched the selection
//       kernel does this instead when it claims a range of the realization
//       (the bound; in the one-launch form the maximum comes from shared
//       memory), and for the realization's first range also the sum.
//   k_batched_select    the selections.  A plan gives each persistent CTA a
//       home list of its realizations (the costliest ones, by
//       longest-processing-time-first list scheduling) in ranges of 64
//       selections claimed in order from a shared-memory counter, so the
//       warps of an SM work on a few realizations at a time and the
//       gathers hit L1; the cheapest realizations form a global queue of
//       64-selection ranges that the warps drain once their home list is
//       empty.  Selections come from runs of 64 (one trial sequence per run,
//       its accepted trials in order are the run's selections): a warp takes
//       one run at a time and evaluates 64, 128 or 192 consecutive trials of
//       it per round (1-3 Philox blocks per lane, all gathers in flight at
//       once); ballots and prefix counts number the accepted trials, and one
//       coalesced copy per run writes them out.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <numeric>
#include <queue>
#include <type_traits>
#include <utility>
#include <vector>

#include "device.cuh"
#include "host.hpp"
#include "select.cuh"

namespace gbar {
namespace {

// selection kernel tile shapes (warps per CTA; 1024 threads per SM): the
// plan's default and the autotuner's candidates
constexpr int kSelShapes[3] = {16, 32, 8};
constexpr int kSelThreadsPerSm = 1024;
constexpr int kBWarps = 8;  // reduction kernels
constexpr int kBNT = kBWarps * 32;
constexpr int kBCtasPerSm = 4;  // k_bound_reg: 32 warps per SM, 64 registers
constexpr uint32_t kChunk = 1024;  // reduction chunk (elements)
constexpr int kVPL = kChunk / 32;  // elements per lane (register path)
constexpr uint32_t kSItem = 64;     // selections per home work item (default)
constexpr uint32_t kGItem = 64;     // selections per global-queue work item

// ---- plan-built work items -------------------------------------------------
struct RItem {  // one reduction chunk: alpha_cat[e0, e0 + n)
  int64_t e0;
  uint32_t n;
  uint32_t pad;
};
struct RInfo {  // chunk partials of one realization
  uint32_t p0, nch;
};
struct SItem {     // selections [s0, s1) of realization b
  int64_t a0, o0;  // first element / first output index of the realization
  uint32_t M, b, s0, s1;
  uint32_t p0, nch;  // its chunk partials
  uint32_t slot;     // the realization's place in its CTA's home list (fused launch)
  uint32_t pad;
};
struct Part {                 // a chunk's partial result
  unsigned long long hi, lo;  // FP32 data: exact sum (hi:lo) 2^e; FP64: lo = sum bits
  unsigned long long vmax;    // maximum (bit pattern)
  int32_t e;
  uint32_t bad;               // 1: invalid value, 2: unusable offsets
};
static_assert(sizeof(Part) == 32, "Part layout");

struct Scratch {
  uint32_t squeue;  // next global work item to claim
  uint32_t sdone;   // CTAs finished (the last one resets squeue)
  uint32_t pad[2];
};

struct Params {
  const uint2* fred;     // fused launch: the chunks each CTA reduces, (chunk, slot)
  const uint32_t* frptr; // [grid + 1] fused launch: a CTA's range of fred
  const RItem* ritems;   // NULL: one item per realization, read from the offsets
  const RInfo* rinfo;    // [B] (plan)
  const SItem* sitems;   // NULL: one item per realization, global queue
  const uint32_t* scta;  // [grid + 1] home lists of the CTAs (plan)
  uint32_t nr;
  uint32_t gq0, gq1;     // global-queue items [gq0, gq1) of sitems (plan)
  Part* parts;           // [NR] (plan) or [B]
  Scratch* scratch;
  const unsigned char* alpha;
  const int64_t* offsets;
  const int64_t* out_offsets;
  double* bound_sum;
  int32_t* idx;
  ar_stats* stats;
  uint32_t* status;
  unsigned long long cap;  // trials per selection, 1 .. 2^32
  uint32_t B;
  uint32_t sel_base;
  uint32_t b_base;
  PhiloxKeys keys;  // round keys of the seed
  uint32_t vec_ok;  // alpha_cat is 16-byte aligned (vector loads)
  // selection bounds: T_b = bound_in[b * bound_stride]
  const double* bound_in;
  int64_t bound_stride;
  uint32_t bound_given;  // caller's bounds: checked like ar_select_k's
  uint32_t zero_status;  // the reduction reports all-zero realizations
  uint32_t nslots;       // fused launch: shared-memory counters per CTA (home realizations)
  uint32_t fold;         // the selection takes T from the chunk partials and the
                         // first range of a realization writes {T, sum}, status
};

// Exact fixed-point windows of non-negative FP32 values, e_ref the biased
// exponent of their maximum (at least 1); value = m 2^(e - 150), d = e_ref - e:
//   d <= 24: a1 += m << (24 - d)   (unit 2^(e_ref - 174))
//   d <= 49: a2 += m << (49 - d)   (unit 2^(e_ref - 199))
//   d <= 74: a3 += m << (74 - d)   (unit 2^(e_ref - 224))
// Smaller values (below 2^-73 of the maximum each) are dropped.  Every term
// is < 2^48, so each window is exact for up to 2^15 terms; the total is
// (a1 2^50 + a2 2^25 + a3) 2^(e_ref - 224), below 2^108 units for a chunk.
struct Fx3 {
  unsigned long long a1 = 0, a2 = 0, a3 = 0;
  __device__ __forceinline__ void add(uint32_t bits, int e_ref) {
    bits &= 0x7fffffffu;
    int e = (int)(bits >> 23);
    uint32_t m = bits & 0x7fffffu;
    if (e) m |= 0x800000u; else e = 1;
    const int d = e_ref - e;
    if (d <= 24) a1 += (unsigned long long)m << (24 - d);
    else if (d <= 49) a2 += (unsigned long long)m << (49 - d);
    else if (d <= 74) a3 += (unsigned long long)m << (74 - d);
  }
  __device__ __forceinline__ U128 total() const {
    return add128(shl128(a1, 50), add128(shl128(a2, 25), U128{0ull, a3}));
  }
};

// 2^k as an FP32 value, -126 <= k <= 127
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }
// f 2^s for an FP32 f that is an integer multiple of 2^-s with |f 2^s| <= 2^24,
// -126 <= s / 2 and s - s / 2 <= 127 (two exact power-of-two scalings)
__device__ __forceinline__ long long scaled_int(float f, int s) {
  const int s1 = s / 2;
  return __float2ll_rn(__fmul_rn(__fmul_rn(f, pow2f(s1)), pow2f(s - s1)));
}

// ===========================================================================
// Reduction kernels
// ===========================================================================

// Partial result of N FP32 values (bit patterns) held in registers plus one
// extra value per lane; zeros are neutral.  All lanes return it.
template <int N>
__device__ __forceinline__ Part reduce_f32(const uint32_t (&v)[N], uint32_t xs) {
  static_assert(N % 2 == 0 && N / 2 + 1 <= 33, "terms per accumulator");
  // maximum of the raw bits; an invalid value or -0 pushes it to >= 2^31 or
  // into the inf/NaN range and sends the chunk to the exact slow path
  uint32_t umax = xs, umin1 = xs - 1u;  // umin1: smallest non-zero value - 1
#pragma unroll
  for (int k = 0; k < N; ++k) {
    umax = max(umax, v[k]);
    umin1 = min(umin1, v[k] - 1u);
  }
  umax = __reduce_max_sync(kFull, umax);
  umin1 = __reduce_min_sync(kFull, umin1);
  Part r;
  const int e_ref = max((int)(umax >> 23), 1);
  if (umax < 0x7f800000u && e_ref >= 25 && e_ref <= 248 &&
      umin1 >= ((uint32_t)(e_ref - 24) << 23) - 1u) {
    // Every non-zero value x lies in [2^24 U, 2^48 U), U = 2^(e_ref - 174),
    // and is a multiple of U.  x = h + m + r with h a multiple of 2^30 U,
    // m of 2^12 U, |r| <= 2^11 U, each split exact (round-to-nearest against
    // 1.5 2^53 U and 1.5 2^35 U, then exact differences); at most 33 terms
    // per accumulator keep every running sum below 2^24 units of its level,
    // so the three FP32 sums are exact.
    const float C1 = __int_as_float(((e_ref + 6) << 23) | 0x400000);
    const float C2 = __int_as_float(((e_ref - 12) << 23) | 0x400000);
    const float2 c1 = make_float2(C1, C1), n1 = make_float2(-C1, -C1);
    const float2 c2 = make_float2(C2, C2), n2 = make_float2(-C2, -C2);
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 s1 = make_float2(0.f, 0.f), s2 = s1, s3 = s1;
    auto split = [&](uint32_t a, uint32_t b) {
      const float2 x = make_float2(__uint_as_float(a), __uint_as_float(b));
      const float2 h = __fadd2_rn(__fadd2_rn(x, c1), n1);
      const float2 l = __ffma2_rn(h, m1, x);  // x - h
      const float2 m = __fadd2_rn(__fadd2_rn(l, c2), n2);
      s1 = __fadd2_rn(s1, h);
      s2 = __fadd2_rn(s2, m);
      s3 = __fadd2_rn(s3, __ffma2_rn(m, m1, l));  // l - m
    };
#pragma unroll
    for (int k = 0; k < N; k += 2) split(v[k], v[k + 1]);
    split(xs, 0u);
    const long long S =
        ((scaled_int(s1.x, 144 - e_ref) + scaled_int(s1.y, 144 - e_ref)) << 30) +
        ((scaled_int(s2.x, 162 - e_ref) + scaled_int(s2.y, 162 - e_ref)) << 12) +
        scaled_int(s3.x, 174 - e_ref) + scaled_int(s3.y, 174 - e_ref);
    const unsigned long long X = warp_sum_u64((unsigned long long)S);  // < 2^58
    const U128 x50 = shl128(X, 50);
    r.hi = x50.hi;
    r.lo = x50.lo;
    r.vmax = umax;
    r.e = e_ref - 224;
    r.bad = 0u;
    return r;
  }
  // exact slow path: validity on signed/unsigned maxima, integer windows
  MaxF32 mx;
#pragma unroll
  for (int k = 0; k < N; ++k) mx.add(v[k]);
  mx.add(xs);
  mx.smax = warp_max_i32(mx.smax);
  mx.umax = warp_max_u32(mx.umax);
  const uint32_t vb = mx.value_bits();
  const int e2 = fx_eref(vb);
  Fx3 fx;
#pragma unroll
  for (int k = 0; k < N; ++k) fx.add(v[k], e2);
  fx.add(xs, e2);
  fx.a1 = warp_sum_u64(fx.a1);
  fx.a2 = warp_sum_u64(fx.a2);
  fx.a3 = warp_sum_u64(fx.a3);
  const U128 X = fx.total();
  r.hi = X.hi;
  r.lo = X.lo;
  r.vmax = vb;
  r.e = e2 - 224;
  r.bad = mx.bad() ? 1u : 0u;
  return r;
}

// Register path: chunk [e0, e0 + n), n <= 1024, loaded straight into lane
// registers (16-byte groups when the buffer is aligned, head and tail
// elements by lanes 0-2 and 3-5).
__device__ __forceinline__ Part chunk_f32(const uint32_t* __restrict__ u, int64_t e0, uint32_t n,
                                          bool vec_ok) {
  const uint32_t lane = threadIdx.x & 31u;
  int64_t g0 = (e0 + 3) & ~int64_t(3), g1 = (e0 + n) & ~int64_t(3);
  if (!vec_ok || g1 < g0) g0 = g1 = e0;  // no vector part
  uint32_t v[kVPL];
  if (vec_ok) {
    const uint32_t ngroups = (uint32_t)((g1 - g0) >> 2);
    const uint4* gp = reinterpret_cast<const uint4*>(u + g0);
#pragma unroll
    for (int k = 0; k < kVPL / 4; ++k) {
      const uint32_t g = lane + 32u * k;
      uint4 x = make_uint4(0u, 0u, 0u, 0u);
      if (g < ngroups) x = __ldg(gp + g);
      v[4 * k] = x.x;
      v[4 * k + 1] = x.y;
      v[4 * k + 2] = x.z;
      v[4 * k + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kVPL; ++k) {
      const uint32_t i = lane + 32u * k;
      v[k] = i < n ? __ldg(u + e0 + i) : 0u;
    }
  }
  const int64_t hn = g0 - e0, tn = vec_ok ? e0 + n - g1 : 0;
  uint32_t xs = 0u;
  if (lane < 3 && (int64_t)lane < hn) xs = __ldg(u + e0 + lane);
  else if (lane >= 3 && lane < 6 && (int64_t)(lane - 3) < tn) xs = __ldg(u + g1 + (lane - 3));
  return reduce_f32<kVPL>(v, xs);
}

// Realizations longer than a chunk (calls without a plan): two passes over
// global memory, per-lane integer windows flushed every 2^15 terms.
__device__ Part long_f32(const uint32_t* __restrict__ w, uint32_t n) {
  const uint32_t lane = threadIdx.x & 31u;
  MaxF32 mx;
  for (uint32_t i = lane; i < n; i += 32) mx.add(__ldg(w + i));
  mx.smax = warp_max_i32(mx.smax);
  mx.umax = warp_max_u32(mx.umax);
  const uint32_t vb = mx.value_bits();
  const int e_ref = fx_eref(vb);
  U128 acc;
  Fx3 fx;
  uint32_t in_block = 0;
  for (uint32_t i = lane; i < n; i += 32) {
    fx.add(__ldg(w + i), e_ref);
    if (++in_block == 32768u) {
      acc = add128(acc, fx.total());
      fx = Fx3();
      in_block = 0;
    }
  }
  acc = add128(acc, fx.total());
  // one bit down: 2^31 values below 2^98 units each would overflow 128 bits
  const U128 X = warp_sum128(shr128(acc, 1));
  Part r;
  r.hi = X.hi;
  r.lo = X.lo;
  r.vmax = vb;
  r.e = e_ref - 223;
  r.bad = mx.bad() ? 1u : 0u;
  return r;
}

__device__ Part reduce_f64(const unsigned long long* __restrict__ w, uint32_t n) {
  const uint32_t lane = threadIdx.x & 31u;
  MaxF64 mx;
  double s = 0.0;
  for (uint32_t i = lane; i < n; i += 32) {
    const unsigned long long x = __ldg(w + i);
    mx.add(x);
    s = __dadd_rn(s, __longlong_as_double((long long)x));
  }
  mx.smax = warp_max_i64(mx.smax);
  mx.umax = warp_max_u64(mx.umax);
  Part r;
  r.hi = 0ull;
  r.lo = (unsigned long long)__double_as_longlong(warp_sum_f64(s));
  r.vmax = mx.value_bits();
  r.e = 0;
  r.bad = mx.bad() ? 1u : 0u;
  return r;
}

__device__ __forceinline__ void store_part(Part* dst, const Part& r) {
  if ((threadIdx.x & 31u) == 0) *dst = r;
}

// reduce with only the first kq groups (of 4 values) per lane live
template <int N>
__device__ __forceinline__ Part reduce_f32q(const uint32_t (&v)[N], uint32_t xs, int kq) {
  uint32_t umax = xs, umin1 = xs - 1u;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (k / 4 < kq) {
      umax = max(umax, v[k]);
      umin1 = min(umin1, v[k] - 1u);
    }
  }
  umax = __reduce_max_sync(kFull, umax);
  umin1 = __reduce_min_sync(kFull, umin1);
  Part r;
  const int e_ref = max((int)(umax >> 23), 1);
  if (umax < 0x7f800000u && e_ref >= 25 && e_ref <= 248 &&
      umin1 >= ((uint32_t)(e_ref - 24) << 23) - 1u) {
    const float C1 = __int_as_float(((e_ref + 6) << 23) | 0x400000);
    const float C2 = __int_as_float(((e_ref - 12) << 23) | 0x400000);
    const float2 c1 = make_float2(C1, C1), n1 = make_float2(-C1, -C1);
    const float2 c2 = make_float2(C2, C2), n2 = make_float2(-C2, -C2);
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 s1 = make_float2(0.f, 0.f), s2 = s1, s3 = s1;
    auto split = [&](uint32_t a, uint32_t b) {
      const float2 x = make_float2(__uint_as_float(a), __uint_as_float(b));
      const float2 h = __fadd2_rn(__fadd2_rn(x, c1), n1);
      const float2 l = __ffma2_rn(h, m1, x);
      const float2 m = __fadd2_rn(__fadd2_rn(l, c2), n2);
      s1 = __fadd2_rn(s1, h);
      s2 = __fadd2_rn(s2, m);
      s3 = __fadd2_rn(s3, __ffma2_rn(m, m1, l));
    };
#pragma unroll
    for (int k = 0; k < N; k += 2)
      if (k / 4 < kq) split(v[k], v[k + 1]);
    split(xs, 0u);
    const int t1 = 144 - e_ref, t2 = 162 - e_ref, t3 = 174 - e_ref;
    const float a1 = pow2f(t1 / 2), b1 = pow2f(t1 - t1 / 2);
    const float a2 = pow2f(t2 / 2), b2 = pow2f(t2 - t2 / 2);
    const float a3 = pow2f(t3 / 2), b3 = pow2f(t3 - t3 / 2);
    auto cv = [](float f, float a, float b) { return __float2int_rn(__fmul_rn(__fmul_rn(f, a), b)); };
    const long long S = ((long long)(cv(s1.x, a1, b1) + cv(s1.y, a1, b1)) << 30) +
                        ((long long)(cv(s2.x, a2, b2) + cv(s2.y, a2, b2)) << 12) +
                        (long long)(cv(s3.x, a3, b3) + cv(s3.y, a3, b3));
    const unsigned long long X = warp_sum_u64((unsigned long long)S);
    const U128 x50 = shl128(X, 50);
    r.hi = x50.hi;
    r.lo = x50.lo;
    r.vmax = umax;
    r.e = e_ref - 224;
    r.bad = 0u;
    return r;
  }
  return reduce_f32<N>(v, xs);  // slow path (zeros beyond kq are loaded as zeros)
}

// Reduces chunk c of the plan (16-byte loads straight into lane registers)
// and stores its partial result.
__device__ __forceinline__ Part reduce_chunk(const Params& p, uint32_t c) {
  const uint32_t* u = reinterpret_cast<const uint32_t*>(p.alpha);
  const uint32_t lane = threadIdx.x & 31u;
  const RItem d = p.ritems[c];
  int64_t g0 = (d.e0 + 3) & ~int64_t(3), g1 = (d.e0 + d.n) & ~int64_t(3);
  if (g1 < g0) g0 = g1 = d.e0;
  const uint32_t ngroups = (uint32_t)((g1 - g0) >> 2);
  const int kq = (int)((ngroups + 31u) >> 5);
  const uint4* gp = reinterpret_cast<const uint4*>(u + g0);
  uint32_t v[kVPL];
#pragma unroll
  for (int k = 0; k < kVPL / 4; ++k) {
    const uint32_t g = lane + 32u * k;
    uint4 x = make_uint4(0u, 0u, 0u, 0u);
    if (k < kq && g < ngroups) x = __ldg(gp + g);
    v[4 * k] = x.x; v[4 * k + 1] = x.y; v[4 * k + 2] = x.z; v[4 * k + 3] = x.w;
  }
  const int64_t hn = g0 - d.e0, tn = d.e0 + d.n - g1;
  uint32_t xs = 0u;
  if (lane < 3 && (int64_t)lane < hn) xs = __ldg(u + d.e0 + lane);
  else if (lane >= 3 && lane < 6 && (int64_t)(lane - 3) < tn) xs = __ldg(u + g1 + (lane - 3));
  const Part r = reduce_f32q<kVPL>(v, xs, kq);
  store_part(p.parts + c, r);
  return r;
}

// One chunk in flight per warp, 32 warps per SM: more warps to cover the
// loads' latency and the reduce work than two chunks per warp at 16 warps.
__global__ void __launch_bounds__(kBNT, kBCtasPerSm) k_bound_reg(const Params p) {
  const uint32_t stride = gridDim.x * kBWarps;
  for (uint32_t it = blockIdx.x * kBWarps + (threadIdx.x >> 5); it < p.nr; it += stride)
    reduce_chunk(p, it);
}

// Register path: FP64 data, unaligned FP32 buffers, calls without a plan.
template <typename TS>
__global__ void __launch_bounds__(kBNT) k_batched_bound(const Params p) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * kBWarps;
  const uint32_t nitems = p.ritems ? p.nr : p.B;
  for (uint32_t it = blockIdx.x * kBWarps + (threadIdx.x >> 5); it < nitems; it += stride) {
    int64_t e0;
    uint32_t n;
    if (p.ritems) {
      e0 = p.ritems[it].e0;
      n = p.ritems[it].n;
    } else {
      int64_t v = 0;
      if (lane < 2) v = __ldg(p.offsets + it + lane);
      const int64_t a0 = __shfl_sync(kFull, v, 0), a1 = __shfl_sync(kFull, v, 1);
      e0 = a0;
      n = (a1 < a0 || a1 - a0 >= (1ll << 31)) ? 0xffffffffu : (uint32_t)(a1 - a0);
    }
    Part r;
    if (n == 0xffffffffu) {  // unusable offsets
      r.hi = r.lo = r.vmax = 0ull;
      r.e = 0;
      r.bad = 2u;
    } else if constexpr (sizeof(TS) == 4) {
      const uint32_t* u = reinterpret_cast<const uint32_t*>(p.alpha);
      r = n <= kChunk ? chunk_f32(u, e0, n, p.vec_ok != 0) : long_f32(u + e0, n);
    } else {
      r = reduce_f64(reinterpret_cast<const unsigned long long*>(p.alpha) + e0, n);
    }
    store_part(p.parts + it, r);
  }
}

// Bound (maximum bit pattern) and validity of one realization from its chunk
// partials; with `write` also its FP64 total (chunk sums aligned to one bit
// above the largest exponent -- chunk sums are < 2^108 units, so 2^21 of them
// fit in 128 bits; bits below 2^-96 of the maximum are dropped -- added
// exactly and rounded once; FP64 data: FP64 sums in chunk order), stored by
// lane 0 as {T, sum} ({NaN, NaN} when invalid), and the status bits.
// Chunk partials are read from L2 (ld.global.cg): in the one-launch form they
// were written earlier in the same launch, so the read-only (non-coherent)
// load path, whose data must not change during the launch, is not theirs.
// The exact total of a realization's FP32 chunk partials (all valid), emax
// above every chunk exponent, rounded once; the value is returned in lane 0.
// Kept out of line: the selection loops that reach it stay small.
__device__ __noinline__ double fold_sum_f32(const Part* parts, uint32_t nch, int emax) {
  const uint32_t lane = threadIdx.x & 31u;
  U128 acc;
  for (uint32_t k = lane; k < nch; k += 32) {
    const Part* q = parts + k;
    U128 y;
    y.hi = __ldcg(&q->hi);
    y.lo = __ldcg(&q->lo);
    acc = add128(acc, shr128(y, emax - __ldcg(&q->e)));
  }
  acc = warp_sum128(acc);
  return lane == 0 ? u128_to_double(acc, emax) : 0.0;
}

template <typename TS>
__device__ __forceinline__ void realization_bound(const Params& p, uint32_t p0, uint32_t nch,
                                                  uint32_t b, bool write, unsigned long long& vm,
                                                  uint32_t& bd, uint32_t& st_acc) {
  const uint32_t lane = threadIdx.x & 31u;
  vm = 0;
  bd = 0;
  int emax = INT32_MIN;
  if constexpr (sizeof(TS) == 4) {
    uint32_t v32 = 0;
    for (uint32_t k = lane; k < nch; k += 32) {
      const Part* q = p.parts + p0 + k;
      v32 = max(v32, (uint32_t)__ldcg(&q->vmax));
      bd |= __ldcg(&q->bad);
      emax = max(emax, __ldcg(&q->e));
    }
    vm = __reduce_max_sync(kFull, v32);
  } else {
    for (uint32_t k = lane; k < nch; k += 32) {
      const Part* q = p.parts + p0 + k;
      const unsigned long long x = __ldcg(&q->vmax);
      vm = x > vm ? x : vm;
      bd |= __ldcg(&q->bad);
    }
    vm = warp_max_u64(vm);
  }
  bd = __reduce_or_sync(kFull, bd);
  if (!write) return;
  double sum = 0.0;
  if (!bd) {
    if constexpr (sizeof(TS) == 4) {
      sum = fold_sum_f32(p.parts + p0, nch, __reduce_max_sync(kFull, emax) + 1);
    } else {
      if (lane == 0)
        for (uint32_t k = 0; k < nch; ++k)
          sum = __dadd_rn(sum, __longlong_as_double((long long)__ldcg(&p.parts[p0 + k].lo)));
    }
  }
  if (lane == 0) {
    double* o = p.bound_sum + 2 * (size_t)b;
    if (bd) {
      st_acc |= (bd & 1u) ? AR_STATUS_BAD_ALPHA : 0u;
      st_acc |= (bd & 2u) ? AR_STATUS_UNSUPPORTED : 0u;
      o[0] = o[1] = __longlong_as_double(0x7ff8000000000000ll);  // NaN: no selections
    } else {
      o[0] = sizeof(TS) == 4 ? (double)__uint_as_float((uint32_t)vm)
                             : __longlong_as_double((long long)vm);
      o[1] = sum;
      if (p.zero_status && vm == 0) st_acc |= AR_STATUS_ALL_ZERO;
    }
  }
}

// One warp per realization: bound, total and status from its chunk partials.
template <typename TS>
__global__ void __launch_bounds__(kBNT) k_batched_combine(const Params p) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t st_acc = 0;
  for (uint32_t b = blockIdx.x * kBWarps + (threadIdx.x >> 5); b < p.B;
       b += gridDim.x * kBWarps) {
    uint32_t p0 = b, nch = 1;
    if (p.rinfo) {
      p0 = p.rinfo[b].p0;
      nch = p.rinfo[b].nch;
    }
    unsigned long long vm;
    uint32_t bd;
    realization_bound<TS>(p, p0, nch, b, true, vm, bd, st_acc);
  }
  st_acc = __reduce_or_sync(kFull, st_acc);
  if (lane == 0 && st_acc) atomicOr(p.status, st_acc);
}

// ===========================================================================
// Selection kernel
// ===========================================================================
// The bound in the comparison's precision.
template <int CMP>
using BoundT = std::conditional_t<CMP == AR_CMP_F32, float, double>;
// The bound a warp's item carries: FP32, or FP64 with the FP32 pre-filter's
// precomputation.
template <int CMP>
using ItemBound = std::conditional_t<CMP == AR_CMP_F32, float, F64Bound>;
template <int CMP>
__device__ __forceinline__ ItemBound<CMP> item_bound(BoundT<CMP> T) {
  if constexpr (CMP == AR_CMP_F32) return T;
  else return f64_bound(T);
}

template <typename TS, int CMP>
struct WItem {  // the warp's current item (identical in every lane)
  uint32_t b = 0, s = 0, s1 = 0, M = 0;
  const TS* a = nullptr;
  int32_t* out = nullptr;
  ItemBound<CMP> T{};
};

// The FP32 comparison's operand alpha_j (FP64 data rounded to FP32).
template <typename TS>
__device__ __forceinline__ float load_alpha(const TS* a, uint32_t j) {
  if constexpr (sizeof(TS) == 4) return __ldg(a + j);
  else return __double2float_rn(__ldg(a + j));
}

// Selections are made in runs of kRun consecutive selection numbers.  Run g
// of realization b draws its trials n = 0, 1, 2, ... in order; trial
// n = 64 G + 32 h + i (h in {0, 1}, i < 32) takes words 2h and 2h + 1 of
// Philox block q = 32 G + i, counter (q mod 2^32, g, b, 256 floor(q / 2^32)).
// Decision r of the run is selection g kRun + r: the first accepted trial
// after decision r - 1 (the classical sequential AR loop), or the sentinel M
// once trial_cap trials in a row were rejected.
constexpr uint32_t kRun = 64;
constexpr uint32_t kUMax = 3;  // Philox blocks per lane per warp round, at most

// One warp round of U groups: lane l evaluates blocks 32 (G0 + u) + l
// (u < U), i.e. trials 64 (G0 + u) + 32 h + l; acc[2u + h] and j[2u + h] are
// that trial's test and candidate, A[u] / Bm[u] the warp's ballots of the
// h = 0 / h = 1 trials of group u.
template <typename TS, int CMP, int U, bool WIDE>
__device__ __forceinline__ void round_eval(const Params& p, unsigned long long q0, uint32_t g,
                                           uint32_t b, const WItem<TS, CMP>& w,
                                           uint32_t (&j)[2 * U], bool (&acc)[2 * U],
                                           uint32_t (&A)[U], uint32_t (&Bm)[U]) {
  uint4 v[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const unsigned long long q = q0 + 32u * (uint32_t)u;
    const uint32_t hi = WIDE ? (uint32_t)(q >> 32) << 8 : (uint32_t)(q0 >> 32) << 8;
    v[u] = philox10k(make_uint4((uint32_t)q, g, b, hi), p.keys);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    j[2 * u] = candidate(v[u].x, w.M);
    j[2 * u + 1] = candidate(v[u].z, w.M);
  }
  if constexpr (CMP == AR_CMP_F32) {
    float x[2 * U];
#pragma unroll
    for (int t = 0; t < 2 * U; ++t) x[t] = load_alpha<TS>(w.a, j[t]);
#pragma unroll
    for (int t = 0; t < 2 * U; ++t) {
      const uint32_t wu = (t & 1) ? v[t >> 1].w : v[t >> 1].y;
      acc[t] = accept_f32(wu, w.T, x[t]);
    }
  } else {
    // the FP64 test, decided in FP32 where the margins allow it
#pragma unroll
    for (int t = 0; t < 2 * U; ++t) {
      const uint32_t wu = (t & 1) ? v[t >> 1].w : v[t >> 1].y;
      acc[t] = accept_f64(wu, w.T, __ldg(w.a + j[t]));
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    A[u] = __ballot_sync(kFull, acc[2 * u]);
    Bm[u] = __ballot_sync(kFull, acc[2 * u + 1]);
  }
}

// Per-run state of a warp (identical in every lane).
struct RunState {
  uint32_t r;               // decisions made
  uint32_t skip, rend;      // the item takes decisions [skip, rend)
  uint32_t ncap;            // capped decisions in [skip, rend)
  unsigned long long n;     // next trial (a multiple of 64)
  unsigned long long since; // trials of decision r so far
  unsigned long long t0;    // first trial of decision skip
  bool done;
};

// A round in which no decision can reach the trial cap: decisions are the
// accepted trials in order.  Candidates go to the warp's staging buffer at
// their decision number (slot kRun for accepted trials past the run's end).
template <typename TS, int CMP, int U>
__device__ __forceinline__ void round_fast(const Params& p, uint32_t g, uint32_t b,
                                           const WItem<TS, CMP>& w, RunState& rs,
                                           int32_t* stage, SelCounters& cnt) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t j[2 * U], A[U], Bm[U];
  bool acc[2 * U];
  round_eval<TS, CMP, U, false>(p, (rs.n >> 1) + lane, g, b, w, j, acc, A, Bm);
  uint32_t c = rs.r, ra[2 * U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const uint32_t na = __popc(A[u]);
    ra[2 * u] = c + __popc(A[u] & lt);
    ra[2 * u + 1] = c + na + __popc(Bm[u] & lt);
    c += na + __popc(Bm[u]);
  }
#pragma unroll
  for (int t = 0; t < 2 * U; ++t)
    stage[(acc[t] && ra[t] < rs.rend) ? ra[t] : kRun] = (int32_t)j[t];
  if (c == rs.r) {
    rs.since += 64u * U;
    rs.n += 64u * U;
    return;
  }
  // the trial offset in this round of decision `want` (one lane holds it)
  auto offset_of = [&](uint32_t want) {
    uint32_t o = 0xffffffffu;
#pragma unroll
    for (int t = 0; t < 2 * U; ++t)
      if (acc[t] && ra[t] == want) o = 64u * (uint32_t)(t >> 1) + 32u * (uint32_t)(t & 1) + lane;
    return __reduce_min_sync(kFull, o);
  };
  if (rs.r < rs.skip && c >= rs.skip) rs.t0 = rs.n + offset_of(rs.skip - 1u) + 1ull;
  if (c >= rs.rend) {
    const uint32_t o = offset_of(rs.rend - 1u);
    if (lane == 0) cnt.trials += rs.n + o + 1ull - rs.t0;
    rs.done = true;
    return;
  }
  uint32_t last = 0;  // offset + 1 of the round's last acceptance
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (Bm[u]) last = 64u * (uint32_t)u + 32u + (32u - __clz(Bm[u]));
    else if (A[u]) last = 64u * (uint32_t)u + (32u - __clz(A[u]));
  }
  rs.since = 64u * U - last;
  rs.r = c;
  rs.n += 64u * U;
}

// A round taken decision by decision, in trial order (a decision may reach
// the trial cap, or the block index passes a multiple of 2^32).
template <typename TS, int CMP>
__device__ __forceinline__ void round_slow(const Params& p, uint32_t g, uint32_t b,
                                           const WItem<TS, CMP>& w, RunState& rs,
                                           int32_t* stage, SelCounters& cnt) {
  constexpr int U = 1;
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t j[2 * U], A[U], Bm[U];
  bool acc[2 * U];
  round_eval<TS, CMP, U, true>(p, (rs.n >> 1) + lane, g, b, w, j, acc, A, Bm);
#pragma unroll
  for (int u = 0; u < U; ++u) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t m = h ? Bm[u] : A[u];
#pragma unroll 1
      for (uint32_t L = 0; L < 32u; ++L) {
        const uint32_t jj = __shfl_sync(kFull, j[2 * u + h], L);
        if (rs.done) continue;
        const bool ok = ((m >> L) & 1u) != 0u;
        ++rs.since;
        if (!ok && rs.since != p.cap) continue;
        if (rs.r >= rs.skip) {
          if (lane == 0) stage[rs.r] = ok ? (int32_t)jj : (int32_t)w.M;
          if (!ok) ++rs.ncap;
        }
        ++rs.r;
        rs.since = 0;
        const unsigned long long t = rs.n + 64u * (uint32_t)u + 32u * (uint32_t)h + L;
        if (rs.r == rs.skip) rs.t0 = t + 1ull;
        if (rs.r == rs.rend) {
          rs.done = true;
          if (lane == 0) cnt.trials += t + 1ull - rs.t0;
        }
      }
    }
  }
  rs.n += 64u * U;
}

// Selections [w.s, w.s1) of the warp's item, run by run.  Each round takes
// 1 .. kUMax blocks per lane, as many as the run's remaining decisions are
// expected to need at the acceptance rate seen so far (the results do not
// depend on the choice).
template <typename TS, int CMP>
__device__ __forceinline__ void run_item(const Params& p, const WItem<TS, CMP>& w,
                                         int32_t* stage, SelCounters& cnt) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t bb = p.b_base + w.b;
  uint32_t k = w.s;
  while (k < w.s1) {
    const uint32_t S = p.sel_base + k;
    const uint32_t g = S / kRun;
    RunState rs;
    rs.skip = S % kRun;
    rs.rend = min(kRun, rs.skip + (w.s1 - k));
    rs.r = 0;
    rs.ncap = 0;
    rs.n = 0;
    rs.since = 0;
    rs.t0 = 0;
    rs.done = false;
    while (!rs.done) {
      const unsigned long long qb = rs.n >> 1;
      if (rs.since + 64u * kUMax < p.cap && (uint32_t)qb <= 0xffffffffu - 32u * kUMax) {
        // expected trials of the remaining decisions: 8 each before the
        // first acceptance, then n / r each
        const unsigned long long left = rs.rend - rs.r;
        const unsigned long long need = rs.r ? left * rs.n : left * 8u;
        const unsigned long long per = rs.r ? (unsigned long long)rs.r : 1ull;
        const uint32_t nu = need <= 64ull * per ? 1u : need <= 128ull * per ? 2u : 3u;
        if (nu == 1u) round_fast<TS, CMP, 1>(p, g, bb, w, rs, stage, cnt);
        else if (nu == 2u) round_fast<TS, CMP, 2>(p, g, bb, w, rs, stage, cnt);
        else round_fast<TS, CMP, 3>(p, g, bb, w, rs, stage, cnt);
      } else {
        round_slow<TS, CMP>(p, g, bb, w, rs, stage, cnt);
      }
    }
    __syncwarp();
    for (uint32_t r = rs.skip + lane; r < rs.rend; r += 32u) w.out[k + (r - rs.skip)] = stage[r];
    __syncwarp();
    if (lane == 0) {
      cnt.accepted += rs.rend - rs.skip - rs.ncap;
      cnt.capped += rs.ncap;
    }
    k += rs.rend - rs.skip;
  }
}

// Work claiming of one warp: the CTA's home list through a shared-memory
// counter, then the global queue, whose next ticket is claimed one item
// ahead so that the atomic's latency overlaps the current item.
struct Claimer {
  bool home = true;
  bool pref = false;  // lane 0: `ticket` holds an unused global ticket
  uint32_t ticket = 0;
};

// Claims the next selection item and gathers what the warp needs about it;
// returns false when no work is left.  Realizations whose bound is unusable
// get their indices set to M here and are skipped.
// Fused launch: how long a warp waits for the reduction of a realization its
// CTA is still reducing (it never waits in practice: every chunk of the
// realization was claimed before any of its selection ranges, by warps that
// reduce it without waiting).  Past the limit the realization's selections
// get the sentinel and AR_STATUS_WAIT_LIMIT is raised.
constexpr uint32_t kFusedWaitLimit = 1u << 22;
// the one-launch form keeps two 32-bit words per home realization of a CTA in
// dynamic shared memory (its reduced-chunk count and its maximum): up to
// 32 KB beside the kernel's 8 KB, under the 48 KB a launch gets without
// opting in; longer home lists take the two-launch form
constexpr uint32_t kMaxFusedSlots = 4096;

template <typename TS, int CMP, bool FUSED = false>
__device__ bool next_item(const Params& p, uint32_t* s_queue, uint32_t q_end, Claimer& cl,
                          WItem<TS, CMP>& w, uint32_t& st_acc, uint32_t* pre = nullptr,
                          const uint32_t* s_done = nullptr, const uint32_t* s_tmax = nullptr) {
  const uint32_t lane = threadIdx.x & 31u;
  for (;;) {
    uint32_t i = 0;
    bool ok = false;
    if (p.sitems && cl.home) {
      if (FUSED && *pre != 0xffffffffu) {  // the range the warp claimed when it left
        i = *pre;                          // the reduction phase
        *pre = 0xffffffffu;
      } else {
        if (lane == 0) i = atomicAdd(s_queue, 1u);
        i = __shfl_sync(kFull, i, 0);
      }
      ok = i < q_end;
      if (!ok) cl.home = false;
    }
    if (!ok) {
      const uint32_t qb = p.sitems ? p.gq0 : 0u, qe = p.sitems ? p.gq1 : p.B;
      if (lane == 0) {
        if (!cl.pref) cl.ticket = atomicAdd(&p.scratch->squeue, 1u);
        i = qb + cl.ticket;
        cl.pref = false;
        if (i < qe) {
          cl.ticket = atomicAdd(&p.scratch->squeue, 1u);
          cl.pref = true;
        }
      }
      i = __shfl_sync(kFull, i, 0);
      if (i >= qe) return false;
    }
    int64_t a0 = 0, o0 = 0;
    uint32_t M = 0, b = 0, s0 = 0, s1 = 0, p0 = 0, nch = 1, slot = 0;
    if (p.sitems) {
      const SItem& si = p.sitems[i];
      a0 = si.a0;
      o0 = si.o0;
      M = si.M;
      b = si.b;
      s0 = si.s0;
      s1 = si.s1;
      p0 = si.p0;
      nch = si.nch;
      slot = si.slot;
    } else {
      b = i;
      p0 = i;
      int64_t v = 0;
      if (lane < 2) v = __ldg(p.offsets + b + lane);
      else if (lane < 4) v = __ldg(p.out_offsets + b + lane - 2);
      a0 = __shfl_sync(kFull, v, 0);
      const int64_t a1 = __shfl_sync(kFull, v, 1);
      o0 = __shfl_sync(kFull, v, 2);
      const int64_t o1 = __shfl_sync(kFull, v, 3);
      M = (a1 < a0 || a1 - a0 >= (1ll << 31)) ? 0x7fffffffu : (uint32_t)(a1 - a0);
      s0 = 0;
      s1 = o1 > o0 ? (uint32_t)(o1 - o0) : 0u;
    }
    // the bound: from the chunk partials (the realization's first range also
    // writes {T, sum} and the status), or the caller's (NaN, < 0 or
    // infinite: BAD_BOUND); st = 1 marks an invalid realization, reported
    // once.  The chunk maxima are bit patterns of non-negative values, so
    // their checks need no FP64 operation (GB300's FP64 pipe is narrow).
    BoundT<CMP> Tc = 0;
    uint32_t st = 0;
    if constexpr (FUSED) {
      // wait until this CTA has reduced every chunk of the realization
      const volatile uint32_t* done = s_done + slot;
      uint32_t spins = 0;
      while (*done < nch && spins < kFusedWaitLimit) {
        __nanosleep(64);
        ++spins;
      }
      __syncwarp();
      // pairs with the reducing warp's CTA-scope fence (both warps are in this
      // CTA): its chunk partials, read below, are visible
      __threadfence_block();
      if (spins >= kFusedWaitLimit) {
        st_acc |= AR_STATUS_WAIT_LIMIT;
        int32_t* out = p.idx + o0;
        for (uint32_t k = s0 + lane; k < s1; k += 32) out[k] = (int32_t)M;
        continue;
      }
    }
    if (FUSED) {
      // fused: the maximum is in shared memory; the realization's first range
      // also combines the chunk partials into {T, sum} and the status
      if (s0 == 0) {
        unsigned long long vm;
        uint32_t bd;
        realization_bound<TS>(p, p0, nch, b, true, vm, bd, st_acc);
      }
      const uint32_t tb = s_tmax[slot];
      if (tb == 0xffffffffu) st = 1;
      else if (tb == 0u || M == 0) st = AR_STATUS_ALL_ZERO;
      else Tc = (BoundT<CMP>)__uint_as_float(tb);
    } else if (p.fold) {
      unsigned long long vm;
      uint32_t bd;
      realization_bound<TS>(p, p0, nch, b, s0 == 0, vm, bd, st_acc);
      if (bd) {
        st = 1;
      } else if (vm == 0 || M == 0) {
        st = AR_STATUS_ALL_ZERO;  // the paper's rejection case
      } else if constexpr (sizeof(TS) == 4) {
        Tc = (BoundT<CMP>)__uint_as_float((uint32_t)vm);
      } else {
        const double T = __longlong_as_double((long long)vm);
        if constexpr (CMP == AR_CMP_F32) {
          const float Tf = __double2float_rn(T);
          if (isinf(Tf)) st = AR_STATUS_BAD_BOUND;
          Tc = Tf;
        } else {
          Tc = T;
        }
      }
    } else {
      const double T = __ldcg(p.bound_in + (size_t)b * (size_t)p.bound_stride);
      const float Tf = __double2float_rn(T);
      if (p.bound_given && (!(T >= 0.0) || isinf(T))) st = AR_STATUS_BAD_BOUND;
      else if (T != T) st = 1;
      else if (CMP == AR_CMP_F32 && isinf(Tf)) st = AR_STATUS_BAD_BOUND;
      else if (T == 0.0 || M == 0) st = AR_STATUS_ALL_ZERO;  // the paper's rejection case
      if constexpr (CMP == AR_CMP_F32) Tc = Tf;
      else Tc = T;
    }
    int32_t* out = p.idx + o0;
    if (st) {
      // BAD_BOUND is reported for every realization it hits, ALL_ZERO only
      // for realizations with selections
      if (st == AR_STATUS_BAD_BOUND || (st == AR_STATUS_ALL_ZERO && s1 > s0)) st_acc |= st;
      for (uint32_t k = s0 + lane; k < s1; k += 32) out[k] = (int32_t)M;
      continue;
    }
    w.b = b;
    w.s = s0;
    w.s1 = s1;
    w.M = M;
    w.a = reinterpret_cast<const TS*>(p.alpha) + a0;
    w.out = out;
    w.T = item_bound<CMP>(Tc);
    return true;
  }
}

// FUSED: one launch for the whole call (FP32 data with a plan whose
// realizations all sit in CTA home lists).  Each CTA first reduces the chunks
// of its own home realizations (every warp claims chunks from a shared
// counter; a chunk's partial goes to global memory, then the realization's
// count of reduced chunks in shared memory is raised), then the warps go on
// to the selections exactly as in the two-launch call, taking a
// realization's bound once all its chunks are counted.  Chunks are claimed
// before any selection range, in home-list order, from the same counter.
template <typename TS, int CMP, int NW, bool FUSED = false>
__global__ void __launch_bounds__(NW * 32, kSelThreadsPerSm / (NW * 32))
    k_batched_select(const Params p) {
  __shared__ uint32_t s_queue;
  __shared__ int32_t s_stage[NW * (kRun + 1)];  // per warp: the current run's decisions
  extern __shared__ uint32_t s_done[];  // fused: reduced chunks per home realization
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t q_end = 0;
  uint32_t nred = 0, r0 = 0;
  uint32_t* s_tmax = s_done + p.nslots;  // fused: maximum per home realization
  if constexpr (FUSED) {
    r0 = p.frptr[blockIdx.x];
    nred = p.frptr[blockIdx.x + 1] - r0;
    for (uint32_t k = threadIdx.x; k < 2u * p.nslots; k += blockDim.x) s_done[k] = 0u;
  }
  if (p.sitems) {
    // fused: the counter starts nred below the first home range, so its
    // first nred values name chunks and the rest are home ranges
    if (threadIdx.x == 0) s_queue = p.scta[blockIdx.x] - nred;
    q_end = p.scta[blockIdx.x + 1];
  }
  __syncthreads();
  uint32_t pre = 0xffffffffu;
  if constexpr (FUSED) {
    const uint32_t base = p.scta[blockIdx.x] - nred;
    for (;;) {
      uint32_t i = 0;
      if (lane == 0) i = atomicAdd(&s_queue, 1u);
      i = __shfl_sync(kFull, i, 0);
      const uint32_t k = i - base;
      if (k >= nred) {
        pre = i;  // the warp's first selection range
        break;
      }
      const uint2 fr = p.fred[r0 + k];  // (chunk, slot)
      const Part part = reduce_chunk(p, fr.x);
      // the realization's maximum (bit pattern; all ones: an invalid value)
      if (lane == 0) atomicMax(s_tmax + fr.y, part.bad ? 0xffffffffu : (uint32_t)part.vmax);
      __syncwarp();
      __threadfence_block();  // the partial and the maximum are visible before the count
      if (lane == 0) atomicAdd(s_done + fr.y, 1u);
    }
  }
  SelCounters cnt;
  uint32_t st_acc = 0;
  WItem<TS, CMP> cur;
  Claimer cl;
  while (next_item<TS, CMP, FUSED>(p, &s_queue, q_end, cl, cur, st_acc, &pre, s_done, s_tmax))
    run_item<TS, CMP>(p, cur, s_stage + (threadIdx.x >> 5) * (kRun + 1), cnt);
  if (cnt.capped) st_acc |= AR_STATUS_TRIAL_CAP;
  flush_counters(cnt, p.stats);
  st_acc = __reduce_or_sync(kFull, st_acc);
  if (lane == 0 && st_acc) atomicOr(p.status, st_acc);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&p.scratch->sdone, 1u) == gridDim.x - 1u) {
      // every CTA has left the claim loop: return the queue to zero
      p.scratch->squeue = 0u;
      p.scratch->sdone = 0u;
      __threadfence();
    }
  }
}

// The reduction and combine kernels (bound_sum and status).
template <typename TS>
int launch_bound(const Params& p, bool stream_path, bool combine, cudaStream_t s) {
  const DeviceInfo& d = device_info();
  const uint32_t sms = (uint32_t)(d.sm_count > 0 ? d.sm_count : 1);
  const uint32_t nitems = p.ritems ? p.nr : p.B;
  const uint32_t need = (nitems + kBWarps - 1) / kBWarps;
  if (stream_path) {  // plan + 16-byte aligned FP32 data
    const uint32_t grid = std::max(1u, std::min(sms * (uint32_t)kBCtasPerSm, need));
    k_bound_reg<<<grid, kBNT, 0, s>>>(p);
  } else {
    const uint32_t grid = std::max(1u, std::min(sms * 8u, need));
    k_batched_bound<TS><<<grid, kBNT, 0, s>>>(p);
  }
  const int rc = check_launch();
  if (rc || !combine) return rc;
  const uint32_t cgrid = std::max(1u, std::min(sms * 8u, (p.B + kBWarps - 1) / kBWarps));
  k_batched_combine<TS><<<cgrid, kBNT, 0, s>>>(p);
  return check_launch();
}

// The selection kernel (bounds from p.bound_in) with tile shape `shape`.
template <typename TS, int CMP>
int launch_select(const Params& p, uint32_t sel_grid, int shape, cudaStream_t s) {
  const DeviceInfo& d = device_info();
  const uint32_t sms = (uint32_t)(d.sm_count > 0 ? d.sm_count : 1);
  const int nw = kSelShapes[shape];
  const uint32_t grid = sel_grid ? sel_grid : sms * (uint32_t)(kSelThreadsPerSm / (nw * 32));
  if (nw == 32) k_batched_select<TS, CMP, 32><<<grid, 32 * 32, 0, s>>>(p);
  else if (nw == 8) k_batched_select<TS, CMP, 8><<<grid, 8 * 32, 0, s>>>(p);
  else k_batched_select<TS, CMP, 16><<<grid, 16 * 32, 0, s>>>(p);
  return check_launch();
}

// The one-launch call (FP32 data, plan with every realization in a home list).
template <int CMP>
int launch_fused(const Params& p, uint32_t sel_grid, int shape, cudaStream_t s) {
  const int nw = kSelShapes[shape];
  const size_t smem = 2 * sizeof(uint32_t) * p.nslots;  // chunk counts and maxima
  if (nw == 32) k_batched_select<float, CMP, 32, true><<<sel_grid, 32 * 32, smem, s>>>(p);
  else if (nw == 8) k_batched_select<float, CMP, 8, true><<<sel_grid, 8 * 32, smem, s>>>(p);
  else k_batched_select<float, CMP, 16, true><<<sel_grid, 16 * 32, smem, s>>>(p);
  return check_launch();
}

}  // namespace
}  // namespace gbar

using namespace gbar;

// ---------------------------------------------------------------------------
// Plan: the work items of the kernels, built on the host from the offsets
// ---------------------------------------------------------------------------
struct ar_plan {
  int device;
  int64_t B;
  uint32_t nr, ns, grid, gq0;
  int shape;            // selection tile shape (index into kSelShapes)
  int gshare_pm;        // estimated cost left to the global queue, per mille
  int ctas_per_sm = 0;  // 0: as many CTAs per SM as the tile's registers allow
  uint32_t item_sel = kSItem;  // selections per home work item
  RItem* d_ritems;
  RInfo* d_rinfo;
  SItem* d_sitems;
  size_t sitems_cap;    // SItem capacity of d_sitems
  uint32_t* d_scta;
  size_t scta_cap;
  // one-launch (fused) form, when every realization sits in a home list: the
  // chunks each CTA reduces, (chunk, slot), and each CTA's range of them
  uint2* d_fred;
  uint32_t* d_frptr;
  uint32_t nslots;  // the longest home list, in realizations
  bool fused;
  unsigned char* d_scratch;  // Scratch | parts[NR]
  std::vector<int64_t> off, oo;  // host copies of the offsets (schedule rebuilds)
  std::vector<double> cost;
  std::vector<RInfo> rinfo;
};

namespace {

// The selection schedule for `grid` CTAs: realizations by decreasing
// estimated cost; the costliest go to the CTAs' home lists (longest
// processing time first onto the least loaded CTA) until the cost left is
// gshare of the total; the rest form the global queue in that order.
void build_selection(const ar_plan& pl, uint32_t grid, double gshare, std::vector<SItem>& sitems,
                     std::vector<uint32_t>& scta, uint32_t& gq0) {
  const int64_t B = pl.B;
  double total_cost = 0.0;
  for (double c : pl.cost) total_cost += c;
  std::vector<int64_t> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t x, int64_t y) { return pl.cost[x] > pl.cost[y]; });
  using Load = std::pair<double, uint32_t>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (uint32_t c = 0; c < grid; ++c) heap.push({0.0, c});
  std::vector<std::vector<int64_t>> lists(grid);
  double left = total_cost;
  size_t n_home = 0;
  for (; n_home < order.size() && left > gshare * total_cost; ++n_home) {
    const int64_t b = order[n_home];
    Load l = heap.top();
    heap.pop();
    lists[l.second].push_back(b);
    l.first += pl.cost[b];
    heap.push(l);
    left -= pl.cost[b];
  }
  sitems.clear();
  auto add_items = [&](int64_t b, uint32_t per) {
    const uint32_t K = (uint32_t)(pl.oo[b + 1] - pl.oo[b]);
    uint32_t s0 = 0;
    do {  // one item even when K = 0
      SItem s{};
      s.a0 = pl.off[b];
      s.o0 = pl.oo[b];
      s.M = (uint32_t)(pl.off[b + 1] - pl.off[b]);
      s.b = (uint32_t)b;
      s.s0 = s0;
      s.s1 = (uint32_t)std::min<uint64_t>(K, (uint64_t)s0 + per);
      s.p0 = pl.rinfo[b].p0;
      s.nch = pl.rinfo[b].nch;
      sitems.push_back(s);
      s0 = s.s1;
    } while (s0 < K);
  };
  scta.assign(grid + 1, 0);
  for (uint32_t c = 0; c < grid; ++c) {
    for (int64_t b : lists[c]) add_items(b, pl.item_sel);
    scta[c + 1] = (uint32_t)sitems.size();
  }
  gq0 = (uint32_t)sitems.size();
  for (size_t k = n_home; k < order.size(); ++k) add_items(order[k], kGItem);
}

// Rebuilds and uploads the plan's selection schedule for a tile shape and
// global-queue share (synchronous).
int set_schedule(ar_plan& pl, int shape, int gshare_pm) {
  const DeviceInfo& dev = device_info();
  // CTAs per SM: as many as fit (at least 1 for every shape), or fewer when
  // the caller runs several calls at once and wants them to share the SMs
  const int fit = kSelThreadsPerSm / (kSelShapes[shape] * 32);
  static_assert(kSelThreadsPerSm % (32 * 32) == 0, "every tile shape fits at least once per SM");
  const int per_sm = pl.ctas_per_sm > 0 ? std::min(pl.ctas_per_sm, fit) : fit;
  const uint32_t grid = (uint32_t)std::max(1, dev.sm_count) * (uint32_t)per_sm;
  std::vector<SItem> sitems;
  std::vector<uint32_t> scta;
  uint32_t gq0 = 0;
  build_selection(pl, grid, gshare_pm * 1e-3, sitems, scta, gq0);
  if (sitems.size() >= (1ull << 31)) return AR_ERR_ARG;
  cudaError_t e = cudaSuccess;
  if (sitems.size() > pl.sitems_cap) {
    cudaFree(pl.d_sitems);
    pl.d_sitems = nullptr;
    pl.sitems_cap = 0;
    e = cudaMalloc(&pl.d_sitems, sizeof(SItem) * sitems.size());
    if (e == cudaSuccess) pl.sitems_cap = sitems.size();
  }
  if (e == cudaSuccess && scta.size() > pl.scta_cap) {
    // room for the largest grid of any tile, so that the array is allocated
    // once and a launch captured with an earlier tile never reads freed memory
    const size_t cap = std::max(scta.size(), (size_t)std::max(1, dev.sm_count) *
                                                 (size_t)(kSelThreadsPerSm / (8 * 32)) + 1);
    cudaFree(pl.d_scta);
    pl.d_scta = nullptr;
    pl.scta_cap = 0;
    e = cudaMalloc(&pl.d_scta, sizeof(uint32_t) * cap);
    if (e == cudaSuccess) pl.scta_cap = cap;
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(pl.d_sitems, sitems.data(), sizeof(SItem) * sitems.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(pl.d_scta, scta.data(), sizeof(uint32_t) * scta.size(), cudaMemcpyHostToDevice);
  // the one-launch form: each CTA reduces the chunks of its own home
  // realizations (in home-list order) before selecting them
  const bool fused = gq0 == (uint32_t)sitems.size();
  uint32_t nslots = 0;
  if (e == cudaSuccess && fused) {
    std::vector<uint2> fred;
    std::vector<uint32_t> frptr(grid + 1, 0);
    fred.reserve(pl.nr);
    for (uint32_t c = 0; c < grid; ++c) {
      uint32_t slot = 0;
      for (uint32_t k = scta[c]; k < scta[c + 1]; ++k) {
        if (k > scta[c] && sitems[k].b != sitems[k - 1].b) ++slot;
        sitems[k].slot = slot;
        if (sitems[k].s0 == 0)
          for (uint32_t q = 0; q < sitems[k].nch; ++q) fred.push_back(make_uint2(sitems[k].p0 + q, slot));
      }
      if (scta[c + 1] > scta[c]) nslots = std::max(nslots, slot + 1);
      frptr[c + 1] = (uint32_t)fred.size();
    }
    if (!pl.d_fred) e = cudaMalloc(&pl.d_fred, sizeof(uint2) * std::max<size_t>(pl.nr, 1));
    if (e == cudaSuccess && !pl.d_frptr) e = cudaMalloc(&pl.d_frptr, sizeof(uint32_t) * pl.scta_cap);
    if (e == cudaSuccess && !fred.empty())
      e = cudaMemcpy(pl.d_fred, fred.data(), sizeof(uint2) * fred.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(pl.d_frptr, frptr.data(), sizeof(uint32_t) * frptr.size(),
                     cudaMemcpyHostToDevice);
    if (e == cudaSuccess)  // the slots were set after the first upload
      e = cudaMemcpy(pl.d_sitems, sitems.data(), sizeof(SItem) * sitems.size(),
                     cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return AR_ERR_CUDA;
  }
  // beyond kMaxFusedSlots home realizations per CTA the call takes two launches
  pl.fused = fused && nslots > 0 && nslots <= kMaxFusedSlots;
  pl.nslots = nslots;
  pl.ns = (uint32_t)sitems.size();
  pl.gq0 = gq0;
  pl.grid = grid;
  pl.shape = shape;
  pl.gshare_pm = gshare_pm;
  return AR_OK;
}

void free_plan(ar_plan* p) {
  cudaFree(p->d_ritems);
  cudaFree(p->d_rinfo);
  cudaFree(p->d_sitems);
  cudaFree(p->d_scta);
  cudaFree(p->d_fred);
  cudaFree(p->d_frptr);
  cudaFree(p->d_scratch);
  delete p;
}

}  // namespace

extern "C" int ar_plan_create(const int64_t* h_offsets, const int64_t* h_out_offsets, int64_t B,
                              ar_plan** out) {
  if (!out || B <= 0 || B >= (1ll << 31) || !h_offsets || !h_out_offsets) return AR_ERR_ARG;
  *out = nullptr;
  const DeviceInfo& dev = device_info();
  auto* p = new ar_plan();
  p->device = dev.device;
  p->B = B;
  p->off.assign(h_offsets, h_offsets + B + 1);
  p->oo.assign(h_out_offsets, h_out_offsets + B + 1);
  p->cost.resize(B);
  for (int64_t b = 0; b < B; ++b) {
    const int64_t M = h_offsets[b + 1] - h_offsets[b];
    const int64_t K = h_out_offsets[b + 1] - h_out_offsets[b];
    if (M < 0 || K < 0 || M >= (1ll << 31) || K >= (1ll << 32)) {
      delete p;
      return AR_ERR_ARG;
    }
    // selections whose expected trial count grows like log M for spread-out
    // propensities, plus the first touch of the realization's lines
    p->cost[b] =
        (double)K * (0.6 + std::log((double)std::max<int64_t>(M, 2))) + 0.05 * (double)M;
  }
  // reduction chunks: each realization cut into ceil(M / 1024) chunks of
  // equal length (a multiple of 4, so that only the realization's own ends
  // are unaligned), in order
  std::vector<RItem> ritems;
  std::vector<RInfo> rinfo(B);
  for (int64_t b = 0; b < B; ++b) {
    const int64_t a0 = h_offsets[b], a1 = h_offsets[b + 1];
    rinfo[b].p0 = (uint32_t)ritems.size();
    const int64_t nc = std::max<int64_t>(1, (a1 - a0 + kChunk - 1) / kChunk);
    const int64_t step = (((a1 - a0 + nc - 1) / nc) + 3) & ~int64_t(3);
    int64_t e = a0;
    do {
      const int64_t nxt = std::min(a1, e + step);
      RItem r{};
      r.e0 = e;
      r.n = (uint32_t)(nxt - e);
      ritems.push_back(r);
      e = nxt;
    } while (e < a1);
    rinfo[b].nch = (uint32_t)ritems.size() - rinfo[b].p0;
    if (ritems.size() >= (1ull << 31)) {
      delete p;
      return AR_ERR_ARG;
    }
  }
  p->nr = (uint32_t)ritems.size();
  p->rinfo = rinfo;
  const size_t scratch_bytes = sizeof(Scratch) + sizeof(Part) * ritems.size();
  cudaError_t e = cudaMalloc(&p->d_ritems, sizeof(RItem) * ritems.size());
  if (e == cudaSuccess) e = cudaMalloc(&p->d_rinfo, sizeof(RInfo) * rinfo.size());
  if (e == cudaSuccess) e = cudaMalloc(&p->d_scratch, scratch_bytes);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_ritems, ritems.data(), sizeof(RItem) * ritems.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_rinfo, rinfo.data(), sizeof(RInfo) * rinfo.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->d_scratch, 0, sizeof(Scratch));
  if (e != cudaSuccess) {
    set_cuda_error(e);
    free_plan(p);
    return AR_ERR_CUDA;
  }
  // default: 32 warps per CTA, every realization in a home list (the one-launch
  // form of ar_select_batched for FP32 data)
  const int rc = set_schedule(*p, 1, 0);
  if (rc) {
    free_plan(p);
    return rc;
  }
  *out = p;
  return AR_OK;
}

extern "C" void ar_plan_destroy(ar_plan* plan) {
  if (!plan) return;
  int cur = 0;
  cudaGetDevice(&cur);
  const int pd = plan->device;
  if (cur != pd) cudaSetDevice(pd);
  free_plan(plan);
  if (cur != pd) cudaSetDevice(cur);
}

extern "C" size_t ar_select_batched_workspace_size(int64_t B) {
  if (B < 0 || B >= (1ll << 31)) return 0;
  return sizeof(Scratch) + sizeof(Part) * (size_t)B;
}

namespace {

// Argument checks and Params common to the batched entry points.
int batched_params(const void* d_alpha_cat, int dtype, const int64_t* d_offsets,
                   const int64_t* d_out_offsets, int64_t B, const ar_plan* plan,
                   uint32_t* d_status, void* d_work, size_t work_bytes, Params& p,
                   uint32_t& sel_grid, int& shape, bool& stream_path) {
  if (!valid_dtype(dtype) || B < 0 || B >= (1ll << 31)) return AR_ERR_ARG;
  if (!d_alpha_cat || !d_offsets || !d_status) return AR_ERR_ARG;
  if (!aligned(d_alpha_cat, dtype_size(dtype)) || !aligned(d_offsets, 8) ||
      !aligned(d_out_offsets, 8) || !aligned(d_status, 4))
    return AR_ERR_ALIGN;
  p = Params{};
  sel_grid = 0;
  shape = 0;
  stream_path = false;
  p.vec_ok = aligned(d_alpha_cat, 16) ? 1u : 0u;
  if (plan) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (plan->B != B || plan->device != dev) return AR_ERR_ARG;
    p.ritems = plan->d_ritems;
    p.rinfo = plan->d_rinfo;
    p.sitems = plan->d_sitems;
    p.scta = plan->d_scta;
    p.nr = plan->nr;
    p.gq0 = plan->gq0;
    p.gq1 = plan->ns;
    p.scratch = reinterpret_cast<Scratch*>(plan->d_scratch);
    p.parts = reinterpret_cast<Part*>(plan->d_scratch + sizeof(Scratch));
    sel_grid = plan->grid;
    shape = plan->shape;
    stream_path = dtype == AR_F32 && p.vec_ok;
    if (plan->fused) {
      p.fred = plan->d_fred;
      p.frptr = plan->d_frptr;
      p.nslots = plan->nslots;
    }
  } else {
    if (!d_work || work_bytes < ar_select_batched_workspace_size(B)) return AR_ERR_WORKSPACE;
    if (!aligned(d_work, 16)) return AR_ERR_ALIGN;
    p.scratch = static_cast<Scratch*>(d_work);
    p.parts = reinterpret_cast<Part*>(static_cast<unsigned char*>(d_work) + sizeof(Scratch));
  }
  p.alpha = static_cast<const unsigned char*>(d_alpha_cat);
  p.offsets = d_offsets;
  p.out_offsets = d_out_offsets;
  p.status = d_status;
  p.B = (uint32_t)B;
  return AR_OK;
}

int selection_params(uint64_t seed, uint64_t sel_offset, uint32_t realization_base, int cmp,
                     uint64_t trial_cap, int64_t B, const int64_t* d_out_offsets, int32_t* d_idx,
                     ar_stats* d_stats, Params& p) {
  if (!valid_cmp(cmp) || trial_cap < 1 || trial_cap > (1ull << 32)) return AR_ERR_ARG;
  if ((uint64_t)realization_base + (uint64_t)B > (1ull << 32)) return AR_ERR_ARG;
  if (sel_offset >= (1ull << 32)) return AR_ERR_ARG;
  if (!d_out_offsets || !d_idx) return AR_ERR_ARG;
  if (!aligned(d_idx, 4) || !aligned(d_stats, 8)) return AR_ERR_ALIGN;
  p.idx = d_idx;
  p.stats = d_stats;
  p.cap = trial_cap;
  p.sel_base = (uint32_t)sel_offset;
  p.b_base = realization_base;
  p.keys = philox_keys(seed);
  return AR_OK;
}

int dispatch_select(int dtype, int cmp, const Params& p, uint32_t sel_grid, int shape,
                    cudaStream_t s) {
  if (dtype == AR_F32)
    return cmp == AR_CMP_F32 ? launch_select<float, AR_CMP_F32>(p, sel_grid, shape, s)
                             : launch_select<float, AR_CMP_F64>(p, sel_grid, shape, s);
  return cmp == AR_CMP_F32 ? launch_select<double, AR_CMP_F32>(p, sel_grid, shape, s)
                           : launch_select<double, AR_CMP_F64>(p, sel_grid, shape, s);
}

}  // namespace

extern "C" int ar_bound_batched(const void* d_alpha_cat, int dtype, const int64_t* d_offsets,
                                int64_t B, const ar_plan* plan, double* d_bound_sum,
                                uint32_t* d_status, void* d_work, size_t work_bytes,
                                void* stream) {
  if (B == 0 && valid_dtype(dtype)) return AR_OK;
  Params p;
  uint32_t sel_grid;
  int shape;
  bool stream_path;
  int rc = batched_params(d_alpha_cat, dtype, d_offsets, d_offsets, B, plan, d_status, d_work,
                          work_bytes, p, sel_grid, shape, stream_path);
  if (rc) return rc;
  if (!d_bound_sum) return AR_ERR_ARG;
  if (!aligned(d_bound_sum, 8)) return AR_ERR_ALIGN;
  p.bound_sum = d_bound_sum;
  p.zero_status = 1u;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return dtype == AR_F32 ? launch_bound<float>(p, stream_path, true, s)
                         : launch_bound<double>(p, stream_path, true, s);
}

extern "C" int ar_select_batched_bounded(const void* d_alpha_cat, int dtype,
                                         const int64_t* d_offsets, const int64_t* d_out_offsets,
                                         int64_t B, const double* d_bound, int64_t bound_stride,
                                         uint64_t seed, uint64_t sel_offset,
                                         uint32_t realization_base, int cmp, uint64_t trial_cap,
                                         const ar_plan* plan, int32_t* d_idx, ar_stats* d_stats,
                                         uint32_t* d_status, void* d_work, size_t work_bytes,
                                         void* stream) {
  if (B == 0 && valid_dtype(dtype) && valid_cmp(cmp)) return AR_OK;
  Params p;
  uint32_t sel_grid;
  int shape;
  bool stream_path;
  int rc = batched_params(d_alpha_cat, dtype, d_offsets, d_out_offsets, B, plan, d_status,
                          d_work, work_bytes, p, sel_grid, shape, stream_path);
  if (rc) return rc;
  rc = selection_params(seed, sel_offset, realization_base, cmp, trial_cap, B, d_out_offsets,
                        d_idx, d_stats, p);
  if (rc) return rc;
  if (!d_bound || bound_stride < 1) return AR_ERR_ARG;
  if (!aligned(d_bound, 8)) return AR_ERR_ALIGN;
  p.bound_in = d_bound;
  p.bound_stride = bound_stride;
  p.bound_given = 1u;
  return dispatch_select(dtype, cmp, p, sel_grid, shape, static_cast<cudaStream_t>(stream));
}

extern "C" int ar_select_batched(const void* d_alpha_cat, int dtype, const int64_t* d_offsets,
                                 const int64_t* d_out_offsets, int64_t B, uint64_t seed,
                                 uint64_t sel_offset, uint32_t realization_base, int cmp,
                                 uint64_t trial_cap, const ar_plan* plan, double* d_bound_sum,
                                 int32_t* d_idx, ar_stats* d_stats, uint32_t* d_status,
                                 void* d_work, size_t work_bytes, void* stream) {
  if (B == 0 && valid_dtype(dtype) && valid_cmp(cmp)) return AR_OK;
  Params p;
  uint32_t sel_grid;
  int shape;
  bool stream_path;
  int rc = batched_params(d_alpha_cat, dtype, d_offsets, d_out_offsets, B, plan, d_status,
                          d_work, work_bytes, p, sel_grid, shape, stream_path);
  if (rc) return rc;
  rc = selection_params(seed, sel_offset, realization_base, cmp, trial_cap, B, d_out_offsets,
                        d_idx, d_stats, p);
  if (rc) return rc;
  if (!d_bound_sum) return AR_ERR_ARG;
  if (!aligned(d_bound_sum, 8)) return AR_ERR_ALIGN;
  p.bound_sum = d_bound_sum;
  p.fold = 1u;  // the selection kernel combines the chunk partials itself
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (stream_path && p.fred) {  // one launch: each CTA reduces its own realizations
    return cmp == AR_CMP_F32 ? launch_fused<AR_CMP_F32>(p, sel_grid, shape, s)
                             : launch_fused<AR_CMP_F64>(p, sel_grid, shape, s);
  }
  rc = dtype == AR_F32 ? launch_bound<float>(p, stream_path, false, s)
                       : launch_bound<double>(p, stream_path, false, s);
  if (rc) return rc;
  return dispatch_select(dtype, cmp, p, sel_grid, shape, s);
}

extern "C" int ar_plan_set_tile(ar_plan* plan, int warps_per_cta, int global_share_pm) {
  if (!plan || global_share_pm < 0 || global_share_pm > 1000) return AR_ERR_ARG;
  int shape = -1;
  for (int k = 0; k < 3; ++k)
    if (kSelShapes[k] == warps_per_cta) shape = k;
  if (shape < 0) return AR_ERR_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != plan->device) return AR_ERR_ARG;
  return set_schedule(*plan, shape, global_share_pm);
}

extern "C" int ar_plan_set_grid(ar_plan* plan, int ctas_per_sm, int selections_per_item) {
  if (!plan || ctas_per_sm < 0 || ctas_per_sm > kSelThreadsPerSm / (8 * 32)) return AR_ERR_ARG;
  if (selections_per_item < 0 || selections_per_item > 1024 || selections_per_item % 64)
    return AR_ERR_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != plan->device) return AR_ERR_ARG;
  const int old = plan->ctas_per_sm;
  const uint32_t old_item = plan->item_sel;
  plan->ctas_per_sm = ctas_per_sm;
  plan->item_sel = selections_per_item ? (uint32_t)selections_per_item : kSItem;
  const int rc = set_schedule(*plan, plan->shape, plan->gshare_pm);
  if (rc != AR_OK) {
    plan->ctas_per_sm = old;
    plan->item_sel = old_item;
  }
  return rc;
}

extern "C" int ar_plan_autotune(ar_plan* plan, const void* d_alpha_cat, int dtype,
                                const int64_t* d_offsets, const int64_t* d_out_offsets,
                                uint64_t seed, int cmp, double* d_bound_sum, int32_t* d_idx,
                                ar_stats* d_stats, uint32_t* d_status, int reps,
                                int32_t* h_choice, void* stream) {
  if (!plan || reps < 1 || reps > 10000) return AR_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int shares[3] = {0, 300, 600};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    set_cuda_error(ce);
    return AR_ERR_CUDA;
  }
  int best_shape = plan->shape, best_share = plan->gshare_pm, rc = AR_OK;
  float best_ms = 0.f;
  bool have = false;
  for (int sh = 0; sh < 3 && rc == AR_OK; ++sh) {
    for (int g = 0; g < 3 && rc == AR_OK; ++g) {
      rc = set_schedule(*plan, sh, shares[g]);
      if (rc) break;
      auto call = [&]() {
        return ar_select_batched(d_alpha_cat, dtype, d_offsets, d_out_offsets, plan->B, seed, 0,
                                 0, cmp, 1ull << 20, plan, d_bound_sum, d_idx, d_stats, d_status,
                                 nullptr, 0, stream);
      };
      for (int w = 0; w < 2 && rc == AR_OK; ++w) rc = call();
      if (rc) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && rc == AR_OK; ++r) rc = call();
      cudaEventRecord(e1, s);
      ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) {
        set_cuda_error(ce);
        rc = AR_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (!have || ms < best_ms) {
        have = true;
        best_ms = ms;
        best_shape = sh;
        best_share = shares[g];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int rc2 = set_schedule(*plan, best_shape, best_share);
  if (rc == AR_OK) rc = rc2;
  if (rc == AR_OK && h_choice) {
    h_choice[0] = kSelShapes[best_shape];
    h_choice[1] = best_share;
    h_choice[2] = (int32_t)(best_ms * 1e6f / (float)reps);  // ns per call
  }
  return rc;
}
