// The two comparators of the paper's method, on the GPU:
//
//   ar_select_paper  the paper's own GPU rule (Sections "Election step" and
//       "Selection step"; the Results' pseudo-code): every reaction j draws
//       u_j in [0, T), is eligible when u_j < D_j (D_j != 0) with rate
//       R_j = u_j / D_j, and the selection is argmin R (lowest j on ties), or
//       the rejection sentinel M when no rate is below 1.  FP32 throughout,
//       as the paper's arrays are float.  The paper runs one block of M
//       threads per selection; here a warp takes a selection at a time, each
//       lane two reactions per Philox block, and the argmin is two warp
//       min-reductions (rate, then index).
//   ar_select_it  the direct method's inverse transform (Section "The
//       Stochastic Simulation Algorithm"): j is the smallest index whose
//       running sum exceeds u alpha_0.  The running sums are the sequential
//       FP64 sums in index order, computed once per call by one thread (the
//       dependence the paper argues against), then every selection is a
//       binary search.
#include <algorithm>

#include "device.cuh"
#include "host.hpp"

namespace gbar {
namespace {

constexpr int kPW = 8;  // warps per CTA (paper rule)
constexpr int kPNT = kPW * 32;

struct PaperParams {
  const float* D;
  uint32_t M;
  const double* bound;
  uint32_t K;
  uint32_t sel_base, b;
  uint32_t k0, k1;
  int32_t* idx;
  unsigned long long* rejections;
};

// order-preserving key of an FP32 value (-0 taken as +0)
__device__ __forceinline__ uint32_t fkey(float x) {
  const uint32_t u = __float_as_uint(__fadd_rn(x, 0.0f));
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <bool SMEM>
__global__ void __launch_bounds__(kPNT) k_paper(const PaperParams p) {
  extern __shared__ float s_D[];
  const uint32_t lane = threadIdx.x & 31u;
  const float* D = p.D;
  if constexpr (SMEM) {
    for (uint32_t j = threadIdx.x; j < p.M; j += kPNT) s_D[j] = p.D[j];
    __syncthreads();
    D = s_D;
  }
  const float T = __double2float_rn(*p.bound);
  const uint32_t npairs = (p.M + 1u) >> 1;
  const uint32_t one_key = fkey(1.0f);
  unsigned long long rej = 0;
  for (uint32_t s = blockIdx.x * kPW + (threadIdx.x >> 5); s < p.K; s += gridDim.x * kPW) {
    uint32_t best = 0xffffffffu, arg = 0xffffffffu;  // (key of R, j)
    for (uint32_t c = lane; c < npairs; c += 32) {
      const uint4 w = philox10(make_uint4(c, p.sel_base + s, p.b, 3u), p.k0, p.k1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t j = 2u * c + (uint32_t)h;
        if (j >= p.M) break;
        const uint32_t wb = h ? w.w : w.y;
        const float uT = __fmul_rn(__fmul_rn(__uint2float_rn(wb >> 8), 0x1p-24f), T);
        const float d = D[j];
        float R = __int_as_float(0x7f800000);  // ineligible: +inf
        if (uT < d && d != 0.0f) R = __fdiv_rn(uT, d);
        const uint32_t k = fkey(R);
        if (k < best) {  // j ascends within a lane: the first minimum is kept
          best = k;
          arg = j;
        }
      }
    }
    const uint32_t kmin = __reduce_min_sync(kFull, best);
    const uint32_t jmin = __reduce_min_sync(kFull, best == kmin ? arg : 0xffffffffu);
    if (lane == 0) {
      const bool ok = p.M > 0 && kmin < one_key;  // min R < 1
      p.idx[s] = ok ? (int32_t)jmin : (int32_t)p.M;
      if (!ok) ++rej;
    }
  }
  if (lane == 0 && rej && p.rejections) atomicAdd(p.rejections, rej);
}

// ---- inverse transform ------------------------------------------------------
// The running sums S_j of the direct method are the exact prefix sums rounded
// once to FP64 (each propensity a whole number of units U, rounded down:
// FP32 data U = 2^(E - 223), FP64 data U = 2^(E - 1119), E the biased
// exponent of the maximum, at least 1 resp. 97), accumulated in 128-bit
// integers.  Integer sums do not depend on the order of the additions, so a
// parallel scan gives the sums a sequential loop gives:
//   k_it_max      maximum, validity and last nonzero index (atomics into the
//                 header, which the call clears first);
//   k_it_tiles    the exact sum of each tile of kItTile propensities;
//   k_it_offsets  one CTA: exclusive scan of the tile sums, alpha_0 = S_{M-1}
//                 and the status;
//   k_it_prefix   per tile: the exact running sums, each rounded once;
//   k_it_select   per selection: bisection for the first S_j > u alpha_0.
constexpr int kItThreads = 256;
constexpr int kItPer = 16;                       // propensities per thread and tile
constexpr int64_t kItTile = kItThreads * kItPer;  // 4096
constexpr int kItScanThreads = 1024;

struct ItHeader {
  unsigned long long skey;     // max over (bits with the sign bit flipped): signed maximum
  unsigned long long umax;     // max over raw bits
  unsigned long long last1;    // last index with a positive propensity, plus one
  double a0;                   // S_{M-1}
  uint32_t status;
  uint32_t pad[3];
};
static_assert(sizeof(ItHeader) % 16 == 0, "header keeps the sums 16-byte aligned");

template <typename TS>
struct ItBits;
template <>
struct ItBits<float> {
  using U = uint32_t;
  static constexpr unsigned long long kSign = 0x80000000ull, kInf = 0x7f800000ull;
};
template <>
struct ItBits<double> {
  using U = unsigned long long;
  static constexpr unsigned long long kSign = 0x8000000000000000ull,
                                      kInf = 0x7ff0000000000000ull;
};

template <typename TS>
__device__ __forceinline__ unsigned long long it_bits(const TS* a, int64_t j) {
  if constexpr (sizeof(TS) == 4) return (unsigned long long)__float_as_uint(__ldg(a + j));
  else return (unsigned long long)__double_as_longlong(__ldg(a + j));
}

// Header -> (invalid?, exponent of the unit, is the maximum zero?)
template <typename TS>
__device__ __forceinline__ bool it_unit(const ItHeader* h, int& uexp, bool* zero = nullptr) {
  using B = ItBits<TS>;
  const unsigned long long smax = h->skey ^ B::kSign;  // back to the signed maximum's bits
  const bool neg_or_zero = (h->skey & B::kSign) == 0;  // signed maximum < 0
  const bool bad = (!neg_or_zero && smax >= B::kInf) || h->umax > B::kSign;
  const unsigned long long vmax = neg_or_zero ? 0ull : smax;
  if (zero) *zero = vmax == 0;
  if constexpr (sizeof(TS) == 4) {
    const int E = max((int)(vmax >> 23), 1);
    uexp = E - 223;
  } else {
    const int E = max((int)(vmax >> 52), 97);
    uexp = E - 1119;
  }
  return bad;
}

// One propensity (bit pattern, valid) in units of 2^uexp, rounded down.
template <typename TS>
__device__ __forceinline__ U128 it_units(unsigned long long bits, int uexp) {
  unsigned long long m;
  int q;
  if constexpr (sizeof(TS) == 4) {
    const int e = (int)((bits >> 23) & 0xffu);
    m = bits & 0x7fffffull;
    if (e) m |= 0x800000ull;
    q = (e ? e : 1) - 150;
  } else {
    const int e = (int)((bits >> 52) & 0x7ffu);
    m = bits & 0xfffffffffffffull;
    if (e) m |= 0x10000000000000ull;
    q = (e ? e : 1) - 1075;
  }
  const int sh = q - uexp;
  U128 r;
  if (sh >= 64) {
    r.hi = m << (sh - 64);
  } else if (sh >= 0) {
    r = shl128(m, sh);
  } else if (sh > -64) {
    r.lo = m >> (-sh);
  }
  return r;
}

template <typename TS>
__global__ void __launch_bounds__(kItThreads) k_it_max(const TS* __restrict__ a, int64_t M,
                                                      ItHeader* h) {
  using B = ItBits<TS>;
  unsigned long long skey = 0, umax = 0, last1 = 0;
  for (int64_t j = (int64_t)blockIdx.x * kItThreads + threadIdx.x; j < M;
       j += (int64_t)gridDim.x * kItThreads) {
    const unsigned long long bits = it_bits(a, j);
    skey = max(skey, bits ^ B::kSign);
    umax = max(umax, bits);
    if (bits != 0 && bits < B::kSign) last1 = (unsigned long long)j + 1;  // positive (or NaN)
  }
  skey = warp_max_u64(skey);
  umax = warp_max_u64(umax);
  last1 = warp_max_u64(last1);
  if ((threadIdx.x & 31u) == 0) {
    atomicMax(&h->skey, skey);
    atomicMax(&h->umax, umax);
    atomicMax(&h->last1, last1);
  }
}

// Block-wide inclusive scan of one U128 per thread; returns the inclusive
// prefix and sets `total` (in every thread).  `sm` holds kItThreads / 32 U128.
__device__ __forceinline__ U128 block_scan128(U128 x, U128* sm, U128& total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    U128 y;
    y.hi = __shfl_up_sync(kFull, x.hi, o);
    y.lo = __shfl_up_sync(kFull, x.lo, o);
    if (lane >= (uint32_t)o) x = add128(x, y);
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  U128 off, tot;
  for (uint32_t w = 0; w < blockDim.x / 32u; ++w) {
    if (w < warp) off = add128(off, sm[w]);
    tot = add128(tot, sm[w]);
  }
  __syncthreads();
  total = tot;
  return add128(x, off);
}

template <typename TS>
__global__ void __launch_bounds__(kItThreads) k_it_tiles(const TS* __restrict__ a, int64_t M,
                                                        const ItHeader* h, U128* tsum) {
  __shared__ U128 sm[kItThreads / 32];
  int uexp;
  const bool bad = it_unit<TS>(h, uexp);
  const int64_t t0 = (int64_t)blockIdx.x * kItTile;
  U128 acc;
  if (!bad) {
#pragma unroll 4
    for (int k = 0; k < kItPer; ++k) {
      const int64_t j = t0 + (int64_t)k * kItThreads + threadIdx.x;
      if (j < M) acc = add128(acc, it_units<TS>(it_bits(a, j), uexp));
    }
  }
  acc = warp_sum128(acc);
  if ((threadIdx.x & 31u) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    U128 t;
    for (int w = 0; w < kItThreads / 32; ++w) t = add128(t, sm[w]);
    tsum[blockIdx.x] = t;
  }
}

// One CTA: tsum[t] <- the exact sum of the tiles before t; alpha_0 and the
// status into the header.
template <typename TS>
__global__ void __launch_bounds__(kItScanThreads) k_it_offsets(U128* tsum, int64_t T,
                                                              ItHeader* h, uint32_t* d_status) {
  __shared__ U128 sm[kItScanThreads / 32];
  int uexp;
  bool zero;
  const bool bad = it_unit<TS>(h, uexp, &zero);
  const int64_t per = (T + kItScanThreads - 1) / kItScanThreads;
  const int64_t b0 = min(T, (int64_t)threadIdx.x * per), b1 = min(T, b0 + per);
  U128 mine;
  for (int64_t t = b0; t < b1; ++t) mine = add128(mine, tsum[t]);
  U128 total;
  const U128 incl = block_scan128(mine, sm, total);
  U128 run;  // exclusive prefix of this thread's first tile
  run.lo = incl.lo - mine.lo;
  run.hi = incl.hi - mine.hi - (incl.lo < mine.lo ? 1ull : 0ull);
  for (int64_t t = b0; t < b1; ++t) {
    const U128 x = tsum[t];
    tsum[t] = run;
    run = add128(run, x);
  }
  if (threadIdx.x == 0) {
    uint32_t st = 0;
    double a0 = 0.0;
    if (bad) {
      st = AR_STATUS_BAD_ALPHA;
    } else {
      a0 = u128_to_double(total, uexp);  // 0 also when every term is below the unit
      if (zero) st = AR_STATUS_ALL_ZERO;
    }
    h->a0 = a0;
    h->status = st;
    if (st) atomicOr(d_status, st);
  }
}

template <typename TS>
__global__ void __launch_bounds__(kItThreads) k_it_prefix(const TS* __restrict__ a, int64_t M,
                                                         const ItHeader* h, const U128* toff,
                                                         double* __restrict__ S) {
  __shared__ U128 sm[kItThreads / 32];
  int uexp;
  if (it_unit<TS>(h, uexp)) return;  // the whole grid takes the same branch
  const int64_t t0 = (int64_t)blockIdx.x * kItTile;
  U128 run = toff[blockIdx.x];
  for (int k = 0; k < kItPer; ++k) {
    const int64_t j = t0 + (int64_t)k * kItThreads + threadIdx.x;
    if (t0 + (int64_t)k * kItThreads >= M) break;  // uniform over the block
    U128 x;
    if (j < M) x = it_units<TS>(it_bits(a, j), uexp);
    U128 total;
    const U128 incl = block_scan128(x, sm, total);
    if (j < M) S[j] = u128_to_double(add128(run, incl), uexp);
    run = add128(run, total);
  }
}

struct ItParams {
  const ItHeader* hdr;
  const double* c;
  int64_t M;
  uint32_t K;
  uint32_t sel_base, b;
  uint32_t k0, k1;
  int32_t* idx;
};

__global__ void __launch_bounds__(256) k_it_select(const ItParams p) {
  const double a0 = p.hdr->a0;
  const int64_t last = (int64_t)p.hdr->last1 - 1;
  const bool ok = p.hdr->status == 0 && a0 > 0.0;  // else the sentinel M
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < p.K; s += gridDim.x * blockDim.x) {
    if (!ok) {
      p.idx[s] = (int32_t)p.M;
      continue;
    }
    const uint4 w = philox10(make_uint4(0u, p.sel_base + s, p.b, 2u), p.k0, p.k1);
    const unsigned long long m = ((unsigned long long)w.x << 21) | (unsigned long long)(w.y >> 11);
    const double target = __dmul_rn(__ull2double_rn(m) * 0x1p-53, a0);
    // the running sums are non-decreasing: first S_j > target by bisection
    int64_t lo = 0, hi = p.M;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (__ldg(p.c + mid) > target) hi = mid;
      else lo = mid + 1;
    }
    p.idx[s] = (int32_t)(lo < p.M ? lo : last);
  }
}

}  // namespace
}  // namespace gbar

using namespace gbar;

extern "C" int ar_select_paper(const float* d_D, int64_t M, const double* d_bound, int64_t K,
                               uint64_t seed, uint64_t sel_offset, uint32_t realization,
                               int32_t* d_idx, unsigned long long* d_rejections, void* stream) {
  if (M < 0 || M >= (1ll << 31) || K < 0 || sel_offset + (uint64_t)K > (1ull << 32))
    return AR_ERR_ARG;
  if (K == 0) return AR_OK;
  if ((M > 0 && !d_D) || !d_bound || !d_idx) return AR_ERR_ARG;
  if (!aligned(d_D, 4) || !aligned(d_bound, 8) || !aligned(d_idx, 4) || !aligned(d_rejections, 8))
    return AR_ERR_ALIGN;
  const DeviceInfo& dev = device_info();
  PaperParams p{};
  p.D = d_D;
  p.M = (uint32_t)M;
  p.bound = d_bound;
  p.K = (uint32_t)K;
  p.sel_base = (uint32_t)sel_offset;
  p.b = realization;
  p.k0 = (uint32_t)(seed & 0xffffffffu);
  p.k1 = (uint32_t)(seed >> 32);
  p.idx = d_idx;
  p.rejections = d_rejections;
  const uint32_t sms = (uint32_t)std::max(1, dev.sm_count);
  const uint32_t need = (uint32_t)((K + kPW - 1) / kPW);
  const size_t smem = (size_t)M * sizeof(float);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (smem <= 48 * 1024) {
    const uint32_t grid = std::max(1u, std::min(need, sms * 8u));
    k_paper<true><<<grid, kPNT, smem, s>>>(p);
  } else {
    const uint32_t grid = std::max(1u, std::min(need, sms * 8u));
    k_paper<false><<<grid, kPNT, 0, s>>>(p);
  }
  return check_launch();
}

namespace {
inline int64_t it_tiles(int64_t M) { return std::max<int64_t>(1, (M + kItTile - 1) / kItTile); }
inline size_t it_sums_bytes(int64_t M) {
  return (sizeof(double) * (size_t)std::max<int64_t>(M, 1) + 15) & ~size_t(15);
}
}  // namespace

extern "C" size_t ar_select_it_workspace_size(int64_t M) {
  if (M < 0) return 0;
  return sizeof(ItHeader) + it_sums_bytes(M) + sizeof(U128) * (size_t)it_tiles(M);
}

extern "C" int ar_select_it(const void* d_alpha, int dtype, int64_t M, int64_t K, uint64_t seed,
                            uint64_t sel_offset, uint32_t realization, int32_t* d_idx,
                            uint32_t* d_status, void* d_work, size_t work_bytes, void* stream) {
  if (!valid_dtype(dtype) || M < 0 || M >= (1ll << 31) || K < 0 ||
      sel_offset + (uint64_t)K > (1ull << 32))
    return AR_ERR_ARG;
  if ((M > 0 && !d_alpha) || !d_status || (K > 0 && !d_idx)) return AR_ERR_ARG;
  if (!d_work || work_bytes < ar_select_it_workspace_size(M)) return AR_ERR_WORKSPACE;
  if (!aligned(d_alpha, dtype_size(dtype)) || !aligned(d_idx, 4) || !aligned(d_status, 4) ||
      !aligned(d_work, 16))
    return AR_ERR_ALIGN;
  unsigned char* w = static_cast<unsigned char*>(d_work);
  auto* hdr = reinterpret_cast<ItHeader*>(w);
  double* c = reinterpret_cast<double*>(w + sizeof(ItHeader));
  U128* tsum = reinterpret_cast<U128*>(w + sizeof(ItHeader) + it_sums_bytes(M));
  const int64_t T = it_tiles(M);
  const DeviceInfo& dev = device_info();
  const uint32_t sms = (uint32_t)std::max(1, dev.sm_count);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(ItHeader), s);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return AR_ERR_CUDA;
  }
  const uint32_t mgrid = (uint32_t)std::max<int64_t>(
      1, std::min<int64_t>((M + kItThreads - 1) / kItThreads, (int64_t)sms * 8));
  if (dtype == AR_F32) {
    const float* a = static_cast<const float*>(d_alpha);
    k_it_max<float><<<mgrid, kItThreads, 0, s>>>(a, M, hdr);
    k_it_tiles<float><<<(uint32_t)T, kItThreads, 0, s>>>(a, M, hdr, tsum);
    k_it_offsets<float><<<1, kItScanThreads, 0, s>>>(tsum, T, hdr, d_status);
    k_it_prefix<float><<<(uint32_t)T, kItThreads, 0, s>>>(a, M, hdr, tsum, c);
  } else {
    const double* a = static_cast<const double*>(d_alpha);
    k_it_max<double><<<mgrid, kItThreads, 0, s>>>(a, M, hdr);
    k_it_tiles<double><<<(uint32_t)T, kItThreads, 0, s>>>(a, M, hdr, tsum);
    k_it_offsets<double><<<1, kItScanThreads, 0, s>>>(tsum, T, hdr, d_status);
    k_it_prefix<double><<<(uint32_t)T, kItThreads, 0, s>>>(a, M, hdr, tsum, c);
  }
  int rc = check_launch();
  if (rc || K == 0) return rc;
  ItParams p{};
  p.hdr = hdr;
  p.c = c;
  p.M = M;
  p.K = (uint32_t)K;
  p.sel_base = (uint32_t)sel_offset;
  p.b = realization;
  p.k0 = (uint32_t)(seed & 0xffffffffu);
  p.k1 = (uint32_t)(seed >> 32);
  p.idx = d_idx;
  const uint32_t grid =
      std::max(1u, std::min((uint32_t)((K + 255) / 256), sms * 8u));
  k_it_select<<<grid, 256, 0, s>>>(p);
  return check_launch();
}
